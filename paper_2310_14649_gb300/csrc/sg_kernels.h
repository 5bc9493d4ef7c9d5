// Launch wrappers shared between the translation units of libsg.
#pragma once

#include <functional>

#include "sg_solver.h"

namespace sg {

// AMG level work buffers ([P][ld_l] blocks per level).
template <typename T>
struct AmgWork {
  std::vector<T*> b, x, t;
};

template <typename T>
sg_status spmm(const DevCsr& A, const T* X, int64_t ldx, const T* B, int64_t ldb, T* Y, int64_t ldy, int P,
               int op, cudaStream_t st);
// prof (may be NULL): times the local-solve launch as kind 4 (FP32) / 5 (FP64)
template <typename T>
sg_status ras_apply(const Precond& pc, int64_t n, int P, const T* R, int64_t ld, T* Z, cudaStream_t st,
                    bool transform, Profiler* prof = nullptr);
template <typename T>
// in place Z <- M Z per node; with Z2, also into slot *j2 of the array Z2
// (slot stride stride2, the same leading dimension)
sg_status node_transform(T* Z, int64_t ld, int64_t n, int P, const T* M, cudaStream_t st, T* Z2 = nullptr,
                         int64_t stride2 = 0, const int* j2 = nullptr);
// RAS local solves by explicit local inverses on tcgen05 (sg_ras_tc.cu):
// built at setup for ras_kernel 2 (FP32 data; P <= 96), applied with the
// Kronecker factor M fused when transform
bool ras_inverse_supported(int P);
sg_status ras_inverse_build(sg_problem* pr, Precond& pc, cudaStream_t st);
sg_status ras_inverse_apply(const Precond& pc, int P, const float* R, int64_t ld, float* Z, const float* M,
                            bool transform, int wait_limit, cudaStream_t st);
sg_status ras_inverse_check(const Precond& pc, cudaStream_t st);
template <typename T>
sg_status amg_vcycle(const AmgHier& H, AmgWork<T>& w, int P, cudaStream_t st, T* out = nullptr, int64_t ldo = 0);
sg_status frobenius_weights(sg_problem* pr, std::vector<double>& w);
// sets the dynamic shared-memory limits of the library's kernels once per
// process (before any graph capture)
sg_status kernel_attrs_init();

// ---- vector kernels (sg_krylov.cu) ----
// grid of the fused multi-vector reductions and the vectors per pass; the
// reduction scratch holds kMdotBlocks x kMdotMaxVectors doubles + a counter
constexpr int kMdotBlocks = 2 * 152;
constexpr int kMdotMaxVectors = 32;
// Device-resident scalar state of one (F)GMRES cycle.
struct GmresState {
  double* H;      // (m+1) x m, column-major; upper triangle R after rotations
  double* cs;     // m
  double* sn;     // m
  double* g;      // m+1
  double* y;      // m
  double* hsum;   // 2 (m+1): Gram-Schmidt coefficients of pass 1 and pass 2 (zero with one pass)
  double* scal;   // [0] norm^2 of w, [1] h_{j+1,j}, [2] estimate |g_{j+1}|, [3] beta, [4] flags
};

template <typename T>
sg_status vec_norm2(const T* x, int64_t len, double* out, double* partial, unsigned* counter, cudaStream_t st);
template <typename T>
sg_status vec_mdot(const T* V, int64_t stride, int nv, const T* w, int64_t len, double* out, double* partial,
                   unsigned* counter, cudaStream_t st);
template <typename T>
sg_status vec_maxpy_mdot(const T* V, int64_t stride, int nv, const double* h, T* w, int64_t len, double* out,
                         double* partial, unsigned* counter, cudaStream_t st);
template <typename T>
sg_status vec_maxpy_norm(const T* V, int64_t stride, int nv, const double* h, T* w, int64_t len, double* out,
                         double* partial, unsigned* counter, cudaStream_t st);
// y = x * (1 / *den) (den on the device; sqrt taken when take_sqrt)
template <typename T>
sg_status vec_scale_by(const T* x, T* y, int64_t len, const double* den, bool take_sqrt, cudaStream_t st);
// x += sum_i coef[i] * V_i
template <typename T>
sg_status vec_axpy_multi(const T* V, int64_t stride, int nv, const double* coef, T* x, int64_t len,
                         cudaStream_t st);
// y = x (with type conversion) and y = alpha * x
template <typename Ti, typename To>
sg_status vec_convert(const Ti* x, To* y, int64_t len, const double* scale_num, const double* scale_den,
                      cudaStream_t st);
// x64 += s * double(d)   (s on the device)
sg_status vec_add_scaled_f32(double* x, const float* d, int64_t len, const double* s, cudaStream_t st);
sg_status gmres_init(GmresState s, int m, const double* beta, cudaStream_t st);

// Device-driven GMRES state: iv[0] j, iv[1] iterations of this solve,
// iv[2] iteration cap, iv[3] stop flag, iv[4] iterations summed over
// solves, iv[5] breakdown flag, iv[6] restart cycles summed over solves;
// dtol[0] absolute tolerance.
struct DevGmres {
  int* iv;
  double* dtol;
};
template <typename T>
sg_status dg_mdot(const T* V, int64_t stride, const T* w, int64_t len, double* out, double* partial, unsigned* counter,
                  const int* jdev, int nv_max, cudaStream_t st);
template <typename T>
sg_status dg_axpy_norm(const T* V, int64_t stride, const double* h, T* w, int64_t len, double* out, double* partial,
                       unsigned* counter, const int* jdev, cudaStream_t st);
template <typename T>
sg_status dg_axpy_multi(const T* V, int64_t stride, const double* coef, T* x, int64_t len, const int* kdev,
                        cudaStream_t st);
template <typename T>
// V_{j+1} = w / h (device j after the Givens step); with dst, also the
// first n rows of every mode into dst (leading dimension ldd; V's is lds)
sg_status dg_scale_next(const T* w, T* V, int64_t stride, int64_t len, DevGmres d, const double* hn, cudaStream_t st,
                        T* dst = nullptr, int64_t ldd = 0, int64_t lds = 0, int64_t n = 0);
template <typename T>
sg_status dg_copy_vj(const T* V, int64_t stride, int64_t lds, T* dst, int64_t ldd, int64_t n, int P, DevGmres d,
                     cudaStream_t st);
// rr2, nf2 (device, may be NULL): squared FP64 residual and right-hand-side
// norms of the enclosing refinement step; with them the tolerance is
// max(rtol, min(0.5, 0.5 target / (||r|| / ||F||)))
sg_status dg_init(DevGmres d, const double* rnorm2, double rtol, cudaGraphConditionalHandle outer, cudaStream_t st,
                  const double* rr2 = nullptr, const double* nf2 = nullptr, double target = 0.0);
sg_status dg_start(DevGmres d, GmresState s, int m, const double* beta2, cudaGraphConditionalHandle inner,
                   cudaStream_t st);
sg_status dg_givens(DevGmres d, GmresState s, int m, cudaGraphConditionalHandle inner, cudaStream_t st);
sg_status dg_end(DevGmres d, GmresState s, cudaGraphConditionalHandle outer, cudaStream_t st, bool trust = true);
// V_j = src for the device index j = d.iv[0]
template <typename T>
sg_status dg_store_j(const T* src, T* V, int64_t stride, int64_t len, DevGmres d, cudaStream_t st);
// refinement loop control of a graph-captured mixed-precision solve
sg_status ir_decide(const double* rr, const double* nf2, int* iv, double rtol, int max_ir, const int* its_total,
                    int max_it, cudaGraphConditionalHandle h, cudaStream_t st);
sg_status dg_backsolve(DevGmres d, GmresState s, int m, cudaStream_t st);
sg_status gmres_givens(GmresState s, int m, int j, double* host_est, cudaStream_t st);
sg_status gmres_backsolve(GmresState s, int m, int k, cudaStream_t st);

}  // namespace sg
