// Newton's method for the nonlinear stochastic Poisson problem
//     -div( k(x, xi) (1 + u^2) grad u ) = 1,   u = 0 on the boundary,
// (Sec. 2.2, Eqs. NLP_StrongPDE, stonlp_system, vectorvalPDENL, AjkTkl,
// with the conductivity (1 + u^2) in place of the paper's (1 + alpha u)).
//
// Discretisation: inside element e the solution enters the conductivity
// through its element average ubar_e, whose square is projected onto the
// output chaos by the triple products,
//     w_{e,f} = sum_{a,b} ubar_{e,a} ubar_{e,b} <psi_a psi_b psi_f>,
// so the element Galerkin matrix is sum_i cbar_i(e) <psi_i psi_l psi_m> +
// sum_{i,f} cbar_i(e) w_{e,f} <psi_i psi_f psi_l psi_m>.  Linearising the
// fourfold product through the chaos, <psi_i psi_f psi_l psi_m> =
// sum_j <psi_i psi_f psi_j> <psi_j psi_l psi_m> (j of degree <= 2p, inside
// the input set when q >= 2p), makes that matrix sum_j ctil_j(e) G_j with
//     ctil_j(e) = cbar_j(e) + sum_{i,f} cbar_i(e) w_{e,f} <psi_i psi_f psi_j>:
// the nonlinear operator A(U) has the linear problem's Kronecker form with
// per-element coefficients ctil(U), so it is assembled into five-slot ELL
// values and applied by the same kernels as the linear operator.  The
// Jacobian adds the derivative through w: J(U) dU = A(U) dU + A(dctil) U with
//     dctil_j = sum_{i,f} cbar_i dw_f <psi_i psi_f psi_j>,
//     dw_f = 2 sum_{a,b} ubar_a dubar_b <psi_a psi_b psi_f>.
// Each Newton step solves J dU = F - A(U) U by flexible GMRES with the
// linear problem's two-level preconditioner (FP32 inside the FP64 Newton
// residual for mode 1), and stops on the relative update ||dU|| / ||U||.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "sg_ctx.h"
#include "sg_stencil.h"

namespace sg {

struct NewtonWork {
  int P = 0, K = 0;
  int64_t E = 0;
  DevBuf cbar64, cbar32;             // [K][E] lognormal input coefficients
  DevBuf coef64, dcoef64, dcoef32;   // [K][E]: ctil(U); dctil of a Jacobian apply
  Ell op;                            // A(U): values of sum_j A(ctil_j) (FP64 and FP32)
  Ell dop;                           // A(dctil), the Jacobian's derivative part
  DevBuf ppp_off, ppp_ab, ppp_m64, ppp_m32;  // <psi_a psi_b psi_f> by rows f
  DevBuf kfj_off, kfj_kf, kfj_m64, kfj_m32;  // <psi_k psi_f psi_j> by rows j (k | f << 16)
  DevBuf u64, u32, f64, r64, r32, d32, d64, tmp32, tmp64, one, scal;
  double* host = nullptr;            // pinned scalars
  ~NewtonWork() {
    if (host) cudaFreeHost(host);
  }
};

void newton_free(sg_problem* pr) {
  delete pr->nl;
  pr->nl = nullptr;
}

namespace {

constexpr int kNlElems = 32;   // elements per CTA, one per lane
constexpr int kNlWarps = 8;

// interior index of grid node (x, y), -1 on the boundary
__device__ inline int64_t node_index(int x, int y, int N) {
  return (x >= 1 && x <= N - 1 && y >= 1 && y <= N - 1) ? int64_t(y - 1) * (N - 1) + (x - 1) : -1;
}

// Per element block: the element averages of U (and dU), the projected
// square w = Pi_p[ubar^2] (or its derivative dw = 2 Pi_p[ubar dubar]), and
// out_j = base_j + sum_{(i,f)} <psi_i psi_f psi_j> cbar_i w_f for j < K.
// Lane = element, warps stride over modes and output rows.
template <typename T>
__global__ void __launch_bounds__(kNlElems* kNlWarps)
    k_nl_coef(int N, int64_t E, int P, int K, const T* __restrict__ U, int64_t ldu, const T* __restrict__ dU,
              int64_t lddu, const T* __restrict__ cbar, const T* __restrict__ base, const int* __restrict__ ppp_off,
              const int2* __restrict__ ppp_ab, const T* __restrict__ ppp_m, const int* __restrict__ kfj_off,
              const int* __restrict__ kfj_kf, const T* __restrict__ kfj_m, T* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sU = reinterpret_cast<T*>(smem_raw);   // [P][32]
  T* sD = sU + P * kNlElems;                // [P][32]
  T* sW = sD + P * kNlElems;                // [P][32]
  T* sC = sW + P * kNlElems;                // [K][32]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t e = int64_t(blockIdx.x) * kNlElems + lane;
  const bool valid = e < E;
  int64_t v[3] = {-1, -1, -1};
  if (valid) {
    const int64_t cell = e >> 1;
    const int i = int(cell % N), j = int(cell / N);
    if ((e & 1) == 0) {  // lower triangle (i,j), (i+1,j), (i+1,j+1)
      v[0] = node_index(i, j, N);
      v[1] = node_index(i + 1, j, N);
      v[2] = node_index(i + 1, j + 1, N);
    } else {             // upper triangle (i,j), (i+1,j+1), (i,j+1)
      v[0] = node_index(i, j, N);
      v[1] = node_index(i + 1, j + 1, N);
      v[2] = node_index(i, j + 1, N);
    }
  }
  const T third = T(1) / T(3);
  for (int a = warp; a < P; a += kNlWarps) {
    T s = 0, sd = 0;
    for (int q = 0; q < 3; ++q) {
      if (v[q] < 0) continue;
      s += U[int64_t(a) * ldu + v[q]];
      if (dU) sd += dU[int64_t(a) * lddu + v[q]];
    }
    sU[a * kNlElems + lane] = s * third;
    sD[a * kNlElems + lane] = sd * third;
  }
  for (int k = warp; k < K; k += kNlWarps) sC[k * kNlElems + lane] = valid ? cbar[int64_t(k) * E + e] : T(0);
  __syncthreads();
  const T* sB = dU ? sD : sU;
  for (int f = warp; f < P; f += kNlWarps) {
    T acc = 0;
    for (int t = ppp_off[f]; t < ppp_off[f + 1]; ++t) {
      const int2 ab = ppp_ab[t];
      acc += ppp_m[t] * sU[ab.x * kNlElems + lane] * sB[ab.y * kNlElems + lane];
    }
    sW[f * kNlElems + lane] = dU ? T(2) * acc : acc;
  }
  __syncthreads();
  for (int j = warp; j < K; j += kNlWarps) {
    T acc = (base && valid) ? base[int64_t(j) * E + e] : T(0);
    for (int t = kfj_off[j]; t < kfj_off[j + 1]; ++t) {
      const int kf = kfj_kf[t];
      acc += kfj_m[t] * sC[(kf & 0xffff) * kNlElems + lane] * sW[(kf >> 16) * kNlElems + lane];
    }
    if (valid) out[int64_t(j) * E + e] = acc;
  }
}

// Five-slot ELL values of sum_j A(coef_j) from per-element coefficients
// [K][E]; thread per (term, row).  v64 and v32 may be NULL.
template <typename Tc>
__global__ void k_nl_ell(const Tc* __restrict__ coef, int N, int64_t n, int64_t ldr, int K, double* __restrict__ v64,
                         float* __restrict__ v32) {
  const int m = N - 1;
  const int64_t E = 2LL * N * N;
  const int64_t total = int64_t(K) * n;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
    const int k = int(t / n);
    const int64_t r = t - int64_t(k) * n;
    const int i = int(r % m) + 1, j = int(r / m) + 1;
    Tc v[5];
    p1_stencil<Tc>(coef + int64_t(k) * E, N, i, j, v);
    for (int s = 0; s < 5; ++s) {
      const int64_t idx = (int64_t(k) * 5 + s) * ldr + r;
      if (v64) v64[idx] = double(v[s]);
      if (v32) v32[idx] = float(v[s]);
    }
  }
}

__global__ void k_to_f32(const double* __restrict__ x, float* __restrict__ y, int64_t len) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < len; e += int64_t(gridDim.x) * blockDim.x)
    y[e] = float(x[e]);
}

unsigned grid_len(int64_t len) { return unsigned(std::min<int64_t>((len + 255) / 256, 152 * 16)); }

size_t coef_smem(int P, int K, size_t elem) { return size_t(3 * P + K) * kNlElems * elem; }

sg_status attrs_once() {
  static bool done = false;
  if (done) return SG_OK;
  SG_CUDA(cudaFuncSetAttribute(k_nl_coef<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  SG_CUDA(cudaFuncSetAttribute(k_nl_coef<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  done = true;
  return SG_OK;
}

template <typename T> const T* sel(const DevBuf& b64, const DevBuf& b32);
template <> const double* sel<double>(const DevBuf& b64, const DevBuf&) { return dp<double>(b64); }
template <> const float* sel<float>(const DevBuf&, const DevBuf& b32) { return dp<float>(b32); }

sg_status upload(DevBuf& d, const void* src, size_t bytes) {
  SG_TRY(d.alloc(std::max<size_t>(bytes, 16)));
  if (bytes) SG_CUDA(cudaMemcpy(d.ptr, src, bytes, cudaMemcpyHostToDevice));
  return SG_OK;
}

sg_status ell_like(const Ell& src, Ell& dst, bool v64, bool v32, int K) {
  dst.S = src.S;
  dst.n = src.n;
  dst.ldr = src.ldr;
  SG_TRY(dst.col.alloc(src.col.bytes));
  SG_CUDA(cudaMemcpy(dst.col.ptr, src.col.ptr, src.col.bytes, cudaMemcpyDeviceToDevice));
  if (v64) SG_TRY(dst.v64.alloc(size_t(K) * src.S * src.ldr * 8));
  if (v32) SG_TRY(dst.v32.alloc(size_t(K) * src.S * src.ldr * 4));
  return SG_OK;
}

// Triple lists, coefficients and operator storage of the nonlinear problem
// (built on first use).
sg_status newton_prepare(sg_problem* pr) {
  if (pr->nl) return SG_OK;
  const int P = pr->P, K = pr->K, L = pr->L;
  SG_ARG(pr->q >= 2 * pr->p,
         "the nonlinear problem needs an input order q_in >= 2 p_out (the fourfold products go through the input set)");
  SG_ARG(K < 65536 && P < 32768, "the nonlinear problem supports K < 65536 and P < 32768");
  if (coef_smem(P, K, 8) > 227 * 1024) {
    set_error("the nonlinear problem's coefficient kernel needs (3 P + K) x 256 bytes of shared memory <= 227 KB");
    return SG_ERR_UNSUPPORTED;
  }
  SG_TRY(attrs_once());
  std::unique_ptr<NewtonWork> w(new NewtonWork());
  w->P = P;
  w->K = K;
  w->E = pr->E;
  // <psi_a psi_b psi_f>, a, b, f < P: the triples (k, a, b) with k < P (the
  // output set is the leading part of the input set), rows by f = k
  std::vector<int> poff(P + 1, 0);
  std::vector<int2> pab;
  std::vector<double> pm;
  for (int64_t t = 0; t < pr->T; ++t) {
    const int k = pr->kab[3 * t];
    if (k >= P) break;
    pab.push_back(make_int2(pr->kab[3 * t + 1], pr->kab[3 * t + 2]));
    pm.push_back(pr->g[t]);
    poff[k + 1] = int(pab.size());
  }
  for (int f = 1; f <= P; ++f) poff[f] = std::max(poff[f], poff[f - 1]);
  // <psi_k psi_f psi_j>, k, j < K, f < P, by rows j (ascending k, f)
  std::vector<int> koff(K + 1, 0), kkf;
  std::vector<double> km;
  std::vector<double> isf(K);
  for (int k = 0; k < K; ++k) {
    double fct = 1.0;
    for (int i = 0; i < L; ++i)
      for (int v = 2; v <= pr->mi_in[size_t(k) * L + i]; ++v) fct *= v;
    isf[k] = 1.0 / std::sqrt(fct);
  }
  // 1D integers <He_a He_b He_c>, a, c <= q, b <= p
  const int q = pr->q, p = pr->p;
  std::vector<double> t1(size_t(q + 1) * (p + 1) * (q + 1));
  for (int a = 0; a <= q; ++a)
    for (int b = 0; b <= p; ++b)
      for (int c = 0; c <= q; ++c) t1[(size_t(a) * (p + 1) + b) * (q + 1) + c] = double(he_triple_1d(a, b, c));
  for (int j = 0; j < K; ++j) {
    const int32_t* aj = &pr->mi_in[size_t(j) * L];
    for (int k = 0; k < K; ++k) {
      const int32_t* ak = &pr->mi_in[size_t(k) * L];
      for (int f = 0; f < P; ++f) {
        const int32_t* af = &pr->mi_in[size_t(f) * L];
        double num = 1.0;
        for (int i = 0; i < L && num != 0.0; ++i) num *= t1[(size_t(ak[i]) * (p + 1) + af[i]) * (q + 1) + aj[i]];
        if (num == 0.0) continue;
        kkf.push_back(k | (f << 16));
        km.push_back(num * isf[k] * isf[f] * isf[j]);
      }
    }
    koff[j + 1] = int(kkf.size());
  }
  auto f32 = [](const std::vector<double>& v) {
    std::vector<float> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) o[i] = float(v[i]);
    return o;
  };
  SG_TRY(upload(w->ppp_off, poff.data(), poff.size() * 4));
  SG_TRY(upload(w->ppp_ab, pab.data(), pab.size() * sizeof(int2)));
  SG_TRY(upload(w->ppp_m64, pm.data(), pm.size() * 8));
  std::vector<float> pm32 = f32(pm);
  SG_TRY(upload(w->ppp_m32, pm32.data(), pm32.size() * 4));
  SG_TRY(upload(w->kfj_off, koff.data(), koff.size() * 4));
  SG_TRY(upload(w->kfj_kf, kkf.data(), kkf.size() * 4));
  SG_TRY(upload(w->kfj_m64, km.data(), km.size() * 8));
  std::vector<float> km32 = f32(km);
  SG_TRY(upload(w->kfj_m32, km32.data(), km32.size() * 4));
  // lognormal coefficients of every input term at every element
  const int64_t E = pr->E, KE = int64_t(K) * E;
  SG_TRY(w->cbar64.alloc(size_t(KE) * 8));
  SG_TRY(w->cbar32.alloc(size_t(KE) * 4));
  SG_TRY(element_coefficients(pr, 0, K, dp<double>(w->cbar64), nullptr));
  k_to_f32<<<grid_len(KE), 256>>>(dp<double>(w->cbar64), dp<float>(w->cbar32), KE);
  note_launch();
  SG_CUDA(cudaGetLastError());
  SG_TRY(w->coef64.alloc(size_t(KE) * 8));
  SG_TRY(w->dcoef32.alloc(size_t(KE) * 4));
  SG_TRY(ell_like(pr->fine, w->op, true, true, K));
  SG_TRY(ell_like(pr->fine, w->dop, false, true, K));
  const size_t len = size_t(P) * pr->ld;
  for (DevBuf* b : {&w->u64, &w->f64, &w->r64, &w->d64, &w->tmp64}) SG_TRY(b->alloc(len * 8));
  for (DevBuf* b : {&w->u32, &w->r32, &w->d32, &w->tmp32}) SG_TRY(b->alloc(len * 4));
  SG_TRY(w->scal.alloc(16 * 8));
  {
    const double one = 1.0;
    SG_TRY(upload(w->one, &one, 8));
  }
  SG_CUDA(cudaHostAlloc(&w->host, 16 * sizeof(double), cudaHostAllocDefault));
  SG_CUDA(cudaDeviceSynchronize());
  pr->nl = w.release();
  return SG_OK;
}

// out = (base ? base : 0) + sum_{(i,f)} <psi_i psi_f psi_j> cbar_i w_f, with w
// the projected square of U's element averages (dU NULL) or its derivative
// along dU
template <typename T>
sg_status nl_coef(sg_problem* pr, const T* U, const T* dU, const T* base, T* out, cudaStream_t st) {
  NewtonWork& w = *pr->nl;
  const unsigned grid = unsigned((w.E + kNlElems - 1) / kNlElems);
  k_nl_coef<T><<<grid, kNlElems * kNlWarps, coef_smem(w.P, w.K, sizeof(T)), st>>>(
      pr->N, w.E, w.P, w.K, U, pr->ld, dU, pr->ld, sel<T>(w.cbar64, w.cbar32), base, dp<int>(w.ppp_off),
      dp<int2>(w.ppp_ab), sel<T>(w.ppp_m64, w.ppp_m32), dp<int>(w.kfj_off), dp<int>(w.kfj_kf),
      sel<T>(w.kfj_m64, w.kfj_m32), out);
  note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

template <typename Tc>
sg_status nl_ell(sg_problem* pr, const Tc* coef, Ell& A, cudaStream_t st) {
  const int64_t total = int64_t(pr->K) * pr->n;
  k_nl_ell<Tc><<<grid_len(total), 256, 0, st>>>(coef, pr->N, pr->n, A.ldr, pr->K, dp<double>(A.v64),
                                                 dp<float>(A.v32));
  note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

// Y = F - A X (F given) or A X with the values of A (same pattern and
// triples as the linear operator)
template <typename T>
sg_status nl_apply(sg_problem* pr, const Ell& A, const T* X, const T* F, T* Y, cudaStream_t st) {
  const int64_t ld = pr->ld;
  // the fine FP32 family may be generated for the edge-flux storage, which
  // these per-step value arrays do not have: the shared-memory kernel then
  if (pr->apply_mode != 1 && jit_eligible(pr) && !(sizeof(T) == 4 && pr->flux_on))
    return jit_apply_launch(pr, sizeof(T) == 8 ? 2 : 0, A, X, ld, F, ld, Y, ld, st);
  return apply_ell<T>(A, pr->tri, pr->P, pr->K, X, ld, F, ld, Y, ld, st);
}

// operator at U (FP64 iterate): ctil(U) and the ELL values of A(U)
sg_status nl_operator(sg_problem* pr, const double* U64, cudaStream_t st) {
  NewtonWork& w = *pr->nl;
  SG_TRY(nl_coef<double>(pr, U64, nullptr, dp<double>(w.cbar64), dp<double>(w.coef64), st));
  return nl_ell<double>(pr, dp<double>(w.coef64), w.op, st);
}

// Y = J(U) X = A(U) X + A(dctil(U; X)) U, with A(U) already in w.op and U
// in the precision T (ld = pr->ld)
template <typename T>
sg_status nl_jacobian(sg_problem* pr, const T* U, const T* X, T* Y, cudaStream_t st) {
  NewtonWork& w = *pr->nl;
  const int64_t len = int64_t(pr->P) * pr->ld;
  T* dcoef = sizeof(T) == 8 ? reinterpret_cast<T*>(w.dcoef64.ptr) : reinterpret_cast<T*>(w.dcoef32.ptr);
  T* tmp = sizeof(T) == 8 ? reinterpret_cast<T*>(w.tmp64.ptr) : reinterpret_cast<T*>(w.tmp32.ptr);
  SG_TRY(nl_coef<T>(pr, U, X, nullptr, dcoef, st));
  SG_TRY(nl_ell<T>(pr, dcoef, w.dop, st));
  SG_TRY(nl_apply<T>(pr, w.op, X, nullptr, Y, st));
  SG_TRY(nl_apply<T>(pr, w.dop, U, nullptr, tmp, st));
  return vec_axpy_multi<T>(tmp, 0, 1, dp<double>(w.one), Y, len, st);
}

sg_status ensure_fp64_jacobian(sg_problem* pr) {
  NewtonWork& w = *pr->nl;
  if (!w.dcoef64.ptr) SG_TRY(w.dcoef64.alloc(size_t(w.K) * w.E * 8));
  if (!w.dop.v64.ptr) SG_TRY(w.dop.v64.alloc(size_t(w.K) * w.dop.S * w.dop.ldr * 8));
  return SG_OK;
}

// a caller block (n rows, leading dimension ldx) into an internal one (pr->ld, padding zero)
template <typename T>
sg_status load_block(sg_problem* pr, const T* X, int64_t ldx, T* dst, cudaStream_t st) {
  SG_CUDA(cudaMemsetAsync(dst, 0, size_t(pr->P) * pr->ld * sizeof(T), st));
  SG_CUDA(cudaMemcpy2DAsync(dst, pr->ld * sizeof(T), X, ldx * sizeof(T), pr->n * sizeof(T), pr->P,
                            cudaMemcpyDeviceToDevice, st));
  return SG_OK;
}

sg_status load_rhs(sg_problem* pr, const double* F, int64_t ldf, double* dst, cudaStream_t st) {
  if (F) return load_block<double>(pr, F, ldf, dst, st);
  SG_CUDA(cudaMemsetAsync(dst, 0, size_t(pr->P) * pr->ld * 8, st));
  SG_CUDA(cudaMemcpyAsync(dst, pr->b.data(), pr->n * 8, cudaMemcpyHostToDevice, st));
  return SG_OK;
}

sg_status norm_host(sg_problem* pr, const double* x, int64_t len, double& out, cudaStream_t st, SolverCtx<double>* c) {
  NewtonWork& w = *pr->nl;
  SG_TRY(vec_norm2<double>(x, len, dp<double>(w.scal), dp<double>(c->fine.partial), dp<unsigned>(c->fine.counter), st));
  SG_CUDA(cudaMemcpyAsync(w.host, w.scal.ptr, 8, cudaMemcpyDeviceToHost, st));
  SG_CUDA(cudaStreamSynchronize(st));
  out = std::sqrt(w.host[0]);
  return SG_OK;
}

sg_status newton_impl(sg_problem* pr, double* X, int64_t ldx, double tol_update, int max_newton,
                      const sg_solve_opts* o, sg_solve_info* info, cudaStream_t st) {
  SG_ARG(pr && X && o, "sg_newton: NULL argument");
  SG_ARG(tol_update > 0 && max_newton > 0, "sg_newton: tol_update and max_newton must be > 0");
  SG_ARG(ldx >= pr->n, "sg_newton: leading dimension < n");
  SG_ARG(o->max_it > 0, "sg_newton: max_it must be > 0");
  SG_ARG(o->mode == 0 || o->mode == 1, "sg_newton: mode must be 0 (FP64) or 1 (FP32 inside the FP64 Newton residual)");
  SG_ARG(o->orth_passes >= 0 && o->orth_passes <= 2, "sg_newton: orth_passes must be 0 (default), 1 or 2");
  SG_ARG(pr->solver && pr->solver->pc.ready, "sg_newton: call sg_precond_setup first");
  SG_TRY(newton_prepare(pr));
  if (o->mode == 0) SG_TRY(ensure_fp64_jacobian(pr));
  NewtonWork& w = *pr->nl;
  SolverState& S = *pr->solver;
  S.restart = o->restart > 0 ? std::min(o->restart, 31) : 30;
  const int64_t len = int64_t(pr->P) * pr->ld;
  const double eta = o->inner_rtol > 0 ? o->inner_rtol : 1e-4;
  auto t0 = std::chrono::steady_clock::now();
  SolverCtx<double>* c64 = nullptr;
  SG_TRY(get_ctx<double>(pr, c64));
  c64->fine.passes = fine_orth_passes(*o);
  SolverCtx<float>* c32 = nullptr;
  if (o->mode == 1) {
    SG_TRY(get_ctx<float>(pr, c32));
    c32->fine.passes = fine_orth_passes(*o);
  }
  if (S.dirty) {
    SG_TRY(c64->scrub(st));
    if (S.c32) SG_TRY(S.c32->scrub(st));
    S.dirty = false;
  }
  S.pc.use_cnn = S.pc.smoother == 1 && pr->cnn && pr->cnn->trained;
  struct ClearCnn {
    Precond& pc;
    ~ClearCnn() { pc.use_cnn = false; }
  } clear_cnn{S.pc};
  S.pc.inner_its_total = 0;
  SG_TRY(c64->clear_counters(st));
  if (c32) SG_TRY(c32->clear_counters(st));
  double* U = dp<double>(w.u64);
  double* F = dp<double>(w.f64);
  double* R = dp<double>(w.r64);
  SG_TRY(load_rhs(pr, nullptr, 0, F, st));
  SG_TRY(load_block<double>(pr, X, ldx, U, st));
  double nF = 0.0;
  SG_TRY(norm_host(pr, F, len, nF, st, c64));
  sg_solve_info inf{};
  std::vector<double> hist;
  bool converged = false;
  for (int it = 0; it < max_newton && nF > 0.0; ++it) {
    // R = F - A(U) U in FP64
    SG_TRY(nl_operator(pr, U, st));
    SG_TRY(nl_apply<double>(pr, w.op, U, F, R, st));
    double nR = 0.0;
    SG_TRY(norm_host(pr, R, len, nR, st, c64));
    if (!std::isfinite(nR)) {
      set_error("sg_newton: non-finite residual");
      return SG_ERR_BREAKDOWN;
    }
    if (nR == 0.0) {
      converged = true;
      break;
    }
    double nd = 0.0;
    GmresResult res;
    if (o->mode == 1) {
      // J(U) d = R / ||R|| in FP32, then U += ||R|| d
      float* U32 = dp<float>(w.u32);
      float* r32 = dp<float>(w.r32);
      float* d32 = dp<float>(w.d32);
      SG_TRY((vec_convert<double, float>(U, U32, len, nullptr, nullptr, st)));
      w.host[1] = nR * nR;
      SG_CUDA(cudaMemcpyAsync(dp<double>(w.scal) + 1, &w.host[1], 8, cudaMemcpyHostToDevice, st));
      SG_TRY((vec_convert<double, float>(R, r32, len, nullptr, dp<double>(w.scal) + 1, st)));
      SG_CUDA(cudaMemsetAsync(d32, 0, len * 4, st));
      Op<float> J = [&](const float* x, float* y) { return nl_jacobian<float>(pr, U32, x, y, st); };
      Op<float> M = [&](const float* r, float* z) { return c32->twolevel(r, z, st); };
      SG_TRY(gmres_run<float>(c32->fine, J, M, r32, d32, true, eta, o->max_it, res, nullptr, 1.0, st, true));
      SG_TRY(vec_add_scaled_f32(U, d32, len, dp<double>(w.scal) + 1, st));
      SG_TRY(vec_norm2<float>(d32, len, dp<double>(w.scal) + 2, dp<double>(c64->fine.partial),
                              dp<unsigned>(c64->fine.counter), st));
      SG_CUDA(cudaMemcpyAsync(w.host + 2, dp<double>(w.scal) + 2, 8, cudaMemcpyDeviceToHost, st));
      SG_CUDA(cudaStreamSynchronize(st));
      nd = nR * std::sqrt(w.host[2]);
    } else {
      double* d64 = dp<double>(w.d64);
      SG_CUDA(cudaMemsetAsync(d64, 0, len * 8, st));
      Op<double> J = [&](const double* x, double* y) { return nl_jacobian<double>(pr, U, x, y, st); };
      Op<double> M = [&](const double* r, double* z) { return c64->twolevel(r, z, st); };
      SG_TRY(gmres_run<double>(c64->fine, J, M, R, d64, true, eta * nR, o->max_it, res, nullptr, 1.0, st, true));
      SG_TRY(vec_axpy_multi<double>(d64, 0, 1, dp<double>(w.one), U, len, st));
      SG_TRY(norm_host(pr, d64, len, nd, st, c64));
    }
    inf.outer_it += res.its;
    inf.ir_steps++;
    double nU = 0.0;
    SG_TRY(norm_host(pr, U, len, nU, st, c64));
    const double change = nU > 0.0 ? nd / nU : 0.0;
    if (!std::isfinite(change)) {
      set_error("sg_newton: non-finite update");
      return SG_ERR_BREAKDOWN;
    }
    hist.push_back(change);
    if (change <= tol_update) {
      converged = true;
      break;
    }
  }
  // nonlinear residual of the returned iterate
  double nR = 0.0;
  if (nF > 0.0) {
    SG_TRY(nl_operator(pr, U, st));
    SG_TRY(nl_apply<double>(pr, w.op, U, F, R, st));
    SG_TRY(norm_host(pr, R, len, nR, st, c64));
  } else {
    SG_CUDA(cudaMemsetAsync(U, 0, len * 8, st));
    converged = true;
  }
  SG_CUDA(cudaMemcpy2DAsync(X, ldx * 8, U, pr->ld * 8, pr->n * 8, pr->P, cudaMemcpyDeviceToDevice, st));
  SG_CUDA(cudaStreamSynchronize(st));
  inf.relres = nF > 0.0 ? nR / nF : 0.0;
  inf.inner_it = S.pc.inner_its_total;
  if (S.pc.device_loops) {
    int64_t graph_kernels = 0;
    for (int which = 0; which < 2; ++which) {
      int fits = 0, cits = 0;
      int64_t k = 0;
      if (which == 0) {
        SG_TRY(c64->read_counters(&fits, &cits));
        SG_TRY(c64->coarse_graph_kernels(&k));
      } else if (S.c32) {
        SG_TRY(S.c32->read_counters(&fits, &cits));
        SG_TRY(S.c32->coarse_graph_kernels(&k));
      }
      inf.inner_it += cits;
      graph_kernels += k;
    }
    note_launches(graph_kernels);
  }
  inf.t_solve = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (o->hist_host && o->hist_cap > 0) {
    const int cnt = std::min<int>(o->hist_cap, int(hist.size()));
    std::memcpy(o->hist_host, hist.data(), cnt * sizeof(double));
    inf.hist_len = cnt;
  }
  if (info) *info = inf;
  if (!converged) {
    set_error("sg_newton: max_newton reached before the relative update fell below tol_update");
    return SG_NOT_CONVERGED;
  }
  return SG_OK;
}

}  // namespace
}  // namespace sg

using namespace sg;

extern "C" {

sg_status sg_newton(sg_problem* pr, double* X, int64_t ldx, double tol_update, int max_newton,
                    const sg_solve_opts* o, sg_solve_info* info, void* stream) {
  const sg_status s = newton_impl(pr, X, ldx, tol_update, max_newton, o, info, static_cast<cudaStream_t>(stream));
  if (s < 0 && pr && pr->solver) pr->solver->dirty = true;
  return s;
}

sg_status sg_nonlinear_residual(sg_problem* pr, const double* F, int64_t ldf, const double* X, int64_t ldx,
                                double* R, int64_t ldr, void* stream) {
  SG_ARG(pr && X && R, "sg_nonlinear_residual: NULL argument");
  SG_ARG(ldx >= pr->n && ldr >= pr->n && (!F || ldf >= pr->n), "sg_nonlinear_residual: leading dimension < n");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SG_TRY(newton_prepare(pr));
  NewtonWork& w = *pr->nl;
  SG_TRY(load_rhs(pr, F, ldf, dp<double>(w.f64), st));
  SG_TRY(load_block<double>(pr, X, ldx, dp<double>(w.u64), st));
  SG_TRY(nl_operator(pr, dp<double>(w.u64), st));
  SG_TRY(nl_apply<double>(pr, w.op, dp<double>(w.u64), dp<double>(w.f64), dp<double>(w.r64), st));
  SG_CUDA(cudaMemcpy2DAsync(R, ldr * 8, w.r64.ptr, pr->ld * 8, pr->n * 8, pr->P, cudaMemcpyDeviceToDevice, st));
  return SG_OK;
}

sg_status sg_nonlinear_jacobian_apply(sg_problem* pr, sg_dtype dtype, const void* U, int64_t ldu, const void* dU,
                                      int64_t lddu, void* Y, int64_t ldy, void* stream) {
  SG_ARG(pr && U && dU && Y, "sg_nonlinear_jacobian_apply: NULL argument");
  SG_ARG(dtype == SG_F64 || dtype == SG_F32, "sg_nonlinear_jacobian_apply: bad dtype");
  SG_ARG(ldu >= pr->n && lddu >= pr->n && ldy >= pr->n, "sg_nonlinear_jacobian_apply: leading dimension < n");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SG_TRY(newton_prepare(pr));
  NewtonWork& w = *pr->nl;
  // the operator at U is formed from the FP64 iterate
  double* U64 = dp<double>(w.u64);
  if (dtype == SG_F64) {
    SG_TRY(ensure_fp64_jacobian(pr));
    SG_TRY(load_block<double>(pr, static_cast<const double*>(U), ldu, U64, st));
    SG_TRY(nl_operator(pr, U64, st));
    SG_TRY(load_block<double>(pr, static_cast<const double*>(dU), lddu, dp<double>(w.d64), st));
    SG_TRY(nl_jacobian<double>(pr, U64, dp<double>(w.d64), dp<double>(w.r64), st));
    SG_CUDA(cudaMemcpy2DAsync(Y, ldy * 8, w.r64.ptr, pr->ld * 8, pr->n * 8, pr->P, cudaMemcpyDeviceToDevice, st));
    return SG_OK;
  }
  const int64_t len = int64_t(pr->P) * pr->ld;
  SG_TRY(load_block<float>(pr, static_cast<const float*>(U), ldu, dp<float>(w.u32), st));
  SG_TRY((vec_convert<float, double>(dp<float>(w.u32), U64, len, nullptr, nullptr, st)));
  SG_TRY(nl_operator(pr, U64, st));
  SG_TRY(load_block<float>(pr, static_cast<const float*>(dU), lddu, dp<float>(w.d32), st));
  SG_TRY(nl_jacobian<float>(pr, dp<float>(w.u32), dp<float>(w.d32), dp<float>(w.r32), st));
  SG_CUDA(cudaMemcpy2DAsync(Y, ldy * 4, w.r32.ptr, pr->ld * 4, pr->n * 4, pr->P, cudaMemcpyDeviceToDevice, st));
  return SG_OK;
}

}  // extern "C"
