// Training targets of the learned smoother: z* = A_0^{-1} r for a batch of
// residual mode images, by conjugate gradients on the fine mean matrix A_0
// preconditioned with one smoothed-aggregation V(1,1) cycle, all columns in
// lockstep (FP64).
#include <algorithm>
#include <cmath>

#include "sg_cnn.h"
#include "sg_kernels.h"
#include "sg_train.h"

namespace sg {

namespace {

// out[c] += sum_{r < n} X[c ld + r] Y[c ld + r]   (column c = blockIdx.y)
__global__ void k_coldot(const double* __restrict__ X, const double* __restrict__ Y, int64_t ld, int64_t n,
                         double* __restrict__ out) {
  const int c = blockIdx.y;
  double s = 0.0;
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < n; r += int64_t(gridDim.x) * blockDim.x)
    s += X[int64_t(c) * ld + r] * Y[int64_t(c) * ld + r];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double ws[8];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) t += ws[w];
    atomicAdd(out + c, t);
  }
}

// x += alpha p, r -= alpha q with alpha = rz / pq per column (0 if pq <= 0)
__global__ void k_pcg_xr(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                         const double* __restrict__ q, int64_t ld, int64_t n, const double* __restrict__ rz,
                         const double* __restrict__ pq) {
  const int c = blockIdx.y;
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  const double d = pq[c];
  const double alpha = d > 0.0 ? rz[c] / d : 0.0;
  const int64_t e = int64_t(c) * ld + i;
  x[e] += alpha * p[e];
  r[e] -= alpha * q[e];
}

// p = z + beta p with beta = rz_new / rz_old per column (0 if rz_old <= 0)
__global__ void k_pcg_p(double* __restrict__ p, const double* __restrict__ z, int64_t ld, int64_t n,
                        const double* __restrict__ rz_new, const double* __restrict__ rz_old) {
  const int c = blockIdx.y;
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  const double d = rz_old[c];
  const double beta = d > 0.0 ? rz_new[c] / d : 0.0;
  const int64_t e = int64_t(c) * ld + i;
  p[e] = z[e] + beta * p[e];
}

template <typename Ti, typename To>
__global__ void k_copy_cols(const Ti* __restrict__ X, int64_t ldx, int64_t n, To* __restrict__ Y, int64_t ldy) {
  const int c = blockIdx.y;
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  Y[int64_t(c) * ldy + i] = To(X[int64_t(c) * ldx + i]);
}

}  // namespace

Cnn::~Cnn() { delete mean; }

sg_status MeanSolver::init(const sg_problem* pr, int cols) {
  if (H.size() == 0) SG_TRY(amg_setup_fine(pr, H));
  if (cols <= nb) return SG_OK;
  nb = cols;
  n = H[0].n;
  ld = H[0].ld;
  const size_t vec = size_t(nb) * ld * 8;
  for (DevBuf* b : {&x, &r, &p, &q, &z}) SG_TRY(b->alloc(vec));
  SG_TRY(scal.alloc(size_t(6) * nb * 8));
  lev.resize(3 * H.size());
  w.b.assign(H.size(), nullptr);
  w.x.assign(H.size(), nullptr);
  w.t.assign(H.size(), nullptr);
  for (size_t l = 0; l < H.size(); ++l) {
    const size_t sz = size_t(nb) * H[l].ld * 8;
    if (l == 0) {
      SG_TRY(lev[2].alloc(sz));
      w.b[0] = dp<double>(r);
      w.x[0] = dp<double>(z);
      w.t[0] = dp<double>(lev[2]);
      continue;
    }
    for (int k = 0; k < 3; ++k) SG_TRY(lev[3 * l + k].alloc(sz));
    w.b[l] = dp<double>(lev[3 * l]);
    w.x[l] = dp<double>(lev[3 * l + 1]);
    w.t[l] = dp<double>(lev[3 * l + 2]);
  }
  return SG_OK;
}

sg_status MeanSolver::solve(const float* B, int64_t ldb, float* Z, int64_t ldz, int cols, double rtol, int max_it,
                            double* relres_max, int* its_out, cudaStream_t st) {
  if (cols > nb) {
    set_error("mean solve: more columns than reserved");
    return SG_ERR_ARG;
  }
  const dim3 gv(unsigned((n + 255) / 256), unsigned(cols));
  const dim3 gd(16, unsigned(cols));
  double* S = dp<double>(scal);
  double *bb = S, *rz = S + nb, *rzn = S + 2 * nb, *pq = S + 3 * nb, *rr = S + 4 * nb;
  double *X = dp<double>(x), *R = dp<double>(r), *Pv = dp<double>(p), *Q = dp<double>(q), *Zv = dp<double>(z);
  const DevCsr& A = H[0].A;
  SG_CUDA(cudaMemsetAsync(X, 0, size_t(cols) * ld * 8, st));
  k_copy_cols<float, double><<<gv, 256, 0, st>>>(B, ldb, n, R, ld); note_launch();
  SG_CUDA(cudaMemsetAsync(S, 0, size_t(6) * nb * 8, st));
  k_coldot<<<gd, 256, 0, st>>>(R, R, ld, n, bb); note_launch();
  SG_TRY(amg_vcycle<double>(H, w, cols, st));
  SG_CUDA(cudaMemcpyAsync(Pv, Zv, size_t(cols) * ld * 8, cudaMemcpyDeviceToDevice, st));
  k_coldot<<<gd, 256, 0, st>>>(R, Zv, ld, n, rz); note_launch();
  SG_CUDA(cudaGetLastError());
  std::vector<double> hb(cols), hr(cols);
  SG_CUDA(cudaMemcpyAsync(hb.data(), bb, size_t(cols) * 8, cudaMemcpyDeviceToHost, st));
  int it = 0;
  double worst = 0.0;
  for (;;) {
    SG_TRY(spmm<double>(A, Pv, ld, nullptr, 0, Q, ld, cols, 0, st));
    SG_CUDA(cudaMemsetAsync(pq, 0, size_t(cols) * 8, st));
    k_coldot<<<gd, 256, 0, st>>>(Pv, Q, ld, n, pq); note_launch();
    k_pcg_xr<<<gv, 256, 0, st>>>(X, R, Pv, Q, ld, n, rz, pq); note_launch();
    ++it;
    if (it % 4 == 0 || it >= max_it) {
      SG_CUDA(cudaMemsetAsync(rr, 0, size_t(cols) * 8, st));
      k_coldot<<<gd, 256, 0, st>>>(R, R, ld, n, rr); note_launch();
      SG_CUDA(cudaMemcpyAsync(hr.data(), rr, size_t(cols) * 8, cudaMemcpyDeviceToHost, st));
      SG_CUDA(cudaStreamSynchronize(st));
      worst = 0.0;
      for (int c = 0; c < cols; ++c) {
        const double rel = hb[c] > 0.0 ? std::sqrt(hr[c] / hb[c]) : 0.0;
        if (!std::isfinite(rel)) {
          set_error("mean solve: non-finite residual");
          return SG_ERR_BREAKDOWN;
        }
        worst = std::max(worst, rel);
      }
      if (worst <= rtol || it >= max_it) break;
    }
    SG_TRY(amg_vcycle<double>(H, w, cols, st));
    SG_CUDA(cudaMemsetAsync(rzn, 0, size_t(cols) * 8, st));
    k_coldot<<<gd, 256, 0, st>>>(R, Zv, ld, n, rzn); note_launch();
    k_pcg_p<<<gv, 256, 0, st>>>(Pv, Zv, ld, n, rzn, rz); note_launch();
    std::swap(rz, rzn);
    SG_CUDA(cudaGetLastError());
  }
  k_copy_cols<double, float><<<gv, 256, 0, st>>>(X, ld, n, Z, ldz); note_launch();
  SG_CUDA(cudaGetLastError());
  if (relres_max) *relres_max = worst;
  if (its_out) *its_out = it;
  return SG_OK;
}

}  // namespace sg
