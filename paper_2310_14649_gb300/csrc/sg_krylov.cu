// Krylov building blocks (Sec. 3: FGMRES outer solver, inner GMRES on the
// coarse problem): fused multi-vector dot products and updates for
// classical Gram-Schmidt (one pass, or two for CGS2), the Givens
// update of the Hessenberg column and the triangular solve, all on the
// device.  Dot products accumulate in FP64 across threads; for FP32 vectors
// each thread first sums its few products in FP32.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "sg_kernels.h"

namespace sg {

namespace {

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = kMdotBlocks;
constexpr int kMaxV = kMdotMaxVectors;  // vectors per fused pass

template <typename T> struct Acc;
template <> struct Acc<double> { using type = double; };
template <> struct Acc<float> { using type = float; };

// One partial sum per (block, vector), reduced by the last block to finish.
// blockIdx.y = vector index i, blockIdx.x = chunk of the elements; every
// block reads its chunk of V_i and w once, so the grid has nv x chunks
// blocks of few registers each.  FP32 products are summed in FP32 over at
// most 8 elements per thread, then in FP64.
template <typename T>
__device__ void last_block_finish(double v, double* __restrict__ partial, unsigned* __restrict__ counter,
                                  double* __restrict__ out, int nv_used) {
  __shared__ double red[kRedThreads / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) red[wid] = v;
  __syncthreads();
  const int nbx = gridDim.x, nv = gridDim.y;
  if (threadIdx.x == 0) {
    double x = 0.0;
    for (int w = 0; w < kRedThreads / 32; ++w) x += red[w];
    partial[blockIdx.y * nbx + blockIdx.x] = x;
    __threadfence();
    last = (atomicAdd(counter, 1u) == unsigned(nbx * nv) - 1u);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    for (int i = wid; i < nv_used; i += kRedThreads / 32) {
      double x = 0.0;
      for (int b = lane; b < nbx; b += 32) x += partial[i * nbx + b];
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) out[i] = x;
    }
    if (threadIdx.x == 0) *counter = 0u;
  }
}

// out[i] = V_i . w  (V_i = V + i * stride), or out[0] = w . w when V == w.
// With jdev the number of vectors is *jdev + 1 (read on the device; the
// grid is sized for the maximum and the extra rows of blocks contribute 0).
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_mdot(const T* __restrict__ V, int64_t stride, const T* __restrict__ w,
                                                      int64_t len, double* __restrict__ partial,
                                                      unsigned* __restrict__ counter, double* __restrict__ out,
                                                      const int* __restrict__ jdev) {
  using A = typename Acc<T>::type;
  const int nv_used = jdev ? *jdev + 1 : int(gridDim.y);
  const T* v = V + int64_t(blockIdx.y) * stride;
  double tot = 0.0;
  A loc = A(0);
  int cnt = 0;
  const int64_t lim = int(blockIdx.y) < nv_used ? len : 0;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < lim; e += int64_t(gridDim.x) * blockDim.x) {
    loc += A(v[e]) * A(w[e]);
    if (++cnt == 8) {
      tot += double(loc);
      loc = A(0);
      cnt = 0;
    }
  }
  tot += double(loc);
  last_block_finish<T>(tot, partial, counter, out, nv_used);
}

// w -= sum_i h_i V_i, and (when out) out[0] = w . w of the updated w.
// With jdev the number of vectors is *jdev + 1.
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_axpy_norm(const T* __restrict__ V, int64_t stride, int nv,
                                                           const double* __restrict__ h, T* __restrict__ w,
                                                           int64_t len, double* __restrict__ partial,
                                                           unsigned* __restrict__ counter, double* __restrict__ out,
                                                           const int* __restrict__ jdev) {
  using A = typename Acc<T>::type;
  __shared__ T hs[kMaxV];
  if (jdev) nv = *jdev + 1;
  if (threadIdx.x < nv) hs[threadIdx.x] = T(h[threadIdx.x]);
  __syncthreads();
  double tot = 0.0;
  A loc = A(0);
  int cnt = 0;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < len; e += int64_t(gridDim.x) * blockDim.x) {
    T we = w[e];
    for (int i = 0; i < nv; ++i) we -= hs[i] * V[int64_t(i) * stride + e];
    w[e] = we;
    loc += A(we) * A(we);
    if (++cnt == 8) {
      tot += double(loc);
      loc = A(0);
      cnt = 0;
    }
  }
  tot += double(loc);
  if (out) last_block_finish<T>(tot, partial, counter, out, 1);
}

inline unsigned chunks_for(int64_t len, int nv) {
  // about 4 x 152 blocks in total, at least one 256-thread block per 1024 elements
  int64_t want = (4 * 152 + nv - 1) / nv;
  int64_t cap = (len + 1023) / 1024;
  int64_t c = want < cap ? want : cap;
  return unsigned(c < 1 ? 1 : c);
}

template <typename T>
__global__ void k_scale_by(const T* __restrict__ x, T* __restrict__ y, int64_t len, const double* __restrict__ den,
                           bool take_sqrt) {
  double d = *den;
  if (take_sqrt) d = sqrt(d);
  const T s = T(d != 0.0 ? 1.0 / d : 0.0);
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < len; e += int64_t(gridDim.x) * blockDim.x)
    y[e] = x[e] * s;
}

template <typename T>
__global__ void k_axpy_multi(const T* __restrict__ V, int64_t stride, int nv, const double* __restrict__ coef,
                             T* __restrict__ x, int64_t len, const int* __restrict__ kdev) {
  if (kdev) nv = *kdev;
  T c[kMaxV];
#pragma unroll
  for (int i = 0; i < kMaxV; ++i) c[i] = i < nv ? T(coef[i]) : T(0);
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < len; e += int64_t(gridDim.x) * blockDim.x) {
    T acc = x[e];
#pragma unroll
    for (int i = 0; i < kMaxV; ++i)
      if (i < nv) acc += c[i] * V[int64_t(i) * stride + e];
    x[e] = acc;
  }
}

template <typename Ti, typename To>
__global__ void k_convert(const Ti* __restrict__ x, To* __restrict__ y, int64_t len, const double* __restrict__ num,
                          const double* __restrict__ den) {
  double s = 1.0;
  if (num) s *= *num;
  if (den) s /= sqrt(*den);
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < len; e += int64_t(gridDim.x) * blockDim.x)
    y[e] = To(double(x[e]) * s);
}

__global__ void k_add_scaled_f32(double* __restrict__ x, const float* __restrict__ d, int64_t len,
                                 const double* __restrict__ s2) {
  const double s = sqrt(*s2);
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < len; e += int64_t(gridDim.x) * blockDim.x)
    x[e] += s * double(d[e]);
}

__global__ void k_gmres_init(GmresState s, int m, const double* beta2) {
  const double beta = sqrt(*beta2);
  for (int i = threadIdx.x; i <= m; i += blockDim.x) s.g[i] = i == 0 ? beta : 0.0;
  if (threadIdx.x == 0) {
    s.scal[2] = beta;
    s.scal[3] = beta;
    s.scal[4] = 0.0;
  }
}

// Column j of the Hessenberg matrix from the Gram-Schmidt coefficients of
// both passes (the second column is zero with one pass), previous
// rotations, new rotation, residual estimate |g_{j+1}|.
__global__ void k_gmres_givens(GmresState s, int m, int j, double* host_est) {
  if (threadIdx.x != 0) return;
  double* col = s.H + int64_t(j) * (m + 1);
  for (int i = 0; i <= j; ++i) col[i] = s.hsum[i] + s.hsum[(m + 1) + i];
  const double hn = sqrt(s.scal[0]);
  col[j + 1] = hn;
  s.scal[1] = hn;
  for (int i = 0; i < j; ++i) {
    double t = s.cs[i] * col[i] + s.sn[i] * col[i + 1];
    col[i + 1] = -s.sn[i] * col[i] + s.cs[i] * col[i + 1];
    col[i] = t;
  }
  double den = hypot(col[j], col[j + 1]);
  double c = den != 0.0 ? col[j] / den : 1.0, sn = den != 0.0 ? col[j + 1] / den : 0.0;
  s.cs[j] = c;
  s.sn[j] = sn;
  col[j] = den;
  col[j + 1] = 0.0;
  s.g[j + 1] = -sn * s.g[j];
  s.g[j] = c * s.g[j];
  const double est = fabs(s.g[j + 1]);
  s.scal[2] = est;
  bool bad = !isfinite(est) || !isfinite(hn) || !isfinite(den);
  s.scal[4] = bad ? 1.0 : 0.0;
  if (host_est) {
    host_est[0] = est;
    host_est[1] = hn;
    host_est[2] = bad ? 1.0 : 0.0;
  }
}

__global__ void k_gmres_backsolve(GmresState s, int m, int k) {
  if (threadIdx.x != 0) return;
  for (int i = k - 1; i >= 0; --i) {
    double acc = s.g[i];
    for (int c = i + 1; c < k; ++c) acc -= s.H[int64_t(c) * (m + 1) + i] * s.y[c];
    double d = s.H[int64_t(i) * (m + 1) + i];
    s.y[i] = d != 0.0 ? acc / d : 0.0;
  }
}

inline unsigned grid_for(int64_t len) {
  int64_t b = (len + 255) / 256;
  return unsigned(b < 4 * 152 ? (b > 0 ? b : 1) : 4 * 152);
}

}  // namespace

template <typename T>
sg_status vec_mdot(const T* V, int64_t stride, int nv, const T* w, int64_t len, double* out, double* partial,
                   unsigned* counter, cudaStream_t st) {
  if (nv < 1 || nv > kMaxV) {
    set_error("vec_mdot: nv must be in [1, 32]");
    return SG_ERR_ARG;
  }
  const unsigned nbx = std::min<unsigned>(chunks_for(len, nv), unsigned(kRedBlocks));
  k_mdot<T><<<dim3(nbx, unsigned(nv)), kRedThreads, 0, st>>>(V, stride, w, len, partial, counter, out, nullptr);
  note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

template <typename T>
sg_status vec_maxpy_mdot(const T* V, int64_t stride, int nv, const double* h, T* w, int64_t len, double* out,
                         double* partial, unsigned* counter, cudaStream_t st) {
  const unsigned nb = std::min<unsigned>(chunks_for(len, 1), unsigned(kRedBlocks));
  k_axpy_norm<T><<<dim3(nb, 1), kRedThreads, 0, st>>>(V, stride, nv, h, w, len, partial, counter, nullptr,
                                                       nullptr);
  note_launch();
  SG_CUDA(cudaGetLastError());
  return vec_mdot<T>(V, stride, nv, w, len, out, partial, counter, st);
}

template <typename T>
sg_status vec_maxpy_norm(const T* V, int64_t stride, int nv, const double* h, T* w, int64_t len, double* out,
                         double* partial, unsigned* counter, cudaStream_t st) {
  const unsigned nb = std::min<unsigned>(chunks_for(len, 1), unsigned(kRedBlocks));
  k_axpy_norm<T><<<dim3(nb, 1), kRedThreads, 0, st>>>(V, stride, nv, h, w, len, partial, counter, out, nullptr);
  note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

template <typename T>
sg_status vec_norm2(const T* x, int64_t len, double* out, double* partial, unsigned* counter, cudaStream_t st) {
  return vec_mdot<T>(x, 0, 1, x, len, out, partial, counter, st);
}

template <typename T>
sg_status vec_scale_by(const T* x, T* y, int64_t len, const double* den, bool take_sqrt, cudaStream_t st) {
  k_scale_by<T><<<grid_for(len), 256, 0, st>>>(x, y, len, den, take_sqrt); note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

template <typename T>
sg_status vec_axpy_multi(const T* V, int64_t stride, int nv, const double* coef, T* x, int64_t len,
                         cudaStream_t st) {
  for (int i0 = 0; i0 < nv; i0 += kMaxV) {
    int cnt = nv - i0 < kMaxV ? nv - i0 : kMaxV;
    k_axpy_multi<T><<<grid_for(len), 256, 0, st>>>(V + int64_t(i0) * stride, stride, cnt, coef + i0, x, len,
                                                   nullptr); note_launch();
    SG_CUDA(cudaGetLastError());
  }
  return SG_OK;
}

template <typename Ti, typename To>
sg_status vec_convert(const Ti* x, To* y, int64_t len, const double* num, const double* den, cudaStream_t st) {
  k_convert<Ti, To><<<grid_for(len), 256, 0, st>>>(x, y, len, num, den); note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

sg_status vec_add_scaled_f32(double* x, const float* d, int64_t len, const double* s2, cudaStream_t st) {
  k_add_scaled_f32<<<grid_for(len), 256, 0, st>>>(x, d, len, s2); note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

sg_status gmres_init(GmresState s, int m, const double* beta2, cudaStream_t st) {
  k_gmres_init<<<1, 64, 0, st>>>(s, m, beta2); note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

sg_status gmres_givens(GmresState s, int m, int j, double* host_est, cudaStream_t st) {
  k_gmres_givens<<<1, 32, 0, st>>>(s, m, j, host_est); note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

sg_status gmres_backsolve(GmresState s, int m, int k, cudaStream_t st) {
  k_gmres_backsolve<<<1, 32, 0, st>>>(s, m, k); note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

// ---------------------------------------------------------------------------
// Device-driven GMRES: the iteration index, the counters and the stopping
// decisions live in device memory (DevGmres), so a whole restarted solve
// runs inside one CUDA graph whose loops are conditional WHILE nodes.
// ---------------------------------------------------------------------------
namespace {

__global__ void k_dg_init(DevGmres d, const double* __restrict__ rnorm2, double rtol, cudaGraphConditionalHandle outer,
                          const double* __restrict__ rr2, const double* __restrict__ nf2, double target) {
  const double nr = sqrt(*rnorm2);
  double tol = rtol;
  // a refinement step within a factor of its target: the reduction still
  // needed, with a factor two of margin (at most 0.5)
  if (rr2 && nf2 && *rr2 > 0.0 && *nf2 > 0.0) tol = fmax(rtol, fmin(0.5, 0.5 * target / sqrt(*rr2 / *nf2)));
  d.dtol[0] = tol * nr;
  d.iv[1] = 0;  // iterations
  d.iv[3] = 0;  // stop
  d.iv[5] = 0;  // breakdown
  cudaGraphSetConditional(outer, nr > 0.0 ? 1u : 0u);
}

// start of a restart cycle: beta = ||r0||, g = beta e_0, j = 0
__global__ void k_dg_start(DevGmres d, GmresState s, int m, const double* __restrict__ beta2,
                           cudaGraphConditionalHandle inner) {
  const double beta = sqrt(*beta2);
  for (int i = threadIdx.x; i <= m; i += blockDim.x) s.g[i] = i == 0 ? beta : 0.0;
  if (threadIdx.x == 0) {
    // scal[3] keeps beta^2: the normalisation of V_0 that follows reads it
    d.iv[0] = 0;
    d.iv[6] += 1;  // restart cycles summed over solves
    const bool go = beta > d.dtol[0] && isfinite(beta) && d.iv[1] < d.iv[2];
    if (!go) d.iv[3] = 1;
    cudaGraphSetConditional(inner, go ? 1u : 0u);
  }
}

// Hessenberg column j (device j), rotations, estimate; j and the iteration
// count advance; the inner loop continues while the estimate is above the
// tolerance, the cycle has room and the iteration cap is not reached.
__global__ void k_dg_givens(DevGmres d, GmresState s, int m, cudaGraphConditionalHandle inner) {
  if (threadIdx.x != 0) return;
  const int j = d.iv[0];
  double* col = s.H + int64_t(j) * (m + 1);
  for (int i = 0; i <= j; ++i) col[i] = s.hsum[i] + s.hsum[(m + 1) + i];
  const double hn = sqrt(s.scal[0]);
  col[j + 1] = hn;
  s.scal[1] = hn;
  for (int i = 0; i < j; ++i) {
    double t = s.cs[i] * col[i] + s.sn[i] * col[i + 1];
    col[i + 1] = -s.sn[i] * col[i] + s.cs[i] * col[i + 1];
    col[i] = t;
  }
  const double den = hypot(col[j], col[j + 1]);
  const double c = den != 0.0 ? col[j] / den : 1.0, sn = den != 0.0 ? col[j + 1] / den : 0.0;
  s.cs[j] = c;
  s.sn[j] = sn;
  col[j] = den;
  col[j + 1] = 0.0;
  s.g[j + 1] = -sn * s.g[j];
  s.g[j] = c * s.g[j];
  const double est = fabs(s.g[j + 1]);
  s.scal[2] = est;
  const bool bad = !isfinite(est) || !isfinite(hn);
  d.iv[0] = j + 1;
  d.iv[1] += 1;
  d.iv[4] += 1;  // iterations summed over solves
  if (bad) d.iv[5] = 1;
  const bool go = !bad && est > d.dtol[0] && hn != 0.0 && j + 1 < m && d.iv[1] < d.iv[2];
  cudaGraphSetConditional(inner, go ? 1u : 0u);
}

// end of a cycle: stop when converged (by the Arnoldi estimate when trust,
// else only by the true residual of the next restart), stalled, failed or
// out of iterations
__global__ void k_dg_end(DevGmres d, GmresState s, cudaGraphConditionalHandle outer, int trust) {
  const double est = s.scal[2];
  const bool done = d.iv[3] || d.iv[5] || (trust && !(est > d.dtol[0])) || d.iv[1] >= d.iv[2];
  cudaGraphSetConditional(outer, done ? 0u : 1u);
}

// V_j = src (device index j), full length
template <typename T>
__global__ void k_dg_store_j(const T* __restrict__ src, T* __restrict__ V, int64_t stride, int64_t len, DevGmres d) {
  T* v = V + int64_t(d.iv[0]) * stride;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < len; e += int64_t(gridDim.x) * blockDim.x)
    v[e] = src[e];
}

// Refinement loop control: rr = ||F - A x||^2, nf2 = ||F||^2; continue
// while sqrt(rr / nf2) > rtol, the step cap and the iteration cap allow it
// and rr is finite.  iv[0] steps taken, iv[1] non-finite flag.
__global__ void k_ir_decide(const double* __restrict__ rr, const double* __restrict__ nf2, int* __restrict__ iv,
                            double rtol, int max_ir, const int* __restrict__ its_total, int max_it,
                            cudaGraphConditionalHandle h) {
  const double r = *rr, f = *nf2;
  const bool bad = !isfinite(r);
  if (bad) iv[1] = 1;
  const double rel = f > 0.0 ? sqrt(r / f) : 0.0;
  const bool go = !bad && rel > rtol && iv[0] < max_ir && *its_total < max_it;
  if (go) iv[0] += 1;
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

__global__ void k_dg_backsolve(DevGmres d, GmresState s, int m) {
  if (threadIdx.x != 0) return;
  const int k = d.iv[0];
  for (int i = k - 1; i >= 0; --i) {
    double acc = s.g[i];
    for (int c = i + 1; c < k; ++c) acc -= s.H[int64_t(c) * (m + 1) + i] * s.y[c];
    const double dg = s.H[int64_t(i) * (m + 1) + i];
    s.y[i] = dg != 0.0 ? acc / dg : 0.0;
  }
}

// V_{j} = w / h_{j,j-1} for the device index j (already advanced)
template <typename T>
__global__ void k_dg_scale_next(const T* __restrict__ w, T* __restrict__ V, int64_t stride, int64_t len, DevGmres d,
                                const double* __restrict__ hn, T* __restrict__ dst, int64_t ldd, int64_t lds,
                                int64_t n) {
  const double h = *hn;
  const T sc = T(h != 0.0 ? 1.0 / h : 0.0);
  T* v = V + int64_t(d.iv[0]) * stride;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < len; e += int64_t(gridDim.x) * blockDim.x) {
    const T x = w[e] * sc;
    v[e] = x;
    if (dst) {
      const int64_t a = e / lds, r = e - a * lds;
      if (r < n) dst[a * ldd + r] = x;
    }
  }
}

// mode-major block copy from V_j (device index j) with a change of
// leading dimension: dst[a * ldd + r] = V_j[a * lds + r], r < n
template <typename T>
__global__ void k_dg_copy_vj(const T* __restrict__ V, int64_t stride, int64_t lds, T* __restrict__ dst, int64_t ldd,
                             int64_t n, DevGmres d) {
  const int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int a = blockIdx.y;
  if (r >= n) return;
  dst[int64_t(a) * ldd + r] = V[int64_t(d.iv[0]) * stride + int64_t(a) * lds + r];
}

}  // namespace

template <typename T>
sg_status dg_mdot(const T* V, int64_t stride, const T* w, int64_t len, double* out, double* partial, unsigned* counter,
                  const int* jdev, int nv_max, cudaStream_t st) {
  const unsigned nbx = std::min<unsigned>(chunks_for(len, nv_max), unsigned(kRedBlocks));
  k_mdot<T><<<dim3(nbx, unsigned(nv_max)), kRedThreads, 0, st>>>(V, stride, w, len, partial, counter, out, jdev);
  note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

template <typename T>
sg_status dg_axpy_norm(const T* V, int64_t stride, const double* h, T* w, int64_t len, double* out, double* partial,
                       unsigned* counter, const int* jdev, cudaStream_t st) {
  const unsigned nb = std::min<unsigned>(chunks_for(len, 1), unsigned(kRedBlocks));
  k_axpy_norm<T><<<dim3(nb, 1), kRedThreads, 0, st>>>(V, stride, 0, h, w, len, partial, counter, out, jdev);
  note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

template <typename T>
sg_status dg_axpy_multi(const T* V, int64_t stride, const double* coef, T* x, int64_t len, const int* kdev,
                        cudaStream_t st) {
  k_axpy_multi<T><<<grid_for(len), 256, 0, st>>>(V, stride, 0, coef, x, len, kdev);
  note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

template <typename T>
sg_status dg_scale_next(const T* w, T* V, int64_t stride, int64_t len, DevGmres d, const double* hn, cudaStream_t st,
                        T* dst, int64_t ldd, int64_t lds, int64_t n) {
  k_dg_scale_next<T><<<grid_for(len), 256, 0, st>>>(w, V, stride, len, d, hn, dst, ldd, lds > 0 ? lds : 1, n);
  note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

template <typename T>
sg_status dg_copy_vj(const T* V, int64_t stride, int64_t lds, T* dst, int64_t ldd, int64_t n, int P, DevGmres d,
                     cudaStream_t st) {
  dim3 g(unsigned((n + 255) / 256), unsigned(P));
  k_dg_copy_vj<T><<<g, 256, 0, st>>>(V, stride, lds, dst, ldd, n, d);
  note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

sg_status dg_init(DevGmres d, const double* rnorm2, double rtol, cudaGraphConditionalHandle outer, cudaStream_t st,
                  const double* rr2, const double* nf2, double target) {
  k_dg_init<<<1, 1, 0, st>>>(d, rnorm2, rtol, outer, rr2, nf2, target);
  note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}
sg_status dg_start(DevGmres d, GmresState s, int m, const double* beta2, cudaGraphConditionalHandle inner,
                   cudaStream_t st) {
  k_dg_start<<<1, 64, 0, st>>>(d, s, m, beta2, inner);
  note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}
sg_status dg_givens(DevGmres d, GmresState s, int m, cudaGraphConditionalHandle inner, cudaStream_t st) {
  k_dg_givens<<<1, 32, 0, st>>>(d, s, m, inner);
  note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}
sg_status dg_end(DevGmres d, GmresState s, cudaGraphConditionalHandle outer, cudaStream_t st, bool trust) {
  k_dg_end<<<1, 1, 0, st>>>(d, s, outer, trust ? 1 : 0);
  note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}
sg_status dg_backsolve(DevGmres d, GmresState s, int m, cudaStream_t st) {
  k_dg_backsolve<<<1, 32, 0, st>>>(d, s, m);
  note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

template <typename T>
sg_status dg_store_j(const T* src, T* V, int64_t stride, int64_t len, DevGmres d, cudaStream_t st) {
  k_dg_store_j<T><<<grid_for(len), 256, 0, st>>>(src, V, stride, len, d);
  note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

sg_status ir_decide(const double* rr, const double* nf2, int* iv, double rtol, int max_ir, const int* its_total,
                    int max_it, cudaGraphConditionalHandle h, cudaStream_t st) {
  k_ir_decide<<<1, 1, 0, st>>>(rr, nf2, iv, rtol, max_ir, its_total, max_it, h);
  note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

#define INST_DG(T)                                                                                             \
  template sg_status dg_mdot<T>(const T*, int64_t, const T*, int64_t, double*, double*, unsigned*, const int*, \
                                int, cudaStream_t);                                                            \
  template sg_status dg_axpy_norm<T>(const T*, int64_t, const double*, T*, int64_t, double*, double*,          \
                                     unsigned*, const int*, cudaStream_t);                                     \
  template sg_status dg_axpy_multi<T>(const T*, int64_t, const double*, T*, int64_t, const int*, cudaStream_t); \
  template sg_status dg_scale_next<T>(const T*, T*, int64_t, int64_t, DevGmres, const double*, cudaStream_t, T*, \
                                      int64_t, int64_t, int64_t);                                                \
  template sg_status dg_copy_vj<T>(const T*, int64_t, int64_t, T*, int64_t, int64_t, int, DevGmres, cudaStream_t); \
  template sg_status dg_store_j<T>(const T*, T*, int64_t, int64_t, DevGmres, cudaStream_t);
INST_DG(float)
INST_DG(double)
#undef INST_DG

#define INST(T)                                                                                                   \
  template sg_status vec_mdot<T>(const T*, int64_t, int, const T*, int64_t, double*, double*, unsigned*,         \
                                 cudaStream_t);                                                                   \
  template sg_status vec_maxpy_mdot<T>(const T*, int64_t, int, const double*, T*, int64_t, double*, double*,     \
                                       unsigned*, cudaStream_t);                                                  \
  template sg_status vec_maxpy_norm<T>(const T*, int64_t, int, const double*, T*, int64_t, double*, double*,     \
                                       unsigned*, cudaStream_t);                                                  \
  template sg_status vec_norm2<T>(const T*, int64_t, double*, double*, unsigned*, cudaStream_t);                 \
  template sg_status vec_scale_by<T>(const T*, T*, int64_t, const double*, bool, cudaStream_t);                  \
  template sg_status vec_axpy_multi<T>(const T*, int64_t, int, const double*, T*, int64_t, cudaStream_t);
INST(float)
INST(double)
#undef INST
// ---------------------------------------------------------------------------
// Allocation-free variant of the multi-vector dot product.  The reduction
// scratch of k_multi (one partial sum per block and vector, plus the
// arrival counter of the last-block reduction) lives in file-scope device
// arrays instead of caller- or handle-owned memory, so the entry point needs
// neither a handle nor any allocation.  Every GPU that loads the library
// holds these arrays (about 78 KB) until the process exits.
// ---------------------------------------------------------------------------
namespace {
__device__ __align__(256) double g_noalloc_partial[kMdotBlocks * kMdotMaxVectors];
__device__ __align__(256) unsigned g_noalloc_counter[64];

constexpr int kMaxDevices = 64;
struct NoallocScratch {
  double* partial = nullptr;
  unsigned* counter = nullptr;
};
std::mutex g_noalloc_mu;
NoallocScratch g_noalloc[kMaxDevices];

// Device address of the arrays on the current device.  In host code the
// array names are host-side stand-ins, not device addresses, so the first
// call on each device asks the runtime for the addresses (with that device
// current) and keeps them.
sg_status noalloc_scratch(NoallocScratch& out) {
  int dev = 0;
  SG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("sg_mdot_noalloc: device index out of range");
    return SG_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  NoallocScratch& s = g_noalloc[dev];
  if (!s.partial) {
    void* p = nullptr;
    void* c = nullptr;
    SG_CUDA(cudaGetSymbolAddress(&p, g_noalloc_partial));
    SG_CUDA(cudaGetSymbolAddress(&c, g_noalloc_counter));
    s.partial = static_cast<double*>(p);
    s.counter = static_cast<unsigned*>(c);
  }
  out = s;
  return SG_OK;
}
}  // namespace

template sg_status vec_convert<double, float>(const double*, float*, int64_t, const double*, const double*,
                                              cudaStream_t);
template sg_status vec_convert<float, double>(const float*, double*, int64_t, const double*, const double*,
                                              cudaStream_t);
template sg_status vec_convert<double, double>(const double*, double*, int64_t, const double*, const double*,
                                               cudaStream_t);
template sg_status vec_convert<float, float>(const float*, float*, int64_t, const double*, const double*,
                                             cudaStream_t);

}  // namespace sg

extern "C" sg_status sg_mdot_noalloc(sg_dtype dtype, const void* V, int64_t stride, int nv, const void* w,
                                     int64_t len, double* out, void* stream) {
  using namespace sg;
  SG_ARG(V && w && out, "sg_mdot_noalloc: NULL argument");
  SG_ARG(dtype == SG_F64 || dtype == SG_F32, "sg_mdot_noalloc: bad dtype");
  SG_ARG(nv >= 1 && nv <= kMdotMaxVectors,
         "sg_mdot_noalloc: nv must be in [1, 32] (the static scratch holds 304 x 32 partial sums)");
  SG_ARG(len >= 0 && (nv == 1 || stride >= len), "sg_mdot_noalloc: len < 0 or stride < len");
  NoallocScratch s;
  SG_TRY(noalloc_scratch(s));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the arrival counter must start at zero; the partial sums are written
  // before they are read
  SG_CUDA(cudaMemsetAsync(s.counter, 0, sizeof(unsigned), st));
  if (dtype == SG_F64)
    return vec_mdot<double>(static_cast<const double*>(V), stride, nv, static_cast<const double*>(w), len, out,
                            s.partial, s.counter, st);
  return vec_mdot<float>(static_cast<const float*>(V), stride, nv, static_cast<const float*>(w), len, out,
                         s.partial, s.counter, st);
}
