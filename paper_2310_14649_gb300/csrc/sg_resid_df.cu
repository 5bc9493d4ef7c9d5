// Refinement residual R = F - sum_k A_k X G_k^T (Sec. 2.1, Eq.
// Galerkin_L_exp) in double-FP32 arithmetic on the FP32 pipes.
//
// GB300 runs FP64 at about 1/64 of its FP32 rate, so the FP64 residual of
// the mixed-precision refinement is bound by the FP64 units.  Here every
// FP64 value v is carried as two FP32 numbers hi + lo (hi = fl32(v), lo =
// fl32(v - hi): 48 significant bits), products are formed exactly with an
// FMA (TwoProd: p = fl(a b), e = fma(a, b, -p)) plus the two cross terms,
// and sums with the error-free TwoSum, the rounding errors collected in the
// low word (the compensated dot product of Ogita, Rump and Oishi, "Accurate
// sum and dot product", 2005).
//
// Form: a row of A_k is the sum over the four edges of its node of
// w_k(e) (x_r - x_neighbour) (P1 element matrices have zero row sums), so
//     y_r = sum_{e in edges(r)} B^e (x_r - x_c(e)),   B^e_ab = sum_k g_kab w_k(e),
// with the neighbour's term dropped on the Dirichlet boundary.  The edge
// blocks are summed once at setup in FP64 and stored split (symmetric, a <=
// b packed), one block per edge shared by its two end nodes: 2.5x fewer
// bytes than one block per stencil slot.  Differencing the iterate first
// also keeps the products small: x_r - x_c is O(h) smaller than x, so the
// cancellation of the stencil happens before the products are rounded.
//
// Kernel: a CTA owns 32 consecutive rows (lane = row) and 8 warps; per edge
// slot the differences d_b = x_r[b] - x_c[b] are formed in double-FP32 into
// shared memory, then warp w accumulates outputs a = w, w + 8, ... over all
// b with the packed block entries of the row's edge (coalesced: the edges of
// consecutive rows are consecutive).  FP64 is used only to split X and to
// form F - (hi + lo) at the store.
#include <algorithm>
#include <vector>

#include "sg_kernels.h"

namespace sg {

namespace {

constexpr int kDfWarps = 8;

// x - y for two double-FP32 values, normalised (|lo| <= ulp(hi) / 2)
__device__ __forceinline__ float2 df_sub(float2 x, float2 y) {
  const float s = __fsub_rn(x.x, y.x);
  const float bb = __fsub_rn(s, x.x);
  const float t = __fadd_rn(__fsub_rn(x.x, __fsub_rn(s, bb)), __fsub_rn(-y.x, bb));
  const float u = __fadd_rn(t, __fsub_rn(x.y, y.y));
  const float h = __fadd_rn(s, u);
  return make_float2(h, __fsub_rn(u, __fsub_rn(h, s)));
}

// (sh, sl) += a b: TwoProd of the high words, the cross terms into the
// error, TwoSum of the running high word, errors collected in sl
__device__ __forceinline__ void df_fma(float& sh, float& sl, float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  const float s = __fadd_rn(sh, p);
  const float bb = __fsub_rn(s, sh);
  const float t = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(t, e));
}

// (sh, sl) <- TwoSum(sh, sl): the low word back to at most half an ulp
__device__ __forceinline__ void df_renorm(float& sh, float& sl) {
  const float s = __fadd_rn(sh, sl);
  const float bb = __fsub_rn(s, sh);
  sl = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(sl, bb));
  sh = s;
}

__device__ __forceinline__ float2 df_split(double v) {
  const float h = __double2float_rn(v);
  return make_float2(h, __double2float_rn(v - double(h)));
}

// Xs[b][r] = split(X[b][r]) for r < n, zero for the padding rows
__global__ void k_split_df(int64_t n, int64_t ldr, const double* __restrict__ X, int64_t ldx,
                           float2* __restrict__ Xs) {
  const int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int b = blockIdx.y;
  if (r >= ldr) return;
  Xs[int64_t(b) * ldr + r] = r < n ? df_split(X[int64_t(b) * ldx + r]) : make_float2(0.f, 0.f);
}

// B[q][e] = split(sum over pair q's list of g w_k(e)) in FP64; thread per
// (edge, pair)
__global__ void k_edge_blocks_df(int64_t ne, int64_t lde, int64_t vkst, const int* __restrict__ pptr,
                                 const int* __restrict__ pk, const double* __restrict__ pg,
                                 const double* __restrict__ w, float2* __restrict__ B) {
  const int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int q = blockIdx.y;
  if (e >= lde) return;
  double c = 0.0;
  if (e < ne)
    for (int t = pptr[q]; t < pptr[q + 1]; ++t) c = fma(pg[t], w[int64_t(pk[t]) * vkst + e], c);
  B[int64_t(q) * lde + e] = df_split(c);
}

// R = F - A X over the edge blocks (R = A X when F is null).  Warp w owns
// outputs a = w + 8 j, j < J.
template <int J>
__global__ void __launch_bounds__(32 * kDfWarps) k_resid_flux_df(int64_t n, int64_t ldr, int P, int64_t lde,
                                                                 const int* __restrict__ col,
                                                                 const int* __restrict__ vidx,
                                                                 const float2* __restrict__ B,
                                                                 const float2* __restrict__ Xs,
                                                                 const double* __restrict__ F, int64_t ldf,
                                                                 double* __restrict__ R, int64_t ldR) {
  extern __shared__ float2 ds[];  // [P][32]: x_r - x_c across the current edge
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t r = int64_t(blockIdx.x) * 32 + lane;
  const bool valid = r < n;
  float sh[J], sl[J];
#pragma unroll
  for (int j = 0; j < J; ++j) sh[j] = sl[j] = 0.f;
  for (int s = 0; s < 4; ++s) {
    const int c = valid ? col[int64_t(s) * ldr + r] : -1;
    const int64_t e = valid ? vidx[int64_t(s) * ldr + r] : 0;
    __syncthreads();  // the previous edge's differences are consumed
    for (int b = w; b < P; b += kDfWarps) {
      float2 d = make_float2(0.f, 0.f);
      if (valid) {
        const float2 xr = Xs[int64_t(b) * ldr + r];
        d = c >= 0 ? df_sub(xr, Xs[int64_t(b) * ldr + c]) : xr;
      }
      ds[b * 32 + lane] = d;
    }
    __syncthreads();
    const float2* Be = B + e;
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int a = w + j * kDfWarps;
      if (a < P) {
        float h = sh[j], l = sl[j];
        // pairs (b, a) for b < a: index off(b) + a, off(b) = b P - b (b - 1) / 2 - b
        int64_t q = a;
        for (int b = 0; b < a; ++b) {
          df_fma(h, l, Be[q * lde], ds[b * 32 + lane]);
          q += P - b - 1;
        }
        // pairs (a, b) for b >= a: consecutive from off(a) + a
        const float2* Ba = Be + q * lde;
        for (int b = a; b < P; ++b) df_fma(h, l, Ba[int64_t(b - a) * lde], ds[b * 32 + lane]);
        df_renorm(h, l);
        sh[j] = h;
        sl[j] = l;
      }
    }
  }
  if (!valid) return;
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int a = w + j * kDfWarps;
    if (a < P) {
      const double y = double(sh[j]) + double(sl[j]);
      R[int64_t(a) * ldR + r] = F ? F[int64_t(a) * ldf + r] - y : y;
    }
  }
}

}  // namespace

constexpr int kDfMaxP = 16 * kDfWarps;

sg_status resid_prepare(sg_problem* pr, cudaStream_t st) {
  FluxDf& D = pr->fdf;
  if (D.tried || pr->res_mode == 1) return SG_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (st) SG_CUDA(cudaStreamIsCapturing(st, &cs));
  if (cs != cudaStreamCaptureStatusNone) return SG_OK;
  D.tried = true;
  const int P = pr->P, N = pr->N;
  const int npair = P * (P + 1) / 2;
  const int64_t ne = 2LL * N * (N - 1), lde = round_up(ne, 64), ldr = pr->fine.ldr;
  if (P > kDfMaxP || npair > 65535 || pr->n == 0) {
    if (pr->res_mode == 2) {
      set_error("sg_set_refine_residual: double-FP32 edge blocks need P <= 128");
      return SG_ERR_ARG;
    }
    return SG_OK;
  }
  const size_t keep = size_t(npair) * lde * 8 + size_t(P) * ldr * 8;
  const size_t temp = size_t(pr->K) * lde * 8;
  if (pr->res_mode == 0) {
    // automatic: only while the blocks and the build's scratch take at most
    // a quarter of free memory
    size_t fr = 0, tot = 0;
    SG_CUDA(cudaMemGetInfo(&fr, &tot));
    if (keep + temp > fr / 4) return SG_OK;
  }
  SG_TRY(flux_build(pr));  // neighbours and edge numbers of every row
  DevBuf w, dptr, dk, dg, b, xs;
  SG_TRY(w.alloc(temp));
  SG_TRY(flux_values64(pr, w.as<double>(), lde));
  std::vector<int> pptr, pk;
  std::vector<double> pg;
  pair_lists(pr, pptr, pk, pg);
  SG_TRY(dptr.alloc(pptr.size() * 4));
  SG_TRY(dk.alloc(std::max<size_t>(1, pk.size()) * 4));
  SG_TRY(dg.alloc(std::max<size_t>(1, pg.size()) * 8));
  SG_CUDA(cudaMemcpy(dptr.ptr, pptr.data(), pptr.size() * 4, cudaMemcpyHostToDevice));
  if (!pk.empty()) {
    SG_CUDA(cudaMemcpy(dk.ptr, pk.data(), pk.size() * 4, cudaMemcpyHostToDevice));
    SG_CUDA(cudaMemcpy(dg.ptr, pg.data(), pg.size() * 8, cudaMemcpyHostToDevice));
  }
  SG_TRY(b.alloc(size_t(npair) * lde * 8));
  SG_TRY(xs.alloc(size_t(P) * ldr * 8));
  k_edge_blocks_df<<<dim3(unsigned((lde + 127) / 128), unsigned(npair)), 128>>>(
      ne, lde, lde, dptr.as<int>(), dk.as<int>(), dg.as<double>(), w.as<double>(), b.as<float2>());
  note_launch();
  SG_CUDA(cudaGetLastError());
  SG_CUDA(cudaDeviceSynchronize());
  D.npair = npair;
  D.lde = lde;
  D.b = std::move(b);
  D.xs = std::move(xs);
  return SG_OK;
}

sg_status resid_df(sg_problem* pr, const double* F, int64_t ldf, const double* X, int64_t ldx, double* R,
                   int64_t ldR, cudaStream_t st) {
  const FluxDf& D = pr->fdf;
  if (!D.b.ptr) {
    set_error("refinement residual: the double-FP32 edge blocks are not built");
    return SG_ERR_UNSUPPORTED;
  }
  const int P = pr->P;
  const int64_t n = pr->n, ldr = pr->fine.ldr;
  if (n == 0) return SG_OK;
  k_split_df<<<dim3(unsigned((ldr + 255) / 256), unsigned(P)), 256, 0, st>>>(n, ldr, X, ldx, D.xs.as<float2>());
  note_launch();
  SG_CUDA(cudaGetLastError());
  const int need = (P + kDfWarps - 1) / kDfWarps;
  const size_t smem = size_t(P) * 32 * sizeof(float2);
  const unsigned grid = unsigned((n + 31) / 32);
  const int* col = pr->flux.col.as<int>();
  const int* vidx = pr->flux.vidx.as<int>();
  const float2* B = D.b.as<float2>();
  const float2* Xs = D.xs.as<float2>();
#define SG_DF_LAUNCH(JJ)                                                                                       \
  k_resid_flux_df<JJ><<<grid, 32 * kDfWarps, smem, st>>>(n, ldr, P, D.lde, col, vidx, B, Xs, F, ldf, R, ldR)
  if (need <= 2)
    SG_DF_LAUNCH(2);
  else if (need <= 5)
    SG_DF_LAUNCH(5);
  else if (need <= 8)
    SG_DF_LAUNCH(8);
  else if (need <= 11)
    SG_DF_LAUNCH(11);
  else
    SG_DF_LAUNCH(16);
#undef SG_DF_LAUNCH
  note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

sg_status refine_residual(sg_problem* pr, const double* F, int64_t ldf, const double* X, int64_t ldx, double* R,
                          int64_t ldR, cudaStream_t st) {
  SG_TRY(resid_prepare(pr, st));
  if (!pr->fdf.b.ptr || pr->res_mode == 1) return apply_op<double>(pr, false, X, ldx, F, ldf, R, ldR, st);
  size_t slot = 0;
  const bool on = pr->prof.on;
  if (on) SG_TRY(pr->prof.begin(1, st, slot));
  SG_TRY(resid_df(pr, F, ldf, X, ldx, R, ldR, st));
  if (on) SG_TRY(pr->prof.end(slot, st));
  return SG_OK;
}

}  // namespace sg
