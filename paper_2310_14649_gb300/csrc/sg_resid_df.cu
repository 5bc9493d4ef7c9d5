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
constexpr int kDfAhead = 8;  // block entries loaded ahead of their products
constexpr int kDfTileRows = 4;  // node rows of a tile (32 node columns)
constexpr size_t kSmemMax = 227 * 1024;

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

// Flux of one edge group: f[a] = sum_b B_ab d_b for the outputs a = w +
// 8 j of this warp (lane = edge), d in shared memory, the block entries of
// pair (a, b) at index off(min) + max, off(b) = b P - b (b - 1) / 2 - b
template <int J>
__device__ __forceinline__ void edge_flux(const float2* __restrict__ Be, int64_t lde, int P, int w, int lane,
                                          const float2* ds, float (&fh)[J], float (&fl)[J]) {
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int a = w + j * kDfWarps;
    float h = 0.f, l = 0.f;
    if (a < P) {
      // pairs (b, a) for b < a: consecutive b are P - b - 1 pairs apart;
      // eight loads in flight ahead of their products
      const float2* pp = Be + int64_t(a) * lde;
      int b = 0;
      for (; b + kDfAhead <= a; b += kDfAhead) {
        float2 cv[kDfAhead];
#pragma unroll
        for (int u = 0; u < kDfAhead; ++u) {
          cv[u] = __ldg(pp);
          pp += int64_t(P - (b + u) - 1) * lde;
        }
#pragma unroll
        for (int u = 0; u < kDfAhead; ++u) df_fma(h, l, cv[u], ds[(b + u) * 32 + lane]);
      }
      for (; b < a; ++b) {
        df_fma(h, l, __ldg(pp), ds[b * 32 + lane]);
        pp += int64_t(P - b - 1) * lde;
      }
      // pairs (a, b) for b >= a: consecutive from off(a) + a
      for (; b + kDfAhead <= P; b += kDfAhead) {
        float2 cv[kDfAhead];
#pragma unroll
        for (int u = 0; u < kDfAhead; ++u) cv[u] = __ldg(pp + int64_t(u) * lde);
        pp += int64_t(kDfAhead) * lde;
#pragma unroll
        for (int u = 0; u < kDfAhead; ++u) df_fma(h, l, cv[u], ds[(b + u) * 32 + lane]);
      }
      for (; b < P; ++b) {
        df_fma(h, l, __ldg(pp), ds[b * 32 + lane]);
        pp += lde;
      }
      df_renorm(h, l);
    }
    fh[j] = h;
    fl[j] = l;
  }
}

// (y.x, y.y) += sign (h, l) in double-FP32
__device__ __forceinline__ void df_acc(float2* y, float h, float l) {
  float2 v = *y;
  const float s = __fadd_rn(v.x, h);
  const float bb = __fsub_rn(s, v.x);
  const float e = __fadd_rn(__fsub_rn(v.x, __fsub_rn(s, bb)), __fsub_rn(h, bb));
  *y = make_float2(s, __fadd_rn(v.y, __fadd_rn(l, e)));
}

// R = F - A X (R = A X when F is null) on a tile of 32 x TY interior nodes
// (I = i0 + 1 .. i0 + 32, J = j0 + 1 .. j0 + TY; row (J - 1) m + I - 1,
// m = N - 1).  The tile's edges are taken in groups of up to 32 (lane =
// edge): TY rows of horizontal edges (the one west of each node), the
// column of edges east of the tile's last node column, TY + 1 rows of
// vertical edges.  Each edge's flux f = B^e (x_hi - x_lo) is formed once
// and added to the node above or right of it (+f) and subtracted from the
// node below or left (-f) where that node is in the tile, in double-FP32
// accumulators in shared memory.
template <int J, int TY>
__global__ void __launch_bounds__(32 * kDfWarps) k_resid_tile_df(int N, int P, int64_t lde, int64_t ldr,
                                                                 const float2* __restrict__ B,
                                                                 const float2* __restrict__ Xs,
                                                                 const double* __restrict__ F, int64_t ldf,
                                                                 double* __restrict__ R, int64_t ldR) {
  extern __shared__ float2 sm[];
  float2* ds = sm;            // [P][32]: x_hi - x_lo across the group's edges
  float2* y = sm + P * 32;    // [P][TY][32]: the tile's outputs
  const int m = N - 1;
  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * TY;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int idx = threadIdx.x; idx < P * TY * 32; idx += 32 * kDfWarps) y[idx] = make_float2(0.f, 0.f);
  auto xrow = [&](int I, int Jr) { return (I >= 1 && I <= m && Jr >= 1 && Jr <= m) ? (Jr - 1) * m + I - 1 : -1; };
  for (int g = 0; g < 2 * TY + 2; ++g) {
    int64_t e = 0;
    int rlo = -1, rhi = -1, tlo = -1, thi = -1;
    if (g < TY) {
      // horizontal edge between (I - 1, Jr) and (I, Jr)
      const int I = i0 + lane + 1, Jr = j0 + g + 1;
      if (Jr <= m && I <= N) {
        e = int64_t(Jr - 1) * N + I - 1;
        rlo = xrow(I - 1, Jr);
        rhi = xrow(I, Jr);
        if (rhi >= 0) thi = g * 32 + lane;
        if (rlo >= 0 && lane >= 1) tlo = g * 32 + lane - 1;
      }
    } else if (g == TY) {
      // horizontal edge east of the last node column: (I, Jr) - (I + 1, Jr)
      const int I = i0 + 32, Jr = j0 + lane + 1;
      if (lane < TY && Jr <= m && I <= m) {
        e = int64_t(Jr - 1) * N + I;
        rlo = xrow(I, Jr);
        rhi = xrow(I + 1, Jr);
        tlo = lane * 32 + 31;
      }
    } else {
      // vertical edge between (I, Jl) and (I, Jl + 1)
      const int t = g - TY - 1, I = i0 + lane + 1, Jl = j0 + t;
      if (I <= m && Jl + 1 <= N) {
        e = int64_t(N) * m + int64_t(Jl) * m + I - 1;
        rlo = xrow(I, Jl);
        rhi = xrow(I, Jl + 1);
        if (rhi >= 0 && t <= TY - 1) thi = t * 32 + lane;
        if (rlo >= 0 && t >= 1) tlo = (t - 1) * 32 + lane;
      }
    }
    const bool active = thi >= 0 || tlo >= 0;
    if (!active) e = 0;
    __syncthreads();  // the previous group's differences are consumed
    for (int b = w; b < P; b += kDfWarps) {
      float2 d = make_float2(0.f, 0.f);
      if (active) {
        const float2 xh = rhi >= 0 ? Xs[int64_t(b) * ldr + rhi] : make_float2(0.f, 0.f);
        const float2 xl = rlo >= 0 ? Xs[int64_t(b) * ldr + rlo] : make_float2(0.f, 0.f);
        d = df_sub(xh, xl);
      }
      ds[b * 32 + lane] = d;
    }
    __syncthreads();
    float fh[J], fl[J];
    edge_flux<J>(B + e, lde, P, w, lane, ds, fh, fl);
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int a = w + j * kDfWarps;
      if (a < P) {
        float2* ya = y + a * TY * 32;
        if (thi >= 0) df_acc(ya + thi, fh[j], fl[j]);
        __syncwarp();
        if (tlo >= 0) df_acc(ya + tlo, -fh[j], -fl[j]);
        __syncwarp();
      }
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < P * TY * 32; idx += 32 * kDfWarps) {
    const int a = idx / (TY * 32), t = (idx / 32) % TY, l = idx % 32;
    const int r = xrow(i0 + l + 1, j0 + t + 1);
    if (r < 0) continue;
    const float2 v = y[idx];
    const double yv = double(v.x) + double(v.y);
    R[int64_t(a) * ldR + r] = F ? F[int64_t(a) * ldf + r] - yv : yv;
  }
}

}  // namespace

constexpr int kDfMaxP = 16 * kDfWarps;

// the tile kernels' shared memory ((1 + TY) P 32 float2, up to 164 KB)
// above the default 48 KB; set once, before any capture
sg_status df_kernel_attrs() {
  static bool done = false;
  if (done) return SG_OK;
  const int lim = int(kSmemMax);
  SG_CUDA(cudaFuncSetAttribute(k_resid_tile_df<2, kDfTileRows>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  SG_CUDA(cudaFuncSetAttribute(k_resid_tile_df<5, kDfTileRows>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  SG_CUDA(cudaFuncSetAttribute(k_resid_tile_df<8, kDfTileRows>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  SG_CUDA(cudaFuncSetAttribute(k_resid_tile_df<11, kDfTileRows>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  SG_CUDA(cudaFuncSetAttribute(k_resid_tile_df<16, kDfTileRows>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  done = true;
  return SG_OK;
}

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
  SG_TRY(df_kernel_attrs());
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
  const size_t smem = size_t(P) * 32 * (1 + kDfTileRows) * sizeof(float2);
  const int m = pr->N - 1;
  const dim3 grid(unsigned((m + 31) / 32), unsigned((m + kDfTileRows - 1) / kDfTileRows));
  const float2* B = D.b.as<float2>();
  const float2* Xs = D.xs.as<float2>();
#define SG_DF_LAUNCH(JJ) \
  k_resid_tile_df<JJ, kDfTileRows><<<grid, 32 * kDfWarps, smem, st>>>(pr->N, P, D.lde, ldr, B, Xs, F, ldf, R, ldR)
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
