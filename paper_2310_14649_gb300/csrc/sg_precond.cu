// Device side of the two-grid preconditioner (Sec. 3, Eqs. RASsto, coarse,
// RAS_2L): restricted additive Schwarz local solves, the Kronecker
// stochastic factor, 2h transfer, Galerkin coarse values, AMG V-cycle.
#include <algorithm>
#include <cmath>

#include "sg_kernels.h"
#include "sg_solver.h"

namespace sg {

namespace {

constexpr int kOwnedBit = 1 << 30;
constexpr int kIdxMask = kOwnedBit - 1;

// ---------------------------------------------------------------------------
// RAS local solve: z_owned = (A_{0,i}^{-1} R_i r)_owned for every box i and
// every PCE mode, with the block-tridiagonal Cholesky factor of A_{0,i}:
//   forward  y_j = Linv_j (r_j - Loff_j y_{j-1})
//   backward x_j = Linv_j^T (y_j - Loff_{j+1}^T x_{j+1})
// One CTA per (box, chunk of MC modes); the local block lives in shared
// memory as y[line][slot][mode] with a padded mode stride.  The two W x W
// matrices of each line step are copied into shared memory with cp.async
// two steps ahead (a ring of three buffers), so every step reads only shared
// memory and the copies' latency hides behind two steps of compute.  W is a
// multiple of 4 (16-byte rows).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
// line steps whose matrices are in flight or resident (ring of buffers):
// the default depth and the deepest ring the kernel takes
constexpr int kRasStages = 3;
constexpr int kRasMaxStages = 8;
// cp.async.wait_group with a run-time count (the instruction takes an immediate)
__device__ __forceinline__ void cp_async_wait_dyn(int n) {
  switch (n) {
    case 0: cp_async_wait_group<0>(); break;
    case 1: cp_async_wait_group<1>(); break;
    case 2: cp_async_wait_group<2>(); break;
    case 3: cp_async_wait_group<3>(); break;
    case 4: cp_async_wait_group<4>(); break;
    case 5: cp_async_wait_group<5>(); break;
    default: cp_async_wait_group<6>(); break;
  }
}

template <typename T>
__device__ __forceinline__ void stage_mats(T* dst_off, T* dst_lin, const T* src_off, const T* src_lin, int WW) {
  const int chunks = WW * int(sizeof(T)) / 16;
  for (int c = threadIdx.x; c < chunks; c += blockDim.x) {
    if (src_off) cp_async16(reinterpret_cast<char*>(dst_off) + 16 * c, reinterpret_cast<const char*>(src_off) + 16 * c);
    cp_async16(reinterpret_cast<char*>(dst_lin) + 16 * c, reinterpret_cast<const char*>(src_lin) + 16 * c);
  }
  cp_async_commit();
}

// Box gather / scatter of the tensor-core RAS kernel: slot q of the box
// (line-major, W per line) and mode a, y[q * MS + a]; every thread keeps
// kRasIlp independent global loads in flight.
constexpr int kRasIlp = 8;
template <typename T>
__device__ __forceinline__ void ras_gather(const T* __restrict__ R, int64_t ld, int P, int a0, int MC, int nslot,
                                           int ncols, const int* __restrict__ gbox, T* y, int MS) {
  const int total = nslot * ncols;
  for (int e0 = threadIdx.x; e0 < total; e0 += kRasIlp * blockDim.x) {
    T v[kRasIlp];
#pragma unroll
    for (int u = 0; u < kRasIlp; ++u) {
      const int e = e0 + u * int(blockDim.x);
      v[u] = T(0);
      if (e < total) {
        const int a = e / nslot, q = e - a * nslot;
        const int gi = gbox[q];
        if (gi >= 0 && a < MC && a0 + a < P) v[u] = R[int64_t(a0 + a) * ld + (gi & kIdxMask)];
      }
    }
#pragma unroll
    for (int u = 0; u < kRasIlp; ++u) {
      const int e = e0 + u * int(blockDim.x);
      if (e < total) {
        const int a = e / nslot, q = e - a * nslot;
        y[q * MS + a] = v[u];
      }
    }
  }
}
template <typename T>
__device__ __forceinline__ void ras_scatter(T* __restrict__ Z, int64_t ld, int P, int a0, int MC, int nslot,
                                            const int* __restrict__ gbox, const T* y, int MS) {
  const int total = nslot * MC;
  for (int e0 = threadIdx.x; e0 < total; e0 += kRasIlp * blockDim.x) {
    int gi[kRasIlp];
#pragma unroll
    for (int u = 0; u < kRasIlp; ++u) {
      const int e = e0 + u * int(blockDim.x);
      gi[u] = e < total ? gbox[e % nslot] : -1;
    }
#pragma unroll
    for (int u = 0; u < kRasIlp; ++u) {
      const int e = e0 + u * int(blockDim.x);
      const int a = e / nslot, q = e - a * nslot;
      if (e < total && gi[u] >= 0 && (gi[u] & kOwnedBit) && a0 + a < P)
        Z[int64_t(a0 + a) * ld + (gi[u] & kIdxMask)] = y[q * MS + a];
    }
  }
}

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

// Four lanes own two adjacent rows (t0, t0 + 1) of a line and two adjacent
// modes (a0, a0 + 1): every shared-memory value a lane loads feeds two
// FMAs, the mode pairs are read as one vector, and each lane sums every
// fourth u, so the dependent chain of a step is a quarter of the line width.
template <typename T>
__global__ void k_ras_local(const T* __restrict__ R, int64_t ld, T* __restrict__ Z, int P, int MC,
                            int W, int Lm, const int* __restrict__ nlines, const int* __restrict__ gidx,
                            const T* __restrict__ linv, const T* __restrict__ loff, int stages) {
  using T2 = typename Vec2<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int MCe = (MC + 1) & ~1, MS = MCe + 2, MS2 = MS / 2, WW = W * W;
  T* mats = reinterpret_cast<T*>(smem_raw);  // [stages buffers][off, lin][W*W]
  T* y = mats + 2 * stages * WW;             // [Lm * W][MS]
  T* s = y + size_t(Lm) * W * MS;            // [W][MS]
  T2* y2 = reinterpret_cast<T2*>(y);
  T2* s2 = reinterpret_cast<T2*>(s);
  const int box = blockIdx.x, a0 = blockIdx.y * MC;
  const int nl = nlines[box];
  const int* gbox = gidx + size_t(box) * Lm * W;
  const T* Li = linv + size_t(box) * Lm * WW;
  const T* Lo = loff + size_t(box) * Lm * WW;
  const int nthr = blockDim.x;
  // matrices of sweep step st (forward j = st, backward j = 2 nl - 1 - st)
  auto step_off = [&](int st) -> const T* {
    if (st < nl) return st > 0 ? Lo + size_t(st) * WW : nullptr;
    const int j = 2 * nl - 1 - st;
    return j + 1 < nl ? Lo + size_t(j + 1) * WW : nullptr;
  };
  auto step_lin = [&](int st) -> const T* { return Li + size_t(st < nl ? st : 2 * nl - 1 - st) * WW; };
  // prologue: the first stages - 1 steps' matrices in flight
  for (int st = 0; st < stages - 1; ++st) {
    T* d = mats + (st % stages) * 2 * WW;
    if (st < 2 * nl)
      stage_mats<T>(d, d + WW, step_off(st), step_lin(st), WW);
    else
      cp_async_commit();
  }
  // gather (nodes fastest across threads); padding modes are zero
  const int nslot = nl * W;
  for (int e = threadIdx.x; e < nslot * MCe; e += nthr) {
    int a = e / nslot, q = e - a * nslot;
    int g = gbox[q];
    T v = T(0);
    if (g >= 0 && a < MC && a0 + a < P) v = R[int64_t(a0 + a) * ld + (g & kIdxMask)];
    y[q * MS + a] = v;
  }
  // thread = (row pair tr, mode pair tm, lane q of 4): the four lanes of a
  // group split every sum over u (u = q, q + 4, ...) and meet by shuffles
  const int np = MCe / 2, q = threadIdx.x & 3, grp = threadIdx.x >> 2;
  const int tm = grp % np, tr = grp / np;
  const int t0 = 2 * tr, t1 = t0 + 1;
  const bool act = t0 < W;
  auto reduce4 = [](T2& c0, T2& c1) {
#pragma unroll
    for (int off = 1; off < 4; off <<= 1) {
      c0.x += __shfl_xor_sync(0xffffffffu, c0.x, off);
      c0.y += __shfl_xor_sync(0xffffffffu, c0.y, off);
      c1.x += __shfl_xor_sync(0xffffffffu, c1.x, off);
      c1.y += __shfl_xor_sync(0xffffffffu, c1.y, off);
    }
  };
  for (int st = 0; st < 2 * nl; ++st) {
    cp_async_wait_dyn(stages - 2);
    __syncthreads();
    const T* Lof = mats + (st % stages) * 2 * WW;
    const T* Lin = Lof + WW;
    {  // keep stages - 1 steps ahead in flight (buffer of step st - 1 is free)
      const int nx = st + stages - 1;
      T* d = mats + (nx % stages) * 2 * WW;
      if (nx < 2 * nl)
        stage_mats<T>(d, d + WW, step_off(nx), step_lin(nx), WW);
      else
        cp_async_commit();
    }
    const bool fwd = st < nl;
    const int j = fwd ? st : 2 * nl - 1 - st;
    // s_t = y_jt - sum_u Loff[t][u] y_{j-1,u}  (forward),
    // s_t = y_jt - sum_u Loff[u][t] y_{j+1,u}  (backward, Loff of line j + 1)
    {
      T2 c0, c1;
      c0.x = c0.y = c1.x = c1.y = T(0);
      const bool has_off = fwd ? j > 0 : j + 1 < nl;
      if (act && has_off) {
        const T2* yp = y2 + size_t(fwd ? j - 1 : j + 1) * W * MS2 + tm;
        for (int u = q; u < W; u += 4) {
          const T2 v = yp[u * MS2];
          T p0, p1;
          if (fwd) {
            p0 = Lof[t0 * W + u];
            p1 = Lof[t1 * W + u];
          } else {
            const T2 p = *reinterpret_cast<const T2*>(Lof + u * W + t0);
            p0 = p.x;
            p1 = p.y;
          }
          c0.x -= p0 * v.x;
          c0.y -= p0 * v.y;
          c1.x -= p1 * v.x;
          c1.y -= p1 * v.y;
        }
      }
      reduce4(c0, c1);
      if (act && q < 2) {
        const int t = q == 0 ? t0 : t1;
        const T2 yv = y2[(j * W + t) * MS2 + tm];
        T2 r = q == 0 ? c0 : c1;
        r.x += yv.x;
        r.y += yv.y;
        s2[t * MS2 + tm] = r;
      }
    }
    __syncthreads();
    // y_jt = sum_{u <= t} Linv[t][u] s_u  (forward),
    // x_jt = sum_{u >= t} Linv[u][t] s_u  (backward)
    {
      T2 c0, c1;
      c0.x = c0.y = c1.x = c1.y = T(0);
      if (act) {
        if (fwd) {
          for (int u = q; u <= t1; u += 4) {
            const T2 v = s2[u * MS2 + tm];
            const T p1 = Lin[t1 * W + u];
            c1.x += p1 * v.x;
            c1.y += p1 * v.y;
            if (u <= t0) {
              const T p0 = Lin[t0 * W + u];
              c0.x += p0 * v.x;
              c0.y += p0 * v.y;
            }
          }
        } else {
          for (int u = t0 + q; u < W; u += 4) {
            const T2 v = s2[u * MS2 + tm];
            const T2 p = *reinterpret_cast<const T2*>(Lin + u * W + t0);  // Linv[u][t0], Linv[u][t1]
            c0.x += p.x * v.x;
            c0.y += p.x * v.y;
            if (u >= t1) {
              c1.x += p.y * v.x;
              c1.y += p.y * v.y;
            }
          }
        }
      }
      reduce4(c0, c1);
      if (act && q < 2) y2[(j * W + (q == 0 ? t0 : t1)) * MS2 + tm] = q == 0 ? c0 : c1;
    }
  }
  cp_async_wait_all();
  __syncthreads();
  // scatter owned nodes
  for (int e = threadIdx.x; e < nslot * MC; e += nthr) {
    int aa = e / nslot, q = e - aa * nslot;
    int g = gbox[q];
    if (g >= 0 && (g & kOwnedBit) && a0 + aa < P) Z[int64_t(a0 + aa) * ld + (g & kIdxMask)] = y[q * MS + aa];
  }
}

// ---------------------------------------------------------------------------
// RAS local solve on the tensor cores (FP32 data).  Each line step is two
// small dense products, (W x W)(W x MC): the off-diagonal coupling and the
// triangular inverse (zero above its diagonal, so the full tile product is
// the same sum).  The FMA kernel above spends eight instructions in nine on
// loads, loop control and lane reductions; here every warp owns one 16 x 8
// tile of the W x MC result and runs m16n8k8 TF32 MMAs over the K = W
// terms, each operand split into a TF32 high part and a TF32 remainder
// (hi*hi + hi*lo + lo*hi, the dropped lo*lo term ~2^-22 relative), with FP32
// accumulation: FP32-level accuracy at a tenth of the instructions.  The
// products sit inside a recurrence of 2 x lines dependent steps, so
// warp-level MMA fits better than a tensor-memory round trip per step.
// Measured on GB300 (64 boxes of 36 x 36 nodes, P = 35) it is the slower
// of the two: 0.30 ms against 0.20 ms for the FMA kernel, whose cost is the
// latency of the dependent steps rather than its instruction count; it is
// kept as an option (ras_kernel = 1).  Layout: y[line * W + t][mode] with a
// mode stride MS = 8 x odd (B-fragment loads hit 32 distinct banks).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t tf32_of(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_of(x);
  lo = tf32_of(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C (16 x 8 tile at rows m0.., cols n0..) = A (W x W, A[t][u] = M[t*W+u], or
// M[u*W+t] when transposed) times B (B[u][n] = Bm[u*MS + n]); rows and
// terms at or past W read as zero.
__device__ __forceinline__ void tile_3xtf32(float (&c)[4], const float* M, bool trans, const float* Bm, int MS,
                                            int W, int m0, int n0, int g, int tig) {
  float big[4] = {0.f, 0.f, 0.f, 0.f}, small[4] = {0.f, 0.f, 0.f, 0.f};
  const int r0 = m0 + g, r1 = r0 + 8;
  for (int k0 = 0; k0 < W; k0 += 8) {
    const int u0 = k0 + tig, u1 = u0 + 4;
    auto at = [&](int t, int u) -> float {
      if (t >= W || u >= W) return 0.f;
      return trans ? M[u * W + t] : M[t * W + u];
    };
    const float av[4] = {at(r0, u0), at(r1, u0), at(r0, u1), at(r1, u1)};
    const float bv[2] = {u0 < W ? Bm[u0 * MS + n0 + g] : 0.f, u1 < W ? Bm[u1 * MS + n0 + g] : 0.f};
    uint32_t ah[4], al[4], bh[2], bl[2];
#pragma unroll
    for (int i = 0; i < 4; ++i) tf32_split(av[i], ah[i], al[i]);
#pragma unroll
    for (int i = 0; i < 2; ++i) tf32_split(bv[i], bh[i], bl[i]);
    mma_tf32(small, al, bh);
    mma_tf32(small, ah, bl);
    mma_tf32(big, ah, bh);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) c[i] = big[i] + small[i];
}

__global__ void k_ras_local_tc(const float* __restrict__ R, int64_t ld, float* __restrict__ Z, int P, int MC, int W,
                               int Lm, const int* __restrict__ nlines, const int* __restrict__ gidx,
                               const float* __restrict__ linv, const float* __restrict__ loff, int stages, int MS) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int WW = W * W;
  const int Nt = (MC + 7) / 8, Np = 8 * Nt;
  float* mats = reinterpret_cast<float*>(smem_raw);  // [stages][off, lin][W*W]
  float* y = mats + 2 * stages * WW;                  // [Lm * W][MS]
  float* sb = y + size_t(Lm) * W * MS;                // [W][MS]
  const int box = blockIdx.x, a0 = blockIdx.y * MC;
  const int nl = nlines[box];
  const int* gbox = gidx + size_t(box) * Lm * W;
  const float* Li = linv + size_t(box) * Lm * WW;
  const float* Lo = loff + size_t(box) * Lm * WW;
  auto step_off = [&](int st) -> const float* {
    if (st < nl) return st > 0 ? Lo + size_t(st) * WW : nullptr;
    const int j = 2 * nl - 1 - st;
    return j + 1 < nl ? Lo + size_t(j + 1) * WW : nullptr;
  };
  auto step_lin = [&](int st) -> const float* { return Li + size_t(st < nl ? st : 2 * nl - 1 - st) * WW; };
  for (int st = 0; st < stages - 1; ++st) {
    float* d = mats + (st % stages) * 2 * WW;
    if (st < 2 * nl)
      stage_mats<float>(d, d + WW, step_off(st), step_lin(st), WW);
    else
      cp_async_commit();
  }
  // gather; padding modes (up to Np) are zero
  const int nslot = nl * W;
  ras_gather<float>(R, ld, P, a0, MC, nslot, Np, gbox, y, MS);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, tig = lane & 3;
  const int m0 = (warp / Nt) * 16, n0 = (warp % Nt) * 8;
  const int r0 = m0 + g, r1 = r0 + 8, c0 = n0 + 2 * tig;
  // warps past the (W / 16) x (MC / 8) tiles only help with the gather and scatter
  const bool tile_warp = warp < ((W + 15) / 16) * Nt;
  for (int st = 0; st < 2 * nl; ++st) {
    cp_async_wait_dyn(stages - 2);
    __syncthreads();
    const float* Lof = mats + (st % stages) * 2 * WW;
    const float* Lin = Lof + WW;
    {
      const int nx = st + stages - 1;
      float* d = mats + (nx % stages) * 2 * WW;
      if (nx < 2 * nl)
        stage_mats<float>(d, d + WW, step_off(nx), step_lin(nx), WW);
      else
        cp_async_commit();
    }
    const bool fwd = st < nl;
    const int j = fwd ? st : 2 * nl - 1 - st;
    const float* yj = y + size_t(j) * W * MS;
    // s = y_j - Loff y_{j-1} (forward), s = y_j - Loff_{j+1}^T y_{j+1} (backward)
    {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      const bool has_off = fwd ? j > 0 : j + 1 < nl;
      if (tile_warp && has_off)
        tile_3xtf32(c, Lof, !fwd, y + size_t(fwd ? j - 1 : j + 1) * W * MS, MS, W, m0, n0, g, tig);
      if (tile_warp && r0 < W) {
        sb[r0 * MS + c0] = yj[r0 * MS + c0] - c[0];
        sb[r0 * MS + c0 + 1] = yj[r0 * MS + c0 + 1] - c[1];
      }
      if (tile_warp && r1 < W) {
        sb[r1 * MS + c0] = yj[r1 * MS + c0] - c[2];
        sb[r1 * MS + c0 + 1] = yj[r1 * MS + c0 + 1] - c[3];
      }
    }
    __syncthreads();
    // y_j = Linv s (forward), x_j = Linv^T s (backward)
    if (tile_warp) {
      float c[4];
      tile_3xtf32(c, Lin, !fwd, sb, MS, W, m0, n0, g, tig);
      float* yw = y + size_t(j) * W * MS;
      if (r0 < W) {
        yw[r0 * MS + c0] = c[0];
        yw[r0 * MS + c0 + 1] = c[1];
      }
      if (r1 < W) {
        yw[r1 * MS + c0] = c[2];
        yw[r1 * MS + c0 + 1] = c[3];
      }
    }
  }
  cp_async_wait_all();
  __syncthreads();
  ras_scatter<float>(Z, ld, P, a0, MC, nslot, gbox, y, MS);
}

// In-place per-node transform z_r <- M z_r with a P x P matrix M (the
// stochastic factor omega G~^{-1}).  128 nodes per CTA staged in shared memory.
template <typename T>
__global__ void k_node_transform(T* __restrict__ Z, int64_t ld, int64_t n, int P, const T* __restrict__ M,
                                 T* __restrict__ Z2, int64_t stride2, const int* __restrict__ j2) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ms = reinterpret_cast<T*>(smem_raw);  // P x P
  T* zs = Ms + size_t(P) * P;               // P x 128
  for (int e = threadIdx.x; e < P * P; e += blockDim.x) Ms[e] = M[e];
  const int64_t r = int64_t(blockIdx.x) * 128 + threadIdx.x;
  const bool valid = r < n;
  for (int b = 0; b < P; ++b) zs[b * 128 + threadIdx.x] = valid ? Z[int64_t(b) * ld + r] : T(0);
  __syncthreads();
  if (!valid) return;
  // optional copy into slot j2 (device index) of a vector array, same ld
  T* z2 = Z2 ? Z2 + int64_t(*j2) * stride2 : nullptr;
  for (int a = 0; a < P; ++a) {
    T acc = T(0);
    for (int b = 0; b < P; ++b) acc += Ms[a * P + b] * zs[b * 128 + threadIdx.x];
    Z[int64_t(a) * ld + r] = acc;
    if (z2) z2[int64_t(a) * ld + r] = acc;
  }
}

// FP32 node transform with the node's P inputs in registers (PM >= P, a
// compile-time bound): M^T staged in shared memory as [b][a] rows padded to
// a multiple of 4, so one 16-byte load feeds four outputs; a smem load per
// four FMAs instead of two per FMA.
template <int PM>
__global__ void __launch_bounds__(128) k_node_transform_reg(float* __restrict__ Z, int64_t ld, int64_t n, int P,
                                                            const float* __restrict__ M, float* __restrict__ Z2,
                                                            int64_t stride2, const int* __restrict__ j2) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* MT = reinterpret_cast<float*>(smem_raw);  // [P][P4]
  const int P4 = (P + 3) & ~3;
  for (int e = threadIdx.x; e < P * P4; e += blockDim.x) {
    const int b = e / P4, a = e - b * P4;
    MT[e] = a < P ? M[a * P + b] : 0.f;
  }
  const int64_t r = int64_t(blockIdx.x) * 128 + threadIdx.x;
  const bool valid = r < n;
  float z[PM];
#pragma unroll
  for (int b = 0; b < PM; ++b) z[b] = (valid && b < P) ? Z[int64_t(b) * ld + r] : 0.f;
  __syncthreads();
  if (!valid) return;
  float* z2 = Z2 ? Z2 + int64_t(*j2) * stride2 : nullptr;
  for (int a = 0; a < P; a += 4) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int b = 0; b < PM; ++b) {
      if (b < P) {
        const float4 m = *reinterpret_cast<const float4*>(MT + b * P4 + a);
        acc.x = fmaf(m.x, z[b], acc.x);
        acc.y = fmaf(m.y, z[b], acc.y);
        acc.z = fmaf(m.z, z[b], acc.z);
        acc.w = fmaf(m.w, z[b], acc.w);
      }
    }
    const float o[4] = {acc.x, acc.y, acc.z, acc.w};
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (a + i < P) {
        Z[int64_t(a + i) * ld + r] = o[i];
        if (z2) z2[int64_t(a + i) * ld + r] = o[i];
      }
  }
}

// Coarse ELL values of all K terms from the fine ELL values by the RAP plan.
__global__ void k_coarse_values(const double* __restrict__ fine, int64_t fine_kstride, const int* __restrict__ rp,
                                const int64_t* __restrict__ src, const double* __restrict__ w, int64_t npos,
                                int K, double* __restrict__ v64, float* __restrict__ v32) {
  int64_t total = npos * K;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
    int k = int(t / npos);
    int64_t q = t - int64_t(k) * npos;
    const double* fk = fine + int64_t(k) * fine_kstride;
    double acc = 0.0;
    for (int u = rp[q]; u < rp[q + 1]; ++u) acc += w[u] * fk[src[u]];
    v64[t] = acc;
    v32[t] = float(acc);
  }
}

// Frobenius products <A_k, A_0> over the ELL values (one CTA per k).
__global__ void k_frob(const double* __restrict__ V, int64_t kstride, int K, double* __restrict__ out) {
  __shared__ double red[32];
  const int k = blockIdx.x;
  double acc = 0.0;
  for (int64_t e = threadIdx.x; e < kstride; e += blockDim.x) acc += V[int64_t(k) * kstride + e] * V[e];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) out[k] = acc;
  }
}

// CSR SpMM over P columns (mode-major blocks):
//   op 0: Y = A X;  op 1: Y += A X;  op 2: Y = B - A X
// G lanes (a power of two <= 32) share each row's entries and meet by
// shuffles; rows per 128-thread block = 128 / G.
template <typename T>
__global__ void __launch_bounds__(128) k_spmm(int64_t nrows, const int* __restrict__ rp, const int* __restrict__ ci,
                                              const T* __restrict__ v, const T* __restrict__ X, int64_t ldx,
                                              const T* __restrict__ B, int64_t ldb, T* __restrict__ Y, int64_t ldy,
                                              int op, int G) {
  const int grp = threadIdx.x / G, lane = threadIdx.x - grp * G;
  const int64_t i = blockIdx.x * int64_t(128 / G) + grp;
  const int a = blockIdx.y;
  const bool live = i < nrows;
  const T* x = X + int64_t(a) * ldx;
  T acc = T(0);
  if (live)
    for (int t = rp[i] + lane; t < rp[i + 1]; t += G) acc += v[t] * x[ci[t]];
  for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (!live || lane != 0) return;
  T* y = Y + int64_t(a) * ldy + i;
  if (op == 0)
    *y = acc;
  else if (op == 1)
    *y += acc;
  else
    *y = B[int64_t(a) * ldb + i] - acc;
}

// Y = diag(d) X  (op 0)   or   Y += diag(d) X  (op 1)
template <typename T>
__global__ void k_diag(int64_t n, const T* __restrict__ d, const T* __restrict__ X, int64_t ldx, T* __restrict__ Y,
                       int64_t ldy, int op) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int a = blockIdx.y;
  if (i >= n) return;
  T v = d[i] * X[int64_t(a) * ldx + i];
  if (op == 0)
    Y[int64_t(a) * ldy + i] = v;
  else
    Y[int64_t(a) * ldy + i] += v;
}

// Coarsest AMG level: X = A^{-1} B with the explicit FP64 inverse.
template <typename T>
__global__ void k_dense_solve(int n, const double* __restrict__ Ainv, const T* __restrict__ B, int64_t ldb,
                              T* __restrict__ X, int64_t ldx) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int a = blockIdx.y;
  if (i >= n) return;
  double acc = 0.0;
  for (int j = 0; j < n; ++j) acc += Ainv[int64_t(i) * n + j] * double(B[int64_t(a) * ldb + j]);
  X[int64_t(a) * ldx + i] = T(acc);
}

// ---------------------------------------------------------------------------
// V-cycle phases with a group of G lanes per sparse row.  The levels below
// the coarse operator are small and their restriction rows long (17 to 55
// entries on the 2h grid of a 256^2 mesh), so one thread per row spends its
// time in a chain of dependent loads; here the G lanes of a group share a
// row's entries and meet by shuffles.  The Jacobi steps are folded into the
// neighbouring products, so a V-cycle over L levels is 4 (L - 1) + 1
// launches.  Per row i of level l and mode a (D = l1 diagonal):
//   kDown      t = b - A (D^{-1} b),  x = D^{-1} b
//   kRestrict  b_{l+1} = R t
//   kProlong   x += P x~_{l+1},  x~_{l+1} = x_{l+1} + D_{l+1}^{-1} t_{l+1}
//              (x_{l+1} alone when l+1 is the coarsest level)
//   kResid     t = b - A x
//   kFinal     out = x + D^{-1} (b - A x)      (out must not alias x)
// ---------------------------------------------------------------------------
enum AmgOp { kDown, kRestrict, kProlong, kResid, kFinal };

template <typename T>
struct AmgPhase {
  int n = 0, G = 1, P = 1;
  const int* rp = nullptr;
  const int* ci = nullptr;
  const T* v = nullptr;
  const T* X = nullptr;   // gathered vector (b for kDown, t for kRestrict, x_{l+1} for kProlong, x otherwise)
  int64_t ldx = 0;
  const T* Xd = nullptr;  // kProlong: D_{l+1}^{-1}; NULL when l+1 is the coarsest level
  const T* Xt = nullptr;  // kProlong: t_{l+1} (ld ldx)
  const T* d = nullptr;   // D_l^{-1} (kDown, kFinal; gathered by kDown)
  const T* B = nullptr;   // b_l (kDown, kResid, kFinal)
  int64_t ldb = 0;
  T* Y = nullptr;         // t (kDown, kResid), b_{l+1}, x (kProlong, +=), out (kFinal)
  int64_t ldy = 0;
  T* Y2 = nullptr;        // kDown: x = D^{-1} b (ld ldy)
};

// MB modes per thread group: the row's pattern and values are read once
// for MB right-hand sides (blockIdx.y covers modes MB y .. MB y + MB - 1)
template <typename T, int OP, int MB>
__global__ void __launch_bounds__(128) k_amg_phase(const __grid_constant__ AmgPhase<T> p) {
  const int G = p.G;
  const int grp = threadIdx.x / G, lane = threadIdx.x - grp * G;
  const int i = blockIdx.x * (128 / G) + grp;
  const int64_t a0 = int64_t(blockIdx.y) * MB;
  const int nm = int(min(int64_t(MB), int64_t(p.P) - a0));
  const bool live = i < p.n;
  T acc[MB];
#pragma unroll
  for (int m = 0; m < MB; ++m) acc[m] = T(0);
  if (live) {
    const int e1 = p.rp[i + 1];
    for (int e = p.rp[i] + lane; e < e1; e += G) {
      const int j = p.ci[e];
      const T v = p.v[e];
      T dj = T(0);
      if (OP == kDown || (OP == kProlong && p.Xd)) dj = OP == kDown ? p.d[j] : p.Xd[j];
#pragma unroll
      for (int m = 0; m < MB; ++m) {
        if (m < nm) {
          const T* X = p.X + (a0 + m) * p.ldx;
          T g;
          if (OP == kDown)
            g = dj * X[j];
          else if (OP == kProlong)
            g = p.Xd ? X[j] + dj * p.Xt[(a0 + m) * p.ldx + j] : X[j];
          else
            g = X[j];
          acc[m] += v * g;
        }
      }
    }
  }
#pragma unroll
  for (int m = 0; m < MB; ++m)
    for (int o = G >> 1; o > 0; o >>= 1) acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], o);
  if (!live || lane != 0) return;
#pragma unroll
  for (int m = 0; m < MB; ++m) {
    if (m >= nm) break;
    const int64_t a = a0 + m;
    T* y = p.Y + a * p.ldy + i;
    if (OP == kDown) {
      const T bi = p.B[a * p.ldb + i];
      *y = bi - acc[m];
      p.Y2[a * p.ldy + i] = p.d[i] * bi;
    } else if (OP == kRestrict) {
      *y = acc[m];
    } else if (OP == kProlong) {
      *y += acc[m];
    } else if (OP == kResid) {
      *y = p.B[a * p.ldb + i] - acc[m];
    } else {
      *y = p.X[a * p.ldx + i] + p.d[i] * (p.B[a * p.ldb + i] - acc[m]);
    }
  }
}

// the phase kernel with the largest MB in {1, 2, 4, 8} that still leaves
// about one wave of resident threads (152 SMs x 2048) of (row, mode group)
// lane groups
template <typename T, int OP>
cudaError_t amg_phase_launch(const AmgPhase<T>& p, cudaStream_t st) {
  const int rows = 128 / p.G;
  const int64_t lanes_per_mode_group = int64_t(p.n) * p.G;
  int MB = 8;
  while (MB > 1 && lanes_per_mode_group * ((p.P + MB - 1) / MB) < 152 * 2048) MB >>= 1;
  const dim3 grid(unsigned((p.n + rows - 1) / rows), unsigned((p.P + MB - 1) / MB));
  switch (MB) {
    case 8: k_amg_phase<T, OP, 8><<<grid, 128, 0, st>>>(p); break;
    case 4: k_amg_phase<T, OP, 4><<<grid, 128, 0, st>>>(p); break;
    case 2: k_amg_phase<T, OP, 2><<<grid, 128, 0, st>>>(p); break;
    default: k_amg_phase<T, OP, 1><<<grid, 128, 0, st>>>(p); break;
  }
  note_launch();
  return cudaGetLastError();
}

// Coarsest level with a warp per row: x = A_c^{-1} b (explicit FP64 inverse)
template <typename T>
__global__ void k_dense_solve_warp(int n, const double* __restrict__ Ainv, const T* __restrict__ B, int64_t ldb,
                                   T* __restrict__ X, int64_t ldx) {
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const int64_t a = blockIdx.y;
  if (row >= n) return;  // whole warps leave together
  double acc = 0.0;
  for (int j = lane; j < n; j += 32) acc += Ainv[int64_t(row) * n + j] * double(B[a * ldb + j]);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) X[a * ldx + row] = T(acc);
}

template <typename T> const T* dv(const DevBuf& b64, const DevBuf& b32);
template <> const double* dv<double>(const DevBuf& b64, const DevBuf&) { return b64.as<double>(); }
template <> const float* dv<float>(const DevBuf&, const DevBuf& b32) { return b32.as<float>(); }

}  // namespace

// ---------------------------------------------------------------------------
template <typename T>
sg_status spmm(const DevCsr& A, const T* X, int64_t ldx, const T* B, int64_t ldb, T* Y, int64_t ldy, int P,
               int op, cudaStream_t st) {
  if (A.n == 0) return SG_OK;
  // about two entries per lane on an average row, while rows x columns x
  // lanes stays within about two waves of resident threads (152 SMs x 2048)
  const int64_t avg = (A.nnz + A.n - 1) / A.n;
  int G = 1;
  while (G < 32 && 2 * G < avg && A.n * int64_t(P) * (2 * G) <= 2 * 152 * 2048) G <<= 1;
  const int rows = 128 / G;
  dim3 grid(unsigned((A.n + rows - 1) / rows), unsigned(P));
  k_spmm<T><<<grid, 128, 0, st>>>(A.n, A.rowptr.as<int>(), A.col.as<int>(), dv<T>(A.v64, A.v32), X, ldx, B, ldb, Y,
                                  ldy, op, G); note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

template <typename T>
sg_status ras_apply(const Precond& pc, int64_t n, int P, const T* R, int64_t ld, T* Z, cudaStream_t st,
                    bool transform, Profiler* prof) {
  const RasData& D = pc.ras;
  if (sizeof(T) == 4 && pc.ras_kernel == 2 && D.d_inv.ptr) {
    // explicit local inverses on tcgen05, the Kronecker factor fused
    size_t slot = 0;
    const bool timed = prof && prof->on;
    if (timed) SG_TRY(prof->begin(4, st, slot));
    SG_TRY(ras_inverse_apply(pc, P, reinterpret_cast<const float*>(R), ld, reinterpret_cast<float*>(Z),
                             reinterpret_cast<const float*>(pc.gtinv32.ptr), transform, pc.wait_limit, st));
    if (timed) SG_TRY(prof->end(slot, st));
    return SG_OK;
  }
  if (sizeof(T) == 4 && pc.ras_kernel == 1) {
    // tensor-core kernel: 8 modes per CTA by default (one 8-wide MMA tile;
    // 64 boxes x 5 chunks of a 35-mode problem are 320 CTAs of 73 KB, all
    // resident at once)
    const int MC = pc.ras_modes > 0 ? std::min(pc.ras_modes, P) : std::min(8, P);
    const int Nt = (MC + 7) / 8;
    int MS = 8 * Nt;
    if (MS % 16 == 0) MS += 8;
    const int Mt = (D.wmax + 15) / 16;
    const int stages = pc.ras_stages > 0 ? pc.ras_stages : kRasStages;
    const size_t smem =
        (2 * size_t(stages) * D.wmax * D.wmax + (size_t(D.lmax) + 1) * D.wmax * MS) * sizeof(float);
    const int threads = std::max(32 * Mt * Nt, 256);
    if (32 * Mt * Nt <= 1024 && smem <= 227 * 1024) {
      static bool attr = false;
      if (!attr) {
        SG_CUDA(cudaFuncSetAttribute(k_ras_local_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        attr = true;
      }
      dim3 grid(unsigned(D.nbox), unsigned((P + MC - 1) / MC));
      size_t slot = 0;
      const bool timed = prof && prof->on;
      if (timed) SG_TRY(prof->begin(4, st, slot));
      k_ras_local_tc<<<grid, threads, smem, st>>>(reinterpret_cast<const float*>(R), ld, reinterpret_cast<float*>(Z),
                                                  P, MC, D.wmax, D.lmax, D.d_nlines.as<int>(), D.d_gidx.as<int>(),
                                                  D.linv32.as<float>(), D.loff32.as<float>(), stages, MS);
      note_launch();
      SG_CUDA(cudaGetLastError());
      if (timed) SG_TRY(prof->end(slot, st));
      if (transform) SG_TRY(node_transform<T>(Z, ld, n, P, dv<T>(pc.gtinv64, pc.gtinv32), st));
      return SG_OK;
    }
  }
  // FMA kernel: modes per CTA at most what shared memory holds next to the
  // ring of line matrices (depths 3 to 8 measured the same at 256^2; a
  // given depth gives way to more modes per CTA unless it was asked for)
  const size_t per_mode = (size_t(D.lmax) * D.wmax + D.wmax) * sizeof(T);
  const size_t mat = 2 * size_t(D.wmax) * D.wmax * sizeof(T);
  int stages = pc.ras_stages > 0 ? pc.ras_stages : kRasStages;
  auto fit_for = [&](int stg) -> int {
    const size_t fixed = size_t(stg) * mat;
    if (fixed + 4 * per_mode > 227 * 1024) return 0;
    return int(std::max<size_t>(2, ((227 * 1024 - fixed) / per_mode - 2) & ~size_t(1)));
  };
  if (pc.ras_stages <= 0)
    while (stages > 2 && (fit_for(stages) < std::min(P, 18) || fit_for(stages) == 0)) --stages;
  const size_t fixed = size_t(stages) * mat;
  const int fit = std::max(2, fit_for(stages));
  const int by_threads = std::max(2, (1024 / std::max(2, D.wmax)) & ~1);  // 4 (W/2) (MC/2) <= 1024
  int maxmc = std::min(fit, by_threads);
  if (pc.ras_modes > 0) maxmc = std::min(maxmc, pc.ras_modes);
  int nchunk = (P + maxmc - 1) / maxmc;
  // about 18 modes per CTA measured best on GB300 (64 boxes of 36^2 nodes)
  if (pc.ras_modes <= 0) nchunk = std::max(nchunk, (P + 17) / 18);
  const int MC = (P + nchunk - 1) / nchunk;
  const int MCe = (MC + 1) & ~1;
  // 4 lanes per (row pair, mode pair), whole warps (the shuffles need them)
  const int threads = ((4 * (D.wmax / 2) * (MCe / 2)) + 31) & ~31;
  const size_t smem = (size_t(D.lmax) * D.wmax + D.wmax) * (MCe + 2) * sizeof(T) + fixed;
  static bool attr[2] = {false, false};
  if (!attr[sizeof(T) == 8]) {
    SG_CUDA(cudaFuncSetAttribute(k_ras_local<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    attr[sizeof(T) == 8] = true;
  }
  if (smem > 227 * 1024) {
    set_error("RAS: overlapped box too large for the shared-memory local solve");
    return SG_ERR_UNSUPPORTED;
  }
  dim3 grid(unsigned(D.nbox), unsigned(nchunk));
  size_t slot = 0;
  const bool timed = prof && prof->on;
  if (timed) SG_TRY(prof->begin(sizeof(T) == 8 ? 5 : 4, st, slot));
  k_ras_local<T><<<grid, threads, smem, st>>>(R, ld, Z, P, MC, D.wmax, D.lmax, D.d_nlines.as<int>(),
                                              D.d_gidx.as<int>(), dv<T>(D.linv64, D.linv32),
                                              dv<T>(D.loff64, D.loff32), stages); note_launch();
  SG_CUDA(cudaGetLastError());
  if (timed) SG_TRY(prof->end(slot, st));
  if (transform) SG_TRY(node_transform<T>(Z, ld, n, P, dv<T>(pc.gtinv64, pc.gtinv32), st));
  return SG_OK;
}

template <int PM>
static sg_status node_transform_reg(float* Z, int64_t ld, int64_t n, int P, const float* M, cudaStream_t st, float* Z2,
                                    int64_t stride2, const int* j2) {
  const size_t smem = size_t(P) * ((P + 3) & ~3) * sizeof(float);
  k_node_transform_reg<PM><<<unsigned((n + 127) / 128), 128, smem, st>>>(Z, ld, n, P, M, Z2, stride2, j2);
  note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

template <typename T>
sg_status node_transform(T* Z, int64_t ld, int64_t n, int P, const T* M, cudaStream_t st, T* Z2, int64_t stride2,
                         const int* j2) {
  if (!M) {
    set_error("node_transform: the Kronecker factor is not on the device yet");
    return SG_ERR_ARG;
  }
  if (sizeof(T) == 4 && P <= 64) {
    float* Zf = reinterpret_cast<float*>(Z);
    const float* Mf = reinterpret_cast<const float*>(M);
    float* Z2f = reinterpret_cast<float*>(Z2);
    if (P <= 16) return node_transform_reg<16>(Zf, ld, n, P, Mf, st, Z2f, stride2, j2);
    if (P <= 40) return node_transform_reg<40>(Zf, ld, n, P, Mf, st, Z2f, stride2, j2);
    return node_transform_reg<64>(Zf, ld, n, P, Mf, st, Z2f, stride2, j2);
  }
  const size_t smem = (size_t(P) * P + size_t(P) * 128) * sizeof(T);
  static bool attr[2] = {false, false};
  if (!attr[sizeof(T) == 8]) {
    SG_CUDA(cudaFuncSetAttribute(k_node_transform<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    attr[sizeof(T) == 8] = true;
  }
  k_node_transform<T><<<unsigned((n + 127) / 128), 128, smem, st>>>(Z, ld, n, P, M, Z2, stride2, j2); note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

// One V(1,1) cycle with l1-Jacobi on every column, from a zero guess.
// Level buffers: b (rhs), x (solution), t (temporary), each [P][ld_l].
// The result goes to `out` (ld `ldo`), or to x_0 when out is NULL.
template <typename T>
sg_status amg_vcycle(const AmgHier& H, AmgWork<T>& w, int P, cudaStream_t st, T* out, int64_t ldo) {
  const int nl = int(H.size());
  if (!out) {
    out = w.x[0];
    ldo = H[0].ld;
  }
  if (H.fused && nl >= 2 && P > 0) {
    auto lanes = [P](const DevCsr& M) {
      // about two entries per lane on an average row, while rows x modes x
      // lanes stays within about two waves of resident threads (152 SMs x 2048)
      const int64_t avg = M.n > 0 ? (M.nnz + M.n - 1) / M.n : 1;
      int G = 1;
      while (G < 32 && 2 * G < avg && M.n * int64_t(P) * (2 * G) <= 2 * 152 * 2048) G <<= 1;
      return G;
    };
    auto phase = [&](const DevCsr& M) {
      AmgPhase<T> p;
      p.n = int(M.n);
      p.P = P;
      p.G = lanes(M);
      p.rp = M.rowptr.as<int>();
      p.ci = M.col.as<int>();
      p.v = dv<T>(M.v64, M.v32);
      return p;
    };
    for (int l = 0; l < nl - 1; ++l) {
      const AmgLevel& L = H[l];
      AmgPhase<T> p = phase(L.A);
      p.X = w.b[l];
      p.ldx = L.ld;
      p.d = dv<T>(L.dinv64, L.dinv32);
      p.B = w.b[l];
      p.ldb = L.ld;
      p.Y = w.t[l];
      p.Y2 = w.x[l];
      p.ldy = L.ld;
      SG_CUDA((amg_phase_launch<T, kDown>(p, st)));
      AmgPhase<T> q = phase(L.R);
      q.X = w.t[l];
      q.ldx = L.ld;
      q.Y = w.b[l + 1];
      q.ldy = H[l + 1].ld;
      SG_CUDA((amg_phase_launch<T, kRestrict>(q, st)));
    }
    {
      const AmgLevel& L = H[nl - 1];
      dim3 g(unsigned((L.n + 3) / 4), unsigned(P));
      k_dense_solve_warp<T><<<g, 128, 0, st>>>(int(L.n), H.coarsest_inv64.as<double>(), w.b[nl - 1], L.ld,
                                               w.x[nl - 1], L.ld); note_launch();
      SG_CUDA(cudaGetLastError());
    }
    for (int l = nl - 2; l >= 0; --l) {
      const AmgLevel& L = H[l];
      const AmgLevel& Ln = H[l + 1];
      AmgPhase<T> p = phase(L.Pm);
      p.X = w.x[l + 1];
      p.ldx = Ln.ld;
      if (l + 1 < nl - 1) {
        p.Xd = dv<T>(Ln.dinv64, Ln.dinv32);
        p.Xt = w.t[l + 1];
      }
      p.Y = w.x[l];
      p.ldy = L.ld;
      SG_CUDA((amg_phase_launch<T, kProlong>(p, st)));
      AmgPhase<T> q = phase(L.A);
      q.X = w.x[l];
      q.ldx = L.ld;
      q.B = w.b[l];
      q.ldb = L.ld;
      q.d = dv<T>(L.dinv64, L.dinv32);
      if (l > 0 || out == w.x[0]) {
        q.Y = w.t[l];
        q.ldy = L.ld;
        SG_CUDA((amg_phase_launch<T, kResid>(q, st)));
      } else {
        q.Y = out;
        q.ldy = ldo;
        SG_CUDA((amg_phase_launch<T, kFinal>(q, st)));
      }
    }
    if (out == w.x[0]) {
      // in place: the last smoothing step on its own
      const AmgLevel& L0 = H[0];
      dim3 g(unsigned((L0.n + 127) / 128), unsigned(P));
      k_diag<T><<<g, 128, 0, st>>>(L0.n, dv<T>(L0.dinv64, L0.dinv32), w.t[0], L0.ld, w.x[0], L0.ld, 1); note_launch();
      SG_CUDA(cudaGetLastError());
    }
    return SG_OK;
  }
  for (int l = 0; l < nl - 1; ++l) {
    const AmgLevel& L = H[l];
    dim3 g(unsigned((L.n + 127) / 128), unsigned(P));
    k_diag<T><<<g, 128, 0, st>>>(L.n, dv<T>(L.dinv64, L.dinv32), w.b[l], L.ld, w.x[l], L.ld, 0); note_launch();
    SG_CUDA(cudaGetLastError());
    SG_TRY(spmm<T>(L.A, w.x[l], L.ld, w.b[l], L.ld, w.t[l], L.ld, P, 2, st));
    SG_TRY(spmm<T>(L.R, w.t[l], L.ld, nullptr, 0, w.b[l + 1], H[l + 1].ld, P, 0, st));
  }
  {
    const AmgLevel& L = H[nl - 1];
    dim3 g(unsigned((L.n + 127) / 128), unsigned(P));
    k_dense_solve<T><<<g, 128, 0, st>>>(int(L.n), H.coarsest_inv64.as<double>(), w.b[nl - 1], L.ld, w.x[nl - 1],
                                        L.ld); note_launch();
    SG_CUDA(cudaGetLastError());
  }
  for (int l = nl - 2; l >= 0; --l) {
    const AmgLevel& L = H[l];
    dim3 g(unsigned((L.n + 127) / 128), unsigned(P));
    SG_TRY(spmm<T>(L.Pm, w.x[l + 1], H[l + 1].ld, nullptr, 0, w.x[l], L.ld, P, 1, st));
    SG_TRY(spmm<T>(L.A, w.x[l], L.ld, w.b[l], L.ld, w.t[l], L.ld, P, 2, st));
    k_diag<T><<<g, 128, 0, st>>>(L.n, dv<T>(L.dinv64, L.dinv32), w.t[l], L.ld, w.x[l], L.ld, 1); note_launch();
    SG_CUDA(cudaGetLastError());
  }
  if (out != w.x[0])
    SG_CUDA(cudaMemcpy2DAsync(out, ldo * sizeof(T), w.x[0], H[0].ld * sizeof(T), H[0].n * sizeof(T), P,
                              cudaMemcpyDeviceToDevice, st));
  return SG_OK;
}

sg_status precond_setup_coarse_plan(sg_problem* pr, Precond& pc, const CoarsePlan& plan) {
  CoarseData& C = pc.co;
  const int K = pr->K, S = C.ell.S;
  const int64_t npos = int64_t(S) * C.ldc;
  DevBuf rp, src, w;
  SG_TRY(rp.alloc(plan.rp.size() * 4));
  SG_TRY(src.alloc(std::max<size_t>(1, plan.src.size()) * 8));
  SG_TRY(w.alloc(std::max<size_t>(1, plan.w.size()) * 8));
  SG_CUDA(cudaMemcpy(rp.ptr, plan.rp.data(), plan.rp.size() * 4, cudaMemcpyHostToDevice));
  if (!plan.src.empty()) {
    SG_CUDA(cudaMemcpy(src.ptr, plan.src.data(), plan.src.size() * 8, cudaMemcpyHostToDevice));
    SG_CUDA(cudaMemcpy(w.ptr, plan.w.data(), plan.w.size() * 8, cudaMemcpyHostToDevice));
  }
  SG_TRY(C.ell.v64.alloc(size_t(K) * npos * 8));
  SG_TRY(C.ell.v32.alloc(size_t(K) * npos * 4));
  k_coarse_values<<<4 * 152, 256>>>(pr->fine.v64.as<double>(), int64_t(pr->fine.S) * pr->fine.ldr, rp.as<int>(),
                                    src.as<int64_t>(), w.as<double>(), npos, K, C.ell.v64.as<double>(),
                                    C.ell.v32.as<float>()); note_launch();
  SG_CUDA(cudaGetLastError());
  SG_CUDA(cudaDeviceSynchronize());
  SG_TRY(build_triple_tables(pr, C.tri, S));
  return SG_OK;
}

sg_status apply_attrs_init();

sg_status kernel_attrs_init() {
  static bool done = false;
  if (done) return SG_OK;
  SG_CUDA(cudaFuncSetAttribute(k_ras_local<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  SG_CUDA(cudaFuncSetAttribute(k_ras_local<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  SG_CUDA(cudaFuncSetAttribute(k_node_transform<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  SG_CUDA(cudaFuncSetAttribute(k_node_transform<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  SG_TRY(apply_attrs_init());
  done = true;
  return SG_OK;
}

sg_status frobenius_weights(sg_problem* pr, std::vector<double>& w) {
  DevBuf out;
  SG_TRY(out.alloc(size_t(pr->K) * 8));
  const int64_t kstride = int64_t(pr->fine.S) * pr->fine.ldr;
  k_frob<<<pr->K, 256>>>(pr->fine.v64.as<double>(), kstride, pr->K, out.as<double>()); note_launch();
  SG_CUDA(cudaGetLastError());
  w.resize(pr->K);
  SG_CUDA(cudaMemcpy(w.data(), out.ptr, size_t(pr->K) * 8, cudaMemcpyDeviceToHost));
  return SG_OK;
}

#define INST(T)                                                                                           \
  template sg_status spmm<T>(const DevCsr&, const T*, int64_t, const T*, int64_t, T*, int64_t, int, int,  \
                             cudaStream_t);                                                               \
  template sg_status ras_apply<T>(const Precond&, int64_t, int, const T*, int64_t, T*, cudaStream_t, bool,        \
                                  Profiler*);                                                                      \
  template sg_status node_transform<T>(T*, int64_t, int64_t, int, const T*, cudaStream_t, T*, int64_t, const int*);                \
  template sg_status amg_vcycle<T>(const AmgHier&, AmgWork<T>&, int, cudaStream_t, T*, int64_t);
INST(float)
INST(double)
#undef INST

}  // namespace sg
