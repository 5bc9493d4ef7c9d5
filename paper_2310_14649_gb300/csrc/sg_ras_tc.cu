// RAS local solves as dense products with explicit local inverses on the
// fifth-generation tensor cores (Sec. 3, Eq. RASsto):
//     z = sum_i R_i^T D_i (I (x) A_{0,i})^{-1} R_i r,
// where D_i keeps the owned nodes, so box i needs only the owned rows of
// A_{0,i}^{-1}: Zowned_i[m][a] = sum_j Ainv_i[m][j] r[idx_i[j]][a] — a
// product of an (owned x overlapped) matrix with the (overlapped x P)
// restricted residual.
//
// Work: the owned rows of every box are cut into tiles of 128 rows (the
// MMA's M), the overlapped nodes into chunks of 32 (K), the P modes padded
// to N (a multiple of 16).  The inverse is stored chunk by chunk in the
// operand layout of the tensor cores, so one bulk copy moves a 16 KB chunk
// from HBM to shared memory; the sequence of all (tile, chunk) pairs is cut
// into one contiguous range per SM (a persistent grid), so every SM streams
// the same number of bytes and a tile is shared by at most two CTAs.
//
// Precision: FP32 operands split into a TF32 high part and the remainder,
// x = xh + xl.  The residual is split once per apply into the stacked
// operand [rh; rl] (2N rows, shared memory), the inverse chunk after its
// arrival, row by row, into tensor memory (the MMA's A operand there, so
// the tensor cores read only the residual from shared memory); per k-step
//     D[:, 0:2N] += Ah [rh; rl]^T,   D[:, 0:N] += Al rh^T
// (kind::tf32, FP32 accumulation in tensor memory) and the epilogue sums
// the two column halves: Ah rh + Ah rl + Al rh, the product to FP32
// accuracy.  The epilogue applies the smoother's Kronecker factor (omega
// G~^{-1} across the modes of a node) before the store.
//
// The inverses are formed once at setup in FP64 from the line-block
// Cholesky factors: the local solve applied to unit right-hand sides, four
// colour classes of boxes (2 x 2 checkerboard) whose overlapped sets are
// disjoint, so one batched solve per class yields every column of every
// box of that class.
#include <algorithm>
#include <cmath>
#include <vector>

#include "sg_kernels.h"

namespace sg {

namespace {

constexpr int kInvKC = 32;                 // overlapped nodes per chunk (K)
constexpr int kInvChunk = 128 * kInvKC;    // floats of one inverse chunk (16 KB)
constexpr int kInvMaxStages = 6;           // chunks in flight
constexpr int kInvThreads = 384;           // 2 copy warps, 2 MMA warps, 4 split warps, 4 epilogue warps
constexpr int kInvDrain = 1 << 24;         // polls of a wait that follows a timed-out one
constexpr size_t kSmemLimit = 227 * 1024;

// index tables of the explicit-inverse data, in ints, in this order
enum InvMeta {
  kTileStart,   // [ntiles + 1]: first chunk of each tile in the global sequence
  kTileBox,     // [ntiles]
  kTileOwned,   // [ntiles][128]: global node of each tile row, -1 for padding
  kBoxChunk0,   // [nbox]: first chunk of the box in the packed residual
  kBoxTile0,    // [nbox]: first tile of the box
  kChunkIdx,    // [bchunks][32]: global nodes of each packed residual chunk, -1 for padding
  kSplitTile,   // [nsplit]: tiles two CTAs accumulate into
  kIdx,         // [nbox][Kp]: overlapped global nodes
  kNov,         // [nbox]: overlapped node counts
  kMetaCount
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return uint64_t((saddr >> 4) & 0x3FFFu) | (uint64_t((lbo >> 4) & 0x3FFFu) << 16) |
         (uint64_t((sbo >> 4) & 0x3FFFu) << 32) | (uint64_t(1) << 46);
}

// kind::tf32 instruction descriptor: D FP32, A and B TF32, both K-major
__host__ __device__ constexpr uint32_t tf32_desc(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

__device__ __forceinline__ void mbar_init(uint64_t* b, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_addr(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(b)), "r"(bytes) : "memory");
}
// polls the phase of parity `parity`; gives up after `limit` polls or when
// another role of the CTA has given up
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, int limit, volatile int* abort) {
  for (int i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(b)), "r"(parity)
        : "memory");
    if (done) return true;
    if (abort && *abort) return false;
  }
  return false;
}
// bulk copy global -> shared, completion counted in bytes on the mbarrier
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void bulk_load_stream(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                                 uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;\n" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_addr(b))
               : "memory");
}
// A operand in tensor memory (row m in lane m, k along the columns)
__device__ __forceinline__ void tc_mma_ta(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
      "r"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
// 32 consecutive columns of this thread's lane
__device__ __forceinline__ void tc_st32(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};\n" ::"r"(taddr),
      "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]), "f"(v[8]), "f"(v[9]),
      "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15]), "f"(v[16]), "f"(v[17]), "f"(v[18]),
      "f"(v[19]), "f"(v[20]), "f"(v[21]), "f"(v[22]), "f"(v[23]), "f"(v[24]), "f"(v[25]), "f"(v[26]), "f"(v[27]),
      "f"(v[28]), "f"(v[29]), "f"(v[30]), "f"(v[31])
      : "memory");
}
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

struct InvArgs {
  float* Z;
  int64_t ld;
  const float* ainv;   // [chunks][kInvChunk]
  const float* bpack;  // [bchunks][2N x kInvKC]
  const int* meta;
  int64_t off[kMetaCount];
  const float* M;      // P x P Kronecker factor (row a: coefficients of output mode a)
  int transform;
  int P, stages, ntiles, tcols;
  int aslots;    // tensor-memory slots of split inverse chunks (64 columns each, from column 0)
  int acc_base;  // first column of the accumulators
  int kch;       // independent accumulation chains per accumulator (k-steps alternate between them)
  int nbuf;      // accumulators (alternating by tile piece)
  int chain_cols;  // columns of one chain: [Ah rh | Ah rl | Al rh], 3N rounded up to 32
  int64_t chunks;
  int* err;
  int wait_limit;
};

// the pieces of this CTA's chunk range: (tile t, chunks [cb, ce) of it)
struct PieceIter {
  const int* ts;
  int64_t g, g1;
  int t;
  __device__ PieceIter(const int* tile_start, int ntiles, int64_t g0, int64_t g1_) : ts(tile_start), g(g0), g1(g1_) {
    int lo = 0, hi = ntiles - 1;  // the last tile starting at or before g0
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (ts[mid] <= g0) lo = mid;
      else hi = mid - 1;
    }
    t = lo;
  }
  __device__ bool next(int& tile, int& cb, int& ce, bool& split) {
    if (g >= g1) return false;
    const int64_t a = ts[t], e = ts[t + 1];
    tile = t;
    cb = int(g - a);
    ce = int(min(g1, e) - a);
    split = cb > 0 || a + ce < e;
    g = a + ce;
    ++t;
    return true;
  }
};

// Persistent kernel, one CTA per SM, chunk range [blockIdx.x * chunks /
// grid, ...).  Roles: warp 0 lane 0 issues the bulk copies of a stage
// (inverse chunk + packed residual chunk); warps 2-5 split the inverse
// chunk, one row per thread, into a tensor-memory slot (high part in
// columns 0-31, remainder in 32-63; the slot of chunk c is free once the
// MMAs of chunk c - aslots completed); lane 0 of warp 1 (and of warp 10
// when there are two chains: each warp issues the k-steps of its chain, so
// the issue of small MMAs runs on two threads) issues the MMAs of a stage
// and commits them to the stage's "empty" barrier and, at the end of a
// tile piece, to the accumulator's "full" barrier; warps
// 6-9 read the accumulator (two in tensor memory, alternating by piece),
// apply the Kronecker factor and store (atomically adding when the tile is
// shared with the neighbouring CTA, whose rows were zeroed by the pack
// kernel; two addends onto zero give the same sum in either order).
// Shared memory:
// stages of {A (raw) 16 KB | packed residual 2N x 32 x 4 B}, the N x N
// factor, barriers.
template <int NB>
__global__ void __launch_bounds__(kInvThreads, 1) k_ras_inv_tc(InvArgs a) {
  constexpr int N = 16 * NB;
  constexpr uint32_t SA = kInvChunk * 4, SB = 2 * N * kInvKC * 4, STAGE = SA + SB;
  extern __shared__ __align__(1024) unsigned char sm[];
  const int S = a.stages;
  float* Ms = reinterpret_cast<float*>(sm + S * STAGE);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + S * STAGE + N * N * 4);
  uint64_t* full = bars;                      // [S] copies landed
  uint64_t* split = bars + kInvMaxStages;     // [S] split done (128 arrivals)
  uint64_t* empty = bars + 2 * kInvMaxStages; // [S] MMAs of the stage done
  uint64_t* accf = bars + 3 * kInvMaxStages;  // [2] accumulator complete
  uint64_t* acce = accf + 2;                  // [2] accumulator read (128 arrivals)
  uint64_t* fin = acce + 2;                   // [2] last MMA of each issuer done
  uint32_t* tslot = reinterpret_cast<uint32_t*>(fin + 2);
  volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int* meta = a.meta;
  const int* tile_start = meta + a.off[kTileStart];
  const int64_t g0 = int64_t(blockIdx.x) * a.chunks / gridDim.x;
  const int64_t g1 = int64_t(blockIdx.x + 1) * a.chunks / gridDim.x;

  if (a.transform)
    for (int e = tid; e < N * N; e += kInvThreads) {
      const int r = e / N, c = e % N;
      Ms[e] = (r < a.P && c < a.P) ? a.M[r * a.P + c] : 0.f;
    }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(tslot)),
                 "r"(a.tcols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < kInvMaxStages; ++s) {
      mbar_init(full + s, 1);
      mbar_init(split + s, 128);
      mbar_init(empty + s, a.kch);
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(accf + k, a.kch);
      mbar_init(acce + k, 128);
    }
    mbar_init(fin, 1);
    mbar_init(fin + 1, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tslot;
  auto fail = [&]() {
    *abort = 1;
    atomicExch(a.err, 1);
  };

  if (warp == 0 || warp == 11) {
    // ---- copies: warp 0 the even chunks, warp 11 the odd ones (a thread
    // has about one bulk copy in issue at a time, so two threads double the
    // copy rate; the stage count is even, so a stage keeps its parity) ----
    const int p = warp == 0 ? 0 : 1;
    if (lane == 0) {
      uint64_t pol;
      asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(pol));
      const int* tile_box = meta + a.off[kTileBox];
      const int* box_chunk0 = meta + a.off[kBoxChunk0];
      PieceIter pi(tile_start, a.ntiles, g0, g1);
      int t, cb, ce;
      bool sp;
      int it = 0;
      bool ok = true;
      while (ok && pi.next(t, cb, ce, sp)) {
        const int64_t gt = tile_start[t];
        const int64_t gb = box_chunk0[tile_box[t]];
        for (int c = cb; c < ce; ++c, ++it) {
          if ((it & 1) != p) continue;
          const int s = it % S;
          if (it >= S && !mbar_wait(empty + s, uint32_t((it / S - 1) & 1), a.wait_limit, abort)) {
            fail();
            ok = false;
            break;
          }
          unsigned char* st = sm + s * STAGE;
          mbar_expect_tx(full + s, SA + SB);
          bulk_load_stream(st, a.ainv + (gt + c) * kInvChunk, SA, full + s, pol);
          bulk_load(st + SA, a.bpack + (gb + c) * (2 * N * kInvKC), SB, full + s);
        }
      }
      // every copy lands before the CTA's shared memory is released (it
      // counts the chunks up to the last one issued, of either parity)
      for (int s = p; s < S && s < it; s += 2) {
        const int u = s + S * ((it - 1 - s) / S);  // last use of stage s
        mbar_wait(full + s, uint32_t((u / S) & 1), kInvDrain, nullptr);
      }
    }
  } else if (warp == 1 || warp == 10) {
    // ---- MMAs: issuer q, k-steps of chain q (all k-steps with one chain) ----
    const int q = warp == 10 ? 1 : 0;
    const int k0 = a.kch == 2 ? 2 * q : 0, k1 = a.kch == 2 ? k0 + 2 : kInvKC / 8;
    if (lane == 0 && q < a.kch) {
      PieceIter pi(tile_start, a.ntiles, g0, g1);
      int t, cb, ce;
      bool sp;
      int it = 0, pc = 0;
      bool ok = true, any = false;
      const uint32_t id2 = tf32_desc(128, 2 * N), id1 = tf32_desc(128, N);
      constexpr uint32_t PLB = 2 * N * 16;
      while (ok && pi.next(t, cb, ce, sp)) {
        const int acc = pc % a.nbuf;
        if (pc >= a.nbuf && !mbar_wait(acce + acc, uint32_t((pc / a.nbuf - 1) & 1), a.wait_limit, abort)) {
          fail();
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        // back-to-back MMAs into one accumulator wait for each other: the
        // high and remainder products, and the k-steps of alternate chains,
        // go to separate columns
        const uint32_t d = tmem + uint32_t(a.acc_base + acc * a.kch * a.chain_cols);
        for (int c = cb; c < ce; ++c, ++it) {
          const int s = it % S;
          if (!mbar_wait(split + s, uint32_t((it / S) & 1), a.wait_limit, abort)) {
            fail();
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
          const uint32_t bb = smem_addr(sm + s * STAGE) + SA;
          const uint32_t ta = tmem + uint32_t(64 * (it % a.aslots));
          const uint32_t dc = d + uint32_t(q * a.chain_cols);
          for (int k8 = k0; k8 < k1; ++k8) {
            const uint64_t db = smem_desc(bb + 2 * k8 * PLB, PLB, 128);
            const uint32_t first = (c == cb && k8 == k0) ? 0u : 1u;
            tc_mma_ta(dc, ta + 8 * k8, db, id2, first);
            tc_mma_ta(dc + 2 * N, ta + 32 + 8 * k8, db, id1, first);
          }
          any = true;
          tc_commit(empty + s);
        }
        if (!ok) break;
        tc_commit(accf + acc);
        ++pc;
      }
      // every MMA completes before tensor memory is freed
      if (any) {
        tc_commit(fin + q);
        mbar_wait(fin + q, 0u, kInvDrain, nullptr);
      }
    }
  } else if (warp < 6) {
    // ---- split of the inverse chunk: row m of the chunk into lane m ----
    const int m = 32 * (warp & 3) + lane;
    const uint32_t trow = tmem + (uint32_t(32 * (warp & 3)) << 16);
    PieceIter pi(tile_start, a.ntiles, g0, g1);
    int t, cb, ce;
    bool sp;
    int it = 0;
    bool ok = true;
    while (ok && pi.next(t, cb, ce, sp)) {
      for (int c = cb; c < ce; ++c, ++it) {
        const int s = it % S;
        bool got = mbar_wait(full + s, uint32_t((it / S) & 1), a.wait_limit, abort);
        // the slot of chunk it - aslots is free once its MMAs completed
        if (got && it >= a.aslots) {
          const int u = it - a.aslots;
          got = mbar_wait(empty + u % S, uint32_t((u / S) & 1), a.wait_limit, abort);
        }
        // the warp converges before the aligned tensor-memory stores
        if (!__all_sync(0xffffffffu, got)) {
          fail();
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const unsigned char* ar = sm + s * STAGE;
        float hi[kInvKC], lo[kInvKC];
#pragma unroll
        for (int q = 0; q < kInvKC / 4; ++q) {
          const float4 v = *reinterpret_cast<const float4*>(ar + q * 2048 + m * 16);
          hi[4 * q] = tf32_hi(v.x);
          hi[4 * q + 1] = tf32_hi(v.y);
          hi[4 * q + 2] = tf32_hi(v.z);
          hi[4 * q + 3] = tf32_hi(v.w);
          lo[4 * q] = v.x - hi[4 * q];
          lo[4 * q + 1] = v.y - hi[4 * q + 1];
          lo[4 * q + 2] = v.z - hi[4 * q + 2];
          lo[4 * q + 3] = v.w - hi[4 * q + 3];
        }
        const uint32_t ta = trow + uint32_t(64 * (it % a.aslots));
        tc_st32(ta, hi);
        tc_st32(ta + 32, lo);
        asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        mbar_arrive(split + s);
      }
    }
  } else {
    // ---- epilogue: rows 32 (warp % 4) + lane of the accumulator ----
    const int lg = warp & 3, m = 32 * lg + lane;
    const int* tile_owned = meta + a.off[kTileOwned];
    PieceIter pi(tile_start, a.ntiles, g0, g1);
    int t, cb, ce;
    bool sp;
    int pc = 0;
    while (pi.next(t, cb, ce, sp)) {
      const int acc = pc % a.nbuf;
      // the warp converges before the aligned tensor-memory loads
      const bool got = mbar_wait(accf + acc, uint32_t((pc / a.nbuf) & 1), a.wait_limit, abort);
      if (!__all_sync(0xffffffffu, got)) {
        fail();
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      float y[N];
      const uint32_t base =
          tmem + (uint32_t(32 * lg) << 16) + uint32_t(a.acc_base + acc * a.kch * a.chain_cols);
#pragma unroll
      for (int j = 0; j < NB; ++j) {
#pragma unroll
        for (int q = 0; q < 16; ++q) y[16 * j + q] = 0.f;
        for (int ch = 0; ch < a.kch; ++ch) {
          float p0[16], p1[16], p2[16];
          const uint32_t cbase = base + uint32_t(ch * a.chain_cols + 16 * j);
          tc_ld16(cbase, p0);
          tc_ld16(cbase + N, p1);
          tc_ld16(cbase + 2 * N, p2);
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
          for (int q = 0; q < 16; ++q) y[16 * j + q] += (p0[q] + p2[q]) + p1[q];
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      mbar_arrive(acce + acc);
      ++pc;
      const int g = tile_owned[int64_t(t) * 128 + m];
      if (g < 0) continue;
      float* zr = a.Z + g;
      if (a.transform) {
        for (int r = 0; r < a.P; ++r) {
          const float4* mr = reinterpret_cast<const float4*>(Ms + r * N);
          float v = 0.f;
#pragma unroll
          for (int b4 = 0; b4 < N / 4; ++b4) {
            const float4 w = mr[b4];
            v = fmaf(w.x, y[4 * b4], v);
            v = fmaf(w.y, y[4 * b4 + 1], v);
            v = fmaf(w.z, y[4 * b4 + 2], v);
            v = fmaf(w.w, y[4 * b4 + 3], v);
          }
          if (sp) atomicAdd(zr + int64_t(r) * a.ld, v);
          else zr[int64_t(r) * a.ld] = v;
        }
      } else {
#pragma unroll
        for (int r = 0; r < N; ++r) {
          if (r < a.P) {
            if (sp) atomicAdd(zr + int64_t(r) * a.ld, y[r]);
            else zr[int64_t(r) * a.ld] = y[r];
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(a.tcols) : "memory");
}

// The residual of every box in the operand layout of its chunks: chunk
// (box b, c) holds, for the overlapped nodes j = 32 c .. 32 c + 31, the
// rows n < N (high parts of r[n][idx_b[j]]) and N + n (remainders), planes
// of 4 nodes (16 bytes per row).  One block per chunk: the gather reads
// runs of consecutive nodes of a mode row into shared memory (one index
// load, then independent loads of the rows), the writes are whole 16-byte
// rows of a plane.  The threads also zero the output rows of the tiles that
// two CTAs accumulate into.
constexpr int kPackThreads = 256;
__global__ void __launch_bounds__(kPackThreads) k_ras_inv_pack(const float* __restrict__ R, int64_t ld, int P, int N,
                                                               int64_t bchunks, InvArgs a, float* __restrict__ bpack,
                                                               int nsplit) {
  __shared__ float tile[96][kInvKC + 1];
  const int* meta = a.meta;
  const int* chunk_idx = meta + a.off[kChunkIdx];
  const int tid = threadIdx.x;
  for (int64_t gc = blockIdx.x; gc < bchunks; gc += gridDim.x) {
    // thread (k, n0): node k of the chunk in every eighth mode row from n0
    const int k = tid % kInvKC, n0 = tid / kInvKC;
    const int gi = chunk_idx[gc * kInvKC + k];
    float v[96 / (kPackThreads / kInvKC)];
#pragma unroll
    for (int i = 0; i < 96 / (kPackThreads / kInvKC); ++i) {
      const int n = n0 + i * (kPackThreads / kInvKC);
      v[i] = (n < P && gi >= 0) ? R[int64_t(n) * ld + gi] : 0.f;
    }
#pragma unroll
    for (int i = 0; i < 96 / (kPackThreads / kInvKC); ++i) {
      const int n = n0 + i * (kPackThreads / kInvKC);
      if (n < N) tile[n][k] = v[i];
    }
    __syncthreads();
    float4* out = reinterpret_cast<float4*>(bpack + gc * (2 * N * kInvKC));
    for (int e = tid; e < (kInvKC / 4) * N; e += kPackThreads) {
      const int q = e / N, n = e % N;
      const float v0 = tile[n][4 * q], v1 = tile[n][4 * q + 1], v2 = tile[n][4 * q + 2], v3 = tile[n][4 * q + 3];
      const float4 h = make_float4(tf32_hi(v0), tf32_hi(v1), tf32_hi(v2), tf32_hi(v3));
      out[q * 2 * N + n] = h;
      out[q * 2 * N + N + n] = make_float4(v0 - h.x, v1 - h.y, v2 - h.z, v3 - h.w);
    }
    __syncthreads();
  }
  const int* split_tile = meta + a.off[kSplitTile];
  const int* tile_owned = meta + a.off[kTileOwned];
  const int64_t nz = int64_t(nsplit) * 128 * P;
  const int64_t stride = int64_t(gridDim.x) * kPackThreads;
  for (int64_t e = blockIdx.x * int64_t(kPackThreads) + tid; e < nz; e += stride) {
    const int c = int(e % P);
    const int64_t r = e / P;
    const int g = tile_owned[int64_t(split_tile[r / 128]) * 128 + int(r % 128)];
    if (g >= 0) a.Z[int64_t(c) * ld + g] = 0.f;
  }
}

// unit right-hand sides of one colour class: R[j][idx_b[j]] = 1 for the
// boxes b of that class (their overlapped sets are disjoint)
__global__ void k_inv_unit_rhs(double* __restrict__ R, int64_t ld, const int* __restrict__ idx,
                               const int* __restrict__ nov, const int* __restrict__ color, int cls, int Kp, int nbox) {
  const int64_t total = int64_t(nbox) * Kp;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
    const int b = int(t / Kp), j = int(t % Kp);
    if (color[b] != cls || j >= nov[b]) continue;
    R[int64_t(j) * ld + idx[size_t(b) * Kp + j]] = 1.0;
  }
}

// Ainv_b[m][j] = Z[j][owned_b[m]] for the boxes of one colour class, into
// the chunk layout: tile box_tile0[b] + m / 128, chunk j / 32, plane
// (j % 32) / 4, row m % 128, word j % 4
__global__ void k_inv_extract(const double* __restrict__ Zs, int64_t ld, float* __restrict__ ainv,
                              const int* __restrict__ meta, InvArgs a, const int* __restrict__ color, int cls,
                              int Mpad, int Kp, int nbox) {
  const int* nov = meta + a.off[kNov];
  const int* box_tile0 = meta + a.off[kBoxTile0];
  const int* tile_start = meta + a.off[kTileStart];
  const int* tile_owned = meta + a.off[kTileOwned];
  const int64_t total = int64_t(nbox) * Mpad * Kp;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
    const int b = int(t / (int64_t(Mpad) * Kp));
    if (color[b] != cls) continue;
    const int64_t rem = t - int64_t(b) * Mpad * Kp;
    const int m = int(rem / Kp), j = int(rem % Kp);
    const int tile = box_tile0[b] + m / 128;
    if (tile >= box_tile0[b + 1]) continue;                 // past the box's last tile
    const int64_t c0 = tile_start[tile];
    if (j >= (tile_start[tile + 1] - c0) * kInvKC) continue;  // past the box's last chunk
    const int g = tile_owned[int64_t(tile) * 128 + m % 128];
    const float v = (g >= 0 && j < nov[b]) ? float(Zs[int64_t(j) * ld + g]) : 0.f;
    ainv[(c0 + j / kInvKC) * kInvChunk + ((j % kInvKC) / 4) * 512 + (m % 128) * 4 + (j % 4)] = v;
  }
}

size_t inv_stage_bytes(int N) { return size_t(kInvChunk) * 4 + 2 * size_t(N) * kInvKC * 4; }
size_t inv_fixed_bytes(int N) { return size_t(N) * N * 4 + (3 * kInvMaxStages + 6) * 8 + 16; }

int inv_stages(int P) {
  const int N = (P + 15) / 16 * 16;
  const size_t room = kSmemLimit - inv_fixed_bytes(N);
  return int(std::min<size_t>(kInvMaxStages, room / inv_stage_bytes(N))) & ~1;  // even: two copy warps
}

template <int NB>
sg_status inv_launch(const InvArgs& args, int grid, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    SG_CUDA(cudaFuncSetAttribute(k_ras_inv_tc<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kSmemLimit)));
    attr = true;
  }
  const size_t smem = args.stages * inv_stage_bytes(16 * NB) + inv_fixed_bytes(16 * NB);
  k_ras_inv_tc<NB><<<unsigned(grid), kInvThreads, smem, st>>>(args);
  note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

InvArgs inv_args(const RasData& D) {
  InvArgs a{};
  a.meta = dp<int>(D.d_inv_meta);
  for (int k = 0; k < kMetaCount; ++k) a.off[k] = D.inv_off[k];
  return a;
}

}  // namespace

// the index list of the widest supported box: 48 x 48 overlapped nodes
constexpr int kInvMaxKp = 48 * 48;
bool ras_inverse_supported(int P) { return P >= 1 && P <= 96 && inv_stages(P) >= 2; }

sg_status ras_inverse_build(sg_problem* pr, Precond& pc, cudaStream_t st) {
  RasData& D = pc.ras;
  if (!ras_inverse_supported(pr->P)) {
    set_error("RAS explicit inverses on tensor cores: P must be in [1, 96]");
    return SG_ERR_UNSUPPORTED;
  }
  D.inv_free();
  const int nbox = D.nbox;
  int nmax = 0, omax = 0;
  std::vector<int> nov(nbox), nown(nbox), color(nbox);
  for (int b = 0; b < nbox; ++b) {
    nov[b] = int(D.idx[b].size());
    nmax = std::max(nmax, nov[b]);
    int o = 0;
    for (int32_t f : D.owned[b]) o += f ? 1 : 0;
    nown[b] = o;
    omax = std::max(omax, o);
    const int bx = b % pc.sx, by = b / pc.sx;
    color[b] = (bx & 1) + 2 * (by & 1);
  }
  // same-colour boxes are a box apart: their overlapped sets stay disjoint
  // when a box is wider than twice the overlap
  const int m = pr->N - 1;
  if (m / pc.sx <= 2 * pc.overlap || m / pc.sy <= 2 * pc.overlap) {
    set_error("RAS explicit inverses: boxes must be wider than twice the overlap");
    return SG_ERR_UNSUPPORTED;
  }
  const int Kp = (nmax + kInvKC - 1) / kInvKC * kInvKC;
  if (Kp > kInvMaxKp) {
    set_error("RAS explicit inverses: overlapped boxes of at most 2,304 nodes");
    return SG_ERR_UNSUPPORTED;
  }
  const int Mpad = (omax + 127) / 128 * 128;
  const int P = pr->P, N = (P + 15) / 16 * 16;
  // tiles (128 owned rows of a box) and chunks (32 overlapped nodes)
  std::vector<int> tile_start{0}, tile_box, tile_owned, box_chunk0(nbox), box_tile0(nbox + 1), chunk_idx, hidx(
      size_t(nbox) * Kp, 0);
  int64_t bchunks = 0;
  int maxlen = 1;
  for (int b = 0; b < nbox; ++b) {
    const int nch = (nov[b] + kInvKC - 1) / kInvKC;
    maxlen = std::max(maxlen, nch);
    box_chunk0[b] = int(bchunks);
    for (int j = 0; j < nch * kInvKC; ++j) chunk_idx.push_back(j < nov[b] ? D.idx[b][j] : -1);
    bchunks += nch;
    box_tile0[b] = int(tile_box.size());
    std::vector<int> own;
    for (int j = 0; j < nov[b]; ++j) {
      hidx[size_t(b) * Kp + j] = D.idx[b][j];
      if (D.owned[b][j]) own.push_back(D.idx[b][j]);
    }
    for (int t = 0; t * 128 < nown[b]; ++t) {
      tile_box.push_back(b);
      tile_start.push_back(tile_start.back() + nch);
      for (int r = 0; r < 128; ++r) tile_owned.push_back(t * 128 + r < nown[b] ? own[t * 128 + r] : -1);
    }
  }
  box_tile0[nbox] = int(tile_box.size());
  const int ntiles = int(tile_box.size());
  const int64_t chunks = tile_start.back();
  // one CTA per SM; each range at least as long as the longest tile, so a
  // tile meets at most two ranges
  int dev = 0, sms = 0;
  SG_CUDA(cudaGetDevice(&dev));
  SG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = int(std::max<int64_t>(1, std::min<int64_t>(sms, chunks / maxlen)));
  std::vector<int> split_tile;
  {
    std::vector<int> pieces(ntiles, 0);
    int t = 0;
    for (int i = 0; i < grid; ++i) {
      const int64_t g0 = int64_t(i) * chunks / grid, g1 = int64_t(i + 1) * chunks / grid;
      while (tile_start[t + 1] <= g0) ++t;
      for (int u = t; u < ntiles && tile_start[u] < g1; ++u) ++pieces[u];
    }
    for (int u = 0; u < ntiles; ++u) {
      if (pieces[u] > 2) {
        set_error("RAS explicit inverses: a tile met more than two chunk ranges");
        return SG_ERR_UNSUPPORTED;
      }
      if (pieces[u] == 2) split_tile.push_back(u);
    }
  }
  // the index tables in one buffer
  std::vector<int> meta;
  const std::vector<int>* parts[kMetaCount] = {&tile_start, &tile_box, &tile_owned, &box_chunk0, &box_tile0,
                                               &chunk_idx,  &split_tile, &hidx, &nov};
  for (int k = 0; k < kMetaCount; ++k) {
    D.inv_off[k] = int64_t(meta.size());
    meta.insert(meta.end(), parts[k]->begin(), parts[k]->end());
    meta.resize((meta.size() + 3) / 4 * 4, 0);
  }
  DevBuf dmeta, dcol, dainv, dbpack;
  SG_TRY(dmeta.alloc(meta.size() * 4));
  SG_TRY(dcol.alloc(color.size() * 4));
  SG_CUDA(cudaMemcpy(dmeta.ptr, meta.data(), meta.size() * 4, cudaMemcpyHostToDevice));
  SG_CUDA(cudaMemcpy(dcol.ptr, color.data(), color.size() * 4, cudaMemcpyHostToDevice));
  SG_TRY(dainv.alloc(size_t(chunks) * kInvChunk * 4));
  SG_TRY(dbpack.alloc(size_t(bchunks) * 2 * N * kInvKC * 4));
  D.d_inv_meta = std::move(dmeta);
  InvArgs ia = inv_args(D);
  const int* dm = dp<int>(D.d_inv_meta);
  // the local solves (FP64, no Kronecker factor) of the unit right-hand sides
  const int64_t ld = pr->ld;
  DevBuf Rs, Zs;
  SG_TRY(Rs.alloc(size_t(nmax) * ld * 8));
  SG_TRY(Zs.alloc(size_t(nmax) * ld * 8));
  for (int cls = 0; cls < 4; ++cls) {
    SG_CUDA(cudaMemsetAsync(Rs.ptr, 0, Rs.bytes, st));
    SG_CUDA(cudaMemsetAsync(Zs.ptr, 0, Zs.bytes, st));
    k_inv_unit_rhs<<<4 * 152, 256, 0, st>>>(dp<double>(Rs), ld, dm + D.inv_off[kIdx], dm + D.inv_off[kNov],
                                            dp<int>(dcol), cls, Kp, nbox);
    note_launch();
    SG_CUDA(cudaGetLastError());
    SG_TRY(ras_apply<double>(pc, pr->n, nmax, dp<double>(Rs), ld, dp<double>(Zs), st, false));
    k_inv_extract<<<4 * 152, 256, 0, st>>>(dp<double>(Zs), ld, dp<float>(dainv), dm, ia, dp<int>(dcol), cls, Mpad,
                                           Kp, nbox);
    note_launch();
    SG_CUDA(cudaGetLastError());
  }
  SG_CUDA(cudaStreamSynchronize(st));
  D.inv_kp = Kp;
  D.inv_n = N;
  D.inv_p = P;
  D.inv_ntiles = ntiles;
  D.inv_grid = grid;
  D.inv_nsplit = int(split_tile.size());
  D.inv_stages = inv_stages(P);
  D.inv_chunks = chunks;
  D.inv_bchunks = bchunks;
  D.d_inv = std::move(dainv);
  D.d_inv_bpack = std::move(dbpack);
  if (!D.d_inv_err.ptr) SG_TRY(D.d_inv_err.alloc(16));
  SG_CUDA(cudaMemset(D.d_inv_err.ptr, 0, 16));
  return SG_OK;
}

sg_status ras_inverse_apply(const Precond& pc, int P, const float* R, int64_t ld, float* Z, const float* M,
                            bool transform, int wait_limit, cudaStream_t st) {
  const RasData& D = pc.ras;
  if (transform && !M) {
    set_error("ras_inverse_apply: the Kronecker factor is not on the device yet");
    return SG_ERR_ARG;
  }
  if (P != D.inv_p || !D.d_inv.ptr) {
    set_error("ras_inverse_apply: the local inverses were built for another number of modes");
    return SG_ERR_ARG;
  }
  // the pack kernel reads R while it zeroes rows of Z
  const float *r0 = R, *r1 = R + int64_t(P) * ld, *z0 = Z, *z1 = Z + int64_t(P) * ld;
  if (r0 < z1 && z0 < r1) {
    set_error("ras_inverse_apply: input and output overlap");
    return SG_ERR_ARG;
  }
  const int N = D.inv_n;
  InvArgs a = inv_args(D);
  a.Z = Z;
  a.ld = ld;
  a.ainv = dp<float>(D.d_inv);
  a.bpack = dp<float>(D.d_inv_bpack);
  a.M = M;
  a.transform = transform ? 1 : 0;
  a.P = P;
  a.stages = D.inv_stages;
  a.ntiles = D.inv_ntiles;
  // tensor memory (512 columns): the split inverse chunks in slots of 64
  // columns from column 0, then the accumulators, each of kch chains of
  // chain_cols columns.  Preferred: two chains, two accumulators, four
  // slots; fewer where 512 columns do not hold them (two chains count more
  // than a second accumulator: a tile piece is 40 chunks of MMAs).
  a.chain_cols = (3 * N + 31) / 32 * 32;
  a.tcols = 512;
  const int shapes[6][3] = {{2, 2, 4}, {2, 2, 2}, {2, 1, 3}, {2, 1, 2}, {1, 1, 4}, {1, 1, 2}};
  a.kch = 0;
  for (const auto& sh : shapes)
    if (64 * sh[2] + sh[0] * sh[1] * a.chain_cols <= 512) {
      a.kch = sh[0];
      a.nbuf = sh[1];
      a.aslots = sh[2];
      break;
    }
  if (!a.kch) {
    set_error("ras_inverse_apply: tensor memory too small for P modes");
    return SG_ERR_UNSUPPORTED;
  }
  a.acc_base = 64 * a.aslots;
  a.chunks = D.inv_chunks;
  a.err = dp<int>(D.d_inv_err);
  a.wait_limit = wait_limit;
  // one block per packed chunk (every chunk's loads in flight at once)
  const int pgrid = int(std::max<int64_t>(1, std::min<int64_t>(D.inv_bchunks, 1 << 30)));
  k_ras_inv_pack<<<unsigned(pgrid), kPackThreads, 0, st>>>(R, ld, P, N, D.inv_bchunks, a, dp<float>(D.d_inv_bpack),
                                                           D.inv_nsplit);
  note_launch();
  SG_CUDA(cudaGetLastError());
  switch (N / 16) {
    case 1: return inv_launch<1>(a, D.inv_grid, st);
    case 2: return inv_launch<2>(a, D.inv_grid, st);
    case 3: return inv_launch<3>(a, D.inv_grid, st);
    case 4: return inv_launch<4>(a, D.inv_grid, st);
    case 5: return inv_launch<5>(a, D.inv_grid, st);
    case 6: return inv_launch<6>(a, D.inv_grid, st);
    default: set_error("ras_inverse_apply: P > 96"); return SG_ERR_ARG;
  }
}

// SG_ERR_TIMEOUT (and the flag cleared) when a completion wait of the
// inverse products ran out since the last check; synchronises the stream
sg_status ras_inverse_check(const Precond& pc, cudaStream_t st) {
  const RasData& D = pc.ras;
  if (!D.d_inv_err.ptr) return SG_OK;
  int e = 0;
  SG_CUDA(cudaMemcpyAsync(&e, D.d_inv_err.ptr, sizeof e, cudaMemcpyDeviceToHost, st));
  SG_CUDA(cudaStreamSynchronize(st));
  if (!e) return SG_OK;
  SG_CUDA(cudaMemsetAsync(D.d_inv_err.ptr, 0, sizeof e, st));
  set_error("RAS: a tensor-core completion wait of the local inverse products timed out");
  return SG_ERR_TIMEOUT;
}

}  // namespace sg
