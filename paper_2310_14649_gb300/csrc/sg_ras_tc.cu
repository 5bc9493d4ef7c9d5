// RAS local solves as dense products with explicit local inverses on the
// fifth-generation tensor cores (Sec. 3, Eq. RASsto):
//     z = sum_i R_i^T D_i (I (x) A_{0,i})^{-1} R_i r,
// where D_i keeps the owned nodes, so box i needs only the owned rows of
// A_{0,i}^{-1}: Zowned_i[m][a] = sum_j Ainv_i[m][j] r[idx_i[j]][a] — a
// product of an (owned x overlapped) matrix with the (overlapped x P)
// restricted residual.
//
// Shape.  One tcgen05.mma costs an SM about the same time for any N up to
// 256 (about 140 cycles for M = 128, K = 8 TF32), so the long dimension
// goes into N: the owned rows of a box are cut into tiles of 256 rows (the
// MMA's N, operand B: the inverse), the residual's modes are the MMA's M
// (operand A, 128 rows), the overlapped nodes are K, in chunks of 16.  The
// inverse is stored chunk by chunk in the operand layout, so one bulk copy
// moves a 16 KB chunk from HBM to shared memory; the sequence of all
// (tile, chunk) pairs is cut into one contiguous range per SM (a persistent
// grid), so every SM streams the same number of bytes and a tile is shared
// by at most two CTAs.
//
// Precision: FP32 operands split into a TF32 high part and the remainder,
// x = xh + xl.  The residual is split once per apply: with 2N <= 128 padded
// modes one operand [rh; rl] (rows a and N + a), else two operands rh, rl.
// The inverse chunk is split in shared memory after its arrival (high part
// in place, remainder in a ring beside it).  Per k-step
//     D += [rh; rl] Ah^T + [rh; rl] Al^T          (2N <= 128)
//     D1 += rh Ah^T + rh Al^T,  D2 += rl Ah^T      (otherwise)
// (kind::tf32, FP32 accumulation in tensor memory, lanes = modes, columns
// = rows of the inverse); the epilogue adds the two halves (rh A + rl A,
// the product to FP32 accuracy), applies the smoother's Kronecker factor
// (omega G~^{-1} across the modes of a node) and stores.
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

constexpr int kInvRows = 256;              // owned rows per tile: the MMA's N
constexpr int kInvKC = 16;                 // overlapped nodes per chunk (K)
constexpr int kInvChunk = kInvRows * kInvKC;  // floats of one inverse chunk (16 KB)
constexpr int kInvAop = 128 * kInvKC;      // floats of one residual operand tile (8 KB)
constexpr int kInvMaxStages = 6;           // chunks in flight
constexpr int kInvMaxLo = 3;               // ring of inverse remainders
constexpr int kInvThreads = 352;           // 2 copy warps, MMA warp, 4 split warps, 4 epilogue warps
constexpr int kInvDrain = 1 << 24;         // polls of a wait that follows a timed-out one
constexpr size_t kSmemLimit = 227 * 1024;

// index tables of the explicit-inverse data, in ints, in this order
enum InvMeta {
  kTileStart,   // [ntiles + 1]: first chunk of each tile in the global sequence
  kTileBox,     // [ntiles]
  kTileOwned,   // [ntiles][256]: global node of each tile row, -1 for padding
  kBoxChunk0,   // [nbox]: first chunk of the box in the packed residual
  kBoxTile0,    // [nbox]: first tile of the box
  kChunkIdx,    // [bchunks][16]: global nodes of each packed residual chunk, -1 for padding
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
// another role of the CTA has given up.  sleep_ns > 0 backs off between
// polls: for long waits off the critical path, whose polling would take
// issue slots from the warps that share the scheduler.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, int limit, volatile int* abort,
                                          unsigned sleep_ns = 0) {
  for (int i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(b)), "r"(parity)
        : "memory");
    if (done) return true;
    if (abort && *abort) return false;
    if (sleep_ns) __nanosleep(sleep_ns);
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
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
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
  const float* apack;  // [bchunks][nop][kInvAop]: the residual operand tiles
  const int* meta;
  int64_t off[kMetaCount];
  const float* M;      // P x P Kronecker factor (row a: coefficients of output mode a)
  int transform;
  int P, stages, nlo, ntiles;
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
// grid, ...): chunk `it` of the CTA is global chunk g0 + it.  Roles (lane 0
// where one thread acts):
//  * warps 0 and 10 copy the even and the odd chunks (a thread keeps about
//    one bulk copy in issue at a time): the inverse chunk and the residual
//    operand tile(s) of its box chunk into a stage;
//  * warps 2-5 split the inverse chunk, high part in place, remainder into
//    the ring slot of the chunk (free once the MMAs of chunk it - nlo
//    completed);
//  * warp 1 issues the MMAs of a chunk and commits them to the stage's and
//    the slot's barriers and, at the end of a tile piece, to the
//    accumulator's "full" barrier;
//  * warps 6-9 read the accumulator 32 rows at a time (lane = mode, column
//    = row), pass it through shared memory so that a thread holds a row's
//    modes, apply the Kronecker factor and store (atomically adding when
//    the tile is shared with the neighbouring CTA, whose rows were zeroed
//    by the pack kernel; two addends onto zero give the same sum in either
//    order).
// Shared memory: stages of {inverse chunk (raw, then high part) 16 KB |
// residual operand(s) 8 or 16 KB}, the remainder ring, the N x N factor,
// the 2 x 32 x (N + 1) epilogue staging, barriers.
template <int NB>
__global__ void __launch_bounds__(kInvThreads, 1) k_ras_inv_tc(InvArgs a) {
  constexpr int N = 16 * NB;                 // padded modes
  constexpr bool STACK = 2 * N <= 128;       // [rh; rl] in one operand
  constexpr int NOP = STACK ? 1 : 2;         // residual operand tiles per chunk
  constexpr uint32_t SI = kInvChunk * 4, SAOP = NOP * kInvAop * 4, STAGE = SI + SAOP;
  constexpr int YS = N + 1;                  // epilogue staging row stride
  extern __shared__ __align__(1024) unsigned char sm[];
  const int S = a.stages, NL = a.nlo;
  unsigned char* lo_ring = sm + S * STAGE;
  float* Ms = reinterpret_cast<float*>(lo_ring + NL * SI);
  float* Ys = Ms + N * N;                    // [2][32][YS]
  uint64_t* bars = reinterpret_cast<uint64_t*>(Ys + 2 * 32 * YS + ((2 * 32 * YS) & 1));
  uint64_t* full = bars;                     // [S] copies landed
  uint64_t* empty = full + kInvMaxStages;    // [S] MMAs of the stage done
  uint64_t* split = empty + kInvMaxStages;   // [NL] remainder written (128 arrivals)
  uint64_t* lofree = split + kInvMaxLo;      // [NL] MMAs reading the slot done
  uint64_t* accf = lofree + kInvMaxLo;       // [2] accumulator complete
  uint64_t* acce = accf + 2;                 // [2] accumulator read (128 arrivals)
  uint64_t* fin = acce + 2;                  // last MMA done
  uint32_t* tslot = reinterpret_cast<uint32_t*>(fin + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);
  volatile int* ewait = abort + 1;           // [4] per epilogue warp: its wait succeeded
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int* meta = a.meta;
  const int* tile_start = meta + a.off[kTileStart];
  const int64_t g0 = int64_t(blockIdx.x) * a.chunks / gridDim.x;
  const int64_t g1 = int64_t(blockIdx.x + 1) * a.chunks / gridDim.x;
  const int nch = int(g1 - g0);
  const int nbuf = STACK ? 2 : 1;            // accumulators: 256 columns each, or D1 and D2 of one

  if (a.transform)
    for (int e = tid; e < N * N; e += kInvThreads) {
      const int r = e / N, c = e % N;
      Ms[e] = (r < a.P && c < a.P) ? a.M[r * a.P + c] : 0.f;
    }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;\n" ::"r"(smem_addr(tslot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < kInvMaxStages; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    for (int s = 0; s < kInvMaxLo; ++s) {
      mbar_init(split + s, 128);
      mbar_init(lofree + s, 1);
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(accf + k, 1);
      mbar_init(acce + k, 128);
    }
    mbar_init(fin, 1);
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

  if (warp == 0 || warp == 10) {
    // ---- copies of the even (warp 0) or odd (warp 10) chunks; S is even,
    // so a stage keeps its parity ----
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
          mbar_expect_tx(full + s, STAGE);
          bulk_load_stream(st, a.ainv + (g0 + it) * kInvChunk, SI, full + s, pol);
          bulk_load(st + SI, a.apack + (gb + c) * (NOP * kInvAop), SAOP, full + s);
        }
      }
      // every copy lands before the CTA's shared memory is released (it
      // counts the chunks up to the last one issued, of either parity)
      for (int s = p; s < S && s < it; s += 2) {
        const int u = s + S * ((it - 1 - s) / S);  // last use of stage s
        mbar_wait(full + s, uint32_t((u / S) & 1), kInvDrain, nullptr);
      }
    }
  } else if (warp == 1) {
    // ---- MMAs ----
    if (lane == 0) {
      PieceIter pi(tile_start, a.ntiles, g0, g1);
      int t, cb, ce;
      bool sp;
      int it = 0, pc = 0;
      bool ok = true, any = false;
      const uint32_t idesc = tf32_desc(128, kInvRows);
      constexpr uint32_t PLA = 128 * 16, PLB = kInvRows * 16;
      while (ok && pi.next(t, cb, ce, sp)) {
        const int acc = pc % nbuf;
        if (pc >= nbuf && !mbar_wait(acce + acc, uint32_t((pc / nbuf - 1) & 1), a.wait_limit, abort)) {
          fail();
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t d1 = tmem + uint32_t(256 * acc), d2 = tmem + 256u;
        for (int c = cb; c < ce; ++c, ++it) {
          const int s = it % S, l = it % NL;
          // the split of chunk it follows the arrival of its stage
          if (!mbar_wait(split + l, uint32_t((it / NL) & 1), a.wait_limit, abort)) {
            fail();
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
          const uint32_t bh = smem_addr(sm + s * STAGE), ap = bh + SI, bl = smem_addr(lo_ring + l * SI);
#pragma unroll
          for (int k8 = 0; k8 < kInvKC / 8; ++k8) {
            const uint64_t dbh = smem_desc(bh + 2 * k8 * PLB, PLB, 128);
            const uint64_t dbl = smem_desc(bl + 2 * k8 * PLB, PLB, 128);
            const uint64_t da = smem_desc(ap + 2 * k8 * PLA, PLA, 128);
            const uint32_t first = (c == cb && k8 == 0) ? 0u : 1u;
            tc_mma(d1, da, dbh, idesc, first);
            tc_mma(d1, da, dbl, idesc, 1u);
            if (!STACK) tc_mma(d2, da + ((kInvAop * 4) >> 4), dbh, idesc, first);
          }
          any = true;
          tc_commit(empty + s);
          tc_commit(lofree + l);
        }
        if (!ok) break;
        tc_commit(accf + acc);
        ++pc;
      }
      // every MMA completes before tensor memory is freed
      if (any) {
        tc_commit(fin);
        mbar_wait(fin, 0u, kInvDrain, nullptr);
      }
    }
  } else if (warp < 6) {
    // ---- split of the inverse chunk: high part in place, remainder in the ring ----
    const int sid = tid - 64;
    for (int it = 0; it < nch; ++it) {
      const int s = it % S, l = it % NL;
      bool got = mbar_wait(full + s, uint32_t((it / S) & 1), a.wait_limit, abort);
      if (got && it >= NL) got = mbar_wait(lofree + l, uint32_t((it / NL - 1) & 1), a.wait_limit, abort);
      if (!got) {
        fail();
        break;
      }
      float4* ar = reinterpret_cast<float4*>(sm + s * STAGE);
      float4* al = reinterpret_cast<float4*>(lo_ring + l * SI);
#pragma unroll
      for (int q = 0; q < kInvChunk / 4 / 128; ++q) {
        const int e = sid + 128 * q;
        const float4 v = ar[e];
        const float4 h = make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z), tf32_hi(v.w));
        ar[e] = h;
        al[e] = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
      }
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      mbar_arrive(split + l);
    }
  } else {
    // ---- epilogue: lane l of the accumulator = mode part l ----
    const int et = tid - 192;                  // 0..127
    const int l = 32 * (warp & 3) + lane;      // this thread's tensor-memory lane
    const int part = STACK ? (l < N ? 0 : (l < 2 * N ? 1 : 2)) : (l < N ? 0 : 2);
    const int am = part == 1 ? l - N : l;      // mode of the lane
    const int r = et & 31, gq = et >> 5;       // row within a block of 32, output group
    const int* tile_owned = meta + a.off[kTileOwned];
    PieceIter pi(tile_start, a.ntiles, g0, g1);
    int t, cb, ce;
    bool sp;
    int pc = 0;
    while (pi.next(t, cb, ce, sp)) {
      const int acc = pc % nbuf;
      const bool got = mbar_wait(accf + acc, uint32_t((pc / nbuf) & 1), a.wait_limit, abort, 256);
      // the four warps agree before the aligned tensor-memory loads and the
      // named barriers below: all go on or all stop
      const bool wok = __all_sync(0xffffffffu, got);
      if (lane == 0) ewait[warp & 3] = wok ? 1 : 0;
      asm volatile("bar.sync 1, 128;\n" ::: "memory");
      if (!(ewait[0] && ewait[1] && ewait[2] && ewait[3])) {
        fail();
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t base = tmem + (uint32_t(32 * (warp & 3)) << 16);
      for (int blk = 0; blk < kInvRows / 32; ++blk) {
        float v[32];
        tc_ld16(base + uint32_t(256 * acc + 32 * blk), v);
        tc_ld16(base + uint32_t(256 * acc + 32 * blk + 16), v + 16);
        if (!STACK) {
          float w[32];
          tc_ld16(base + uint32_t(256 + 32 * blk), w);
          tc_ld16(base + uint32_t(256 + 32 * blk + 16), w + 16);
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
          for (int q = 0; q < 32; ++q) v[q] += w[q];
        } else {
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        }
        if (blk == kInvRows / 32 - 1) {
          asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
          mbar_arrive(acce + acc);
        }
        if (part < 2) {
          float* y = Ys + part * 32 * YS + am;
#pragma unroll
          for (int q = 0; q < 32; ++q) y[q * YS] = v[q];
        }
        asm volatile("bar.sync 1, 128;\n" ::: "memory");
        // thread (r, gq): row blk * 32 + r, outputs gq, gq + 4, ...
        const int g = tile_owned[int64_t(t) * kInvRows + blk * 32 + r];
        if (g >= 0) {
          float yr[N];
#pragma unroll
          for (int b = 0; b < N; ++b) yr[b] = STACK ? Ys[r * YS + b] + Ys[32 * YS + r * YS + b] : Ys[r * YS + b];
          float* zr = a.Z + g;
          if (a.transform) {
            for (int o = gq; o < a.P; o += 4) {
              const float4* mr = reinterpret_cast<const float4*>(Ms + o * N);
              float x = 0.f;
#pragma unroll
              for (int b4 = 0; b4 < N / 4; ++b4) {
                const float4 m4 = mr[b4];
                x = fmaf(m4.x, yr[4 * b4], x);
                x = fmaf(m4.y, yr[4 * b4 + 1], x);
                x = fmaf(m4.z, yr[4 * b4 + 2], x);
                x = fmaf(m4.w, yr[4 * b4 + 3], x);
              }
              if (sp) atomicAdd(zr + int64_t(o) * a.ld, x);
              else zr[int64_t(o) * a.ld] = x;
            }
          } else {
#pragma unroll
            for (int o = 0; o < N; ++o) {
              if ((o & 3) == gq && o < a.P) {
                if (sp) atomicAdd(zr + int64_t(o) * a.ld, yr[o]);
                else zr[int64_t(o) * a.ld] = yr[o];
              }
            }
          }
        }
        asm volatile("bar.sync 1, 128;\n" ::: "memory");
      }
      ++pc;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;\n" ::"r"(tmem) : "memory");
}

// The residual operand tiles of every box chunk: chunk (box b, c) covers
// the overlapped nodes j = 16 c .. 16 c + 15; tile rows are modes (with
// 2N <= 128: rows n < P the high parts of r[n][idx_b[j]], rows N + n the
// remainders; else tile 0 the high parts, tile 1 the remainders), planes
// of 4 nodes (16 bytes per row); the padding rows stay zero from setup.
// One block per chunk: the gather reads runs of consecutive nodes of a mode
// row into shared memory, the writes are whole 16-byte rows of a plane.
// The threads also zero the output rows of the tiles that two CTAs
// accumulate into.
constexpr int kPackThreads = 256;
__global__ void __launch_bounds__(kPackThreads) k_ras_inv_pack(const float* __restrict__ R, int64_t ld, int P, int N,
                                                               int64_t bchunks, InvArgs a, float* __restrict__ apack,
                                                               int nsplit) {
  __shared__ float tile[96][kInvKC + 1];
  const int* meta = a.meta;
  const int* chunk_idx = meta + a.off[kChunkIdx];
  const int tid = threadIdx.x;
  const bool stack = 2 * N <= 128;
  const int nop = stack ? 1 : 2;
  for (int64_t gc = blockIdx.x; gc < bchunks; gc += gridDim.x) {
    // thread (k, n0): node k of the chunk in every 16th mode row from n0
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
    float4* out = reinterpret_cast<float4*>(apack + gc * (nop * kInvAop));
    for (int e = tid; e < (kInvKC / 4) * N; e += kPackThreads) {
      const int q = e / N, n = e % N;
      const float v0 = tile[n][4 * q], v1 = tile[n][4 * q + 1], v2 = tile[n][4 * q + 2], v3 = tile[n][4 * q + 3];
      const float4 h = make_float4(tf32_hi(v0), tf32_hi(v1), tf32_hi(v2), tf32_hi(v3));
      const float4 lo = make_float4(v0 - h.x, v1 - h.y, v2 - h.z, v3 - h.w);
      out[q * 128 + n] = h;
      if (stack) out[q * 128 + N + n] = lo;
      else out[kInvAop / 4 + q * 128 + n] = lo;
    }
    __syncthreads();
  }
  const int* split_tile = meta + a.off[kSplitTile];
  const int* tile_owned = meta + a.off[kTileOwned];
  const int64_t nz = int64_t(nsplit) * kInvRows * P;
  const int64_t stride = int64_t(gridDim.x) * kPackThreads;
  for (int64_t e = blockIdx.x * int64_t(kPackThreads) + tid; e < nz; e += stride) {
    const int c = int(e % P);
    const int64_t r = e / P;
    const int g = tile_owned[int64_t(split_tile[r / kInvRows]) * kInvRows + int(r % kInvRows)];
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
// the chunk layout: tile box_tile0[b] + m / 256, chunk j / 16, plane
// (j % 16) / 4, row m % 256, word j % 4
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
    const int tile = box_tile0[b] + m / kInvRows;
    if (tile >= box_tile0[b + 1]) continue;                 // past the box's last tile
    const int64_t c0 = tile_start[tile];
    if (j >= (tile_start[tile + 1] - c0) * kInvKC) continue;  // past the box's last chunk
    const int g = tile_owned[int64_t(tile) * kInvRows + m % kInvRows];
    const float v = (g >= 0 && j < nov[b]) ? float(Zs[int64_t(j) * ld + g]) : 0.f;
    ainv[(c0 + j / kInvKC) * kInvChunk + ((j % kInvKC) / 4) * (kInvRows * 4) + (m % kInvRows) * 4 + (j % 4)] = v;
  }
}

// stage depth (even: two copy warps) and remainder ring for N padded modes
struct InvShape {
  int stages, nlo;
  size_t smem;
};
InvShape inv_shape(int P) {
  const int N = (P + 15) / 16 * 16;
  const int nop = 2 * N <= 128 ? 1 : 2;
  const size_t si = size_t(kInvChunk) * 4, stage = si + size_t(nop) * kInvAop * 4;
  const size_t fixed = size_t(N) * N * 4 + (2 * 32 * (N + 1) + 1) * 4 +
                       (2 * kInvMaxStages + 2 * kInvMaxLo + 5) * 8 + 32;
  for (int nlo = kInvMaxLo; nlo >= 2; --nlo) {
    if (fixed + nlo * si > kSmemLimit) continue;
    const int s = int(std::min<size_t>(kInvMaxStages, (kSmemLimit - fixed - nlo * si) / stage)) & ~1;
    if (s >= 4 || (nlo == 2 && s >= 2)) return InvShape{s, nlo, fixed + nlo * si + s * stage};
  }
  return InvShape{0, 0, 0};
}

template <int NB>
sg_status inv_launch(const InvArgs& args, int grid, size_t smem, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    SG_CUDA(cudaFuncSetAttribute(k_ras_inv_tc<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kSmemLimit)));
    attr = true;
  }
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
bool ras_inverse_supported(int P) { return P >= 1 && P <= 96 && inv_shape(P).stages >= 2; }

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
  const int Mpad = (omax + kInvRows - 1) / kInvRows * kInvRows;
  const int P = pr->P, N = (P + 15) / 16 * 16, nop = 2 * N <= 128 ? 1 : 2;
  // tiles (256 owned rows of a box) and chunks (16 overlapped nodes)
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
    for (int t = 0; t * kInvRows < nown[b]; ++t) {
      tile_box.push_back(b);
      tile_start.push_back(tile_start.back() + nch);
      for (int r = 0; r < kInvRows; ++r)
        tile_owned.push_back(t * kInvRows + r < nown[b] ? own[t * kInvRows + r] : -1);
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
  DevBuf dmeta, dcol, dainv, dapack;
  SG_TRY(dmeta.alloc(meta.size() * 4));
  SG_TRY(dcol.alloc(color.size() * 4));
  SG_CUDA(cudaMemcpy(dmeta.ptr, meta.data(), meta.size() * 4, cudaMemcpyHostToDevice));
  SG_CUDA(cudaMemcpy(dcol.ptr, color.data(), color.size() * 4, cudaMemcpyHostToDevice));
  SG_TRY(dainv.alloc(size_t(chunks) * kInvChunk * 4));
  SG_TRY(dapack.alloc(size_t(bchunks) * nop * kInvAop * 4));
  // the operand rows past the modes stay zero; the pack writes the others
  SG_CUDA(cudaMemsetAsync(dapack.ptr, 0, dapack.bytes, st));
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
  D.inv_chunks = chunks;
  D.inv_bchunks = bchunks;
  D.d_inv = std::move(dainv);
  D.d_inv_bpack = std::move(dapack);
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
  const InvShape sh = inv_shape(P);
  InvArgs a = inv_args(D);
  a.Z = Z;
  a.ld = ld;
  a.ainv = dp<float>(D.d_inv);
  a.apack = dp<float>(D.d_inv_bpack);
  a.M = M;
  a.transform = transform ? 1 : 0;
  a.P = P;
  a.stages = sh.stages;
  a.nlo = sh.nlo;
  a.ntiles = D.inv_ntiles;
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
    case 1: return inv_launch<1>(a, D.inv_grid, sh.smem, st);
    case 2: return inv_launch<2>(a, D.inv_grid, sh.smem, st);
    case 3: return inv_launch<3>(a, D.inv_grid, sh.smem, st);
    case 4: return inv_launch<4>(a, D.inv_grid, sh.smem, st);
    case 5: return inv_launch<5>(a, D.inv_grid, sh.smem, st);
    case 6: return inv_launch<6>(a, D.inv_grid, sh.smem, st);
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
