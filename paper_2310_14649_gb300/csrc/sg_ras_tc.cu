// RAS local solves as dense products with explicit local inverses on the
// fifth-generation tensor cores (Sec. 3, Eq. RASsto):
//     z = sum_i R_i^T D_i (I (x) A_{0,i})^{-1} R_i r,
// where D_i keeps the owned nodes, so box i needs only the owned rows of
// A_{0,i}^{-1}: Zowned_i[m][a] = sum_j Ainv_i[m][j] r[idx_i[j]][a] — a
// product of an (owned x overlapped) matrix with the (overlapped x P)
// restricted residual.  The rows are tiled by 128 (M), the P modes padded
// to N (a multiple of 16), the overlapped nodes (K) streamed in chunks of 32.
// The operands are FP32 split into a TF32 high part and the remainder,
// D += Ah Bh + Ah Bl + Al Bh (kind::tf32, FP32 accumulation in tensor
// memory), which keeps FP32 accuracy.  The epilogue applies the smoother's
// Kronecker factor (omega G~^{-1} across the modes of a node) before the
// store, so no separate node transform follows.
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

constexpr int kInvKC = 16;           // overlapped nodes per chunk (K)
constexpr int kInvStages = 4;        // chunks in flight
constexpr int kInvDrain = 1 << 24;   // polls of the wait that follows a timed-out one

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

// (row m, k) of a K-major operand tile with `rows` rows and 32 k: planes of
// 4 k (16 bytes per row), rows 16 bytes apart, 8-row core matrices 128 bytes
__device__ __forceinline__ int tile_off(int rows, int m, int k) {
  return (k >> 2) * (rows * 16) + (m >> 3) * 128 + (m & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ void cp16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
// 4-byte copy; src_bytes 0 fills zero
__device__ __forceinline__ void cp4(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(smem_addr(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}

// One CTA per (box, 128-row tile of its owned nodes); 128 threads.  The
// inverse rows and the gathered residual stream through kInvStages stages
// of shared memory by asynchronous copies, kInvStages - 1 chunks ahead;
// each thread splits the values it copied into a TF32 high part (in place)
// and the remainder, so no barrier separates a chunk's arrival from its
// split.  smem: stages of {A (128 x KC), A remainder, B (N x KC), B
// remainder}, the transform matrix [P][P], one mbarrier per stage, the
// tensor-memory address.
__global__ void __launch_bounds__(128) k_ras_inv_tc(const float* __restrict__ R, int64_t ld, float* __restrict__ Z,
                                                    int P, int N, int Kp, int Mpad, const int2* __restrict__ items,
                                                    const float* __restrict__ ainv, const int* __restrict__ owned,
                                                    const int* __restrict__ idx, const int* __restrict__ nov,
                                                    const float* __restrict__ M, int transform, int tcols,
                                                    int* __restrict__ err, int wait_limit) {
  extern __shared__ __align__(128) unsigned char sm[];
  const int SA = 128 * kInvKC * 4, SB = N * kInvKC * 4, STAGE = 2 * SA + 2 * SB;
  float* Ms = reinterpret_cast<float*>(sm + kInvStages * STAGE);
  int* Is = reinterpret_cast<int*>(sm + kInvStages * STAGE + ((P * P * 4 + 15) & ~15));  // [Kp] box indices
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + kInvStages * STAGE + ((P * P * 4 + 15) & ~15) + Kp * 4);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + kInvStages);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int2 it = items[blockIdx.x];
  const int box = it.x, row0 = it.y * 128;
  const int nb = nov[box];
  const int nchunk = (nb + kInvKC - 1) / kInvKC;
  const float* A = ainv + (size_t(box) * Mpad + row0) * Kp;
  const int* ix = idx + size_t(box) * Kp;
  if (transform)
    for (int e = tid; e < P * P; e += 128) Ms[e] = M[e];
  for (int e = tid; e < Kp; e += 128) Is[e] = e < nb ? ix[e] : 0;
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(tslot)),
                 "r"(tcols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < kInvStages; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(mbar + s)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  // copies of chunk c into its stage: A rows by 16-byte pieces (thread =
  // row, one piece per 4-column plane), B gathered by 4-byte words with the
  // mode rows of a plane contiguous across the threads
  auto issue = [&](int c) {
    if (c < nchunk) {
      unsigned char* st = sm + (c % kInvStages) * STAGE;
      const int k0 = c * kInvKC;
#pragma unroll
      for (int q = 0; q < kInvKC / 4; ++q) cp16(st + q * 2048 + tid * 16, A + size_t(tid) * Kp + k0 + 4 * q);
      float* Bs = reinterpret_cast<float*>(st + 2 * SA);
      for (int e = tid; e < N * kInvKC; e += 128) {
        const int kk = e & 3, n = (e >> 2) % N, q = (e >> 2) / N;
        const int j = k0 + 4 * q + kk;
        const bool in = n < P && j < nb;
        cp4(Bs + e, in ? R + int64_t(n) * ld + Is[j] : R, in ? 4 : 0);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  auto poll = [&](int s, uint32_t parity, int limit) {
    uint32_t done = 0;
    for (int i = 0; i < limit && !done; ++i)
      asm volatile(
          "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(done)
          : "r"(smem_addr(mbar + s)), "r"(parity)
          : "memory");
    return done;
  };
  for (int c = 0; c < kInvStages - 1; ++c) issue(c);
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t idesc = tf32_desc(128, N);
  bool ok = true;
  int issued = 0;  // chunks whose MMAs were committed
  for (int c = 0; c < nchunk; ++c) {
    const int s = c % kInvStages;
    unsigned char* st = sm + s * STAGE;
    asm volatile("cp.async.wait_group %0;\n" ::"n"(kInvStages - 2) : "memory");
    // split this thread's copies: high part in place, remainder beside it
    {
      float* Ar = reinterpret_cast<float*>(st);
      float* Al = reinterpret_cast<float*>(st + SA);
#pragma unroll
      for (int q = 0; q < kInvKC / 4; ++q) {
        const int off = (q * 2048 + tid * 16) / 4;
        const float4 v = *reinterpret_cast<const float4*>(Ar + off);
        const float4 h = make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z), tf32_hi(v.w));
        *reinterpret_cast<float4*>(Ar + off) = h;
        *reinterpret_cast<float4*>(Al + off) = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
      }
      float* Br = reinterpret_cast<float*>(st + 2 * SA);
      float* Bl = reinterpret_cast<float*>(st + 2 * SA + SB);
      for (int e = tid; e < N * kInvKC; e += 128) {
        const float v = Br[e], h = tf32_hi(v);
        Br[e] = h;
        Bl[e] = v - h;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (tid == 0) {
      const uint32_t ah = smem_addr(st), al = smem_addr(st + SA), bh = smem_addr(st + 2 * SA),
                     bl = smem_addr(st + 2 * SA + SB);
      const uint32_t PLA = 128 * 16, PLB = uint32_t(N) * 16;
#pragma unroll
      for (int k8 = 0; k8 < kInvKC / 8; ++k8) {
        const uint32_t oa = 2 * k8 * PLA, ob = 2 * k8 * PLB;
        const uint64_t dah = smem_desc(ah + oa, PLA, 128), dal = smem_desc(al + oa, PLA, 128);
        const uint64_t dbh = smem_desc(bh + ob, PLB, 128), dbl = smem_desc(bl + ob, PLB, 128);
        const uint64_t da[3] = {dah, dah, dal}, db[3] = {dbh, dbl, dbh};
#pragma unroll
        for (int pass = 0; pass < 3; ++pass) {
          const uint32_t acc = (c > 0 || k8 > 0 || pass > 0) ? 1u : 0u;
          asm volatile(
              "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
              "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
              "l"(da[pass]), "l"(db[pass]), "r"(idesc), "r"(acc)
              : "memory");
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       smem_addr(mbar + s))
                   : "memory");
    }
    issued = c + 1;
    // the stage of chunk c + kInvStages - 1 was read by the MMAs of chunk c - 1
    if (c >= 1) {
      const int cp = c - 1;
      const uint32_t done = poll(cp % kInvStages, uint32_t((cp / kInvStages) & 1), wait_limit);
      if (!__syncthreads_and(done != 0)) {
        ok = false;
        break;
      }
    }
    issue(c + kInvStages - 1);
  }
  // the last commit arrives when every MMA of this CTA has completed
  if (ok && issued > 0) {
    const int cl = issued - 1;
    const uint32_t done = poll(cl % kInvStages, uint32_t((cl / kInvStages) & 1), wait_limit);
    ok = __syncthreads_and(done != 0) != 0;
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (!ok) {
    if (tid == 0) atomicExch(err, 1);
    // MMAs already issued must finish before their tensor memory is freed
    if (issued > 0) {
      const int cl = issued - 1;
      poll(cl % kInvStages, uint32_t((cl / kInvStages) & 1), kInvDrain);
    }
  }
  __syncthreads();
  if (ok && issued > 0) {
    // accumulator rows to shared memory (the stages are free now), row
    // stride odd so that the per-row reads of a warp hit distinct banks
    const int ys = P | 1;
    float* Ys = reinterpret_cast<float*>(sm);
    const int m = warp * 32 + lane;
#pragma unroll
    for (int c16 = 0; c16 < 8; ++c16) {
      if (c16 * 16 >= N) break;
      uint32_t r[16];
      const uint32_t taddr = tmem + (uint32_t(warp * 32) << 16) + uint32_t(16 * c16);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
          "%14, %15}, [%16];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
      for (int q = 0; q < 16; ++q)
        if (c16 * 16 + q < P) Ys[m * ys + c16 * 16 + q] = __uint_as_float(r[q]);
    }
    __syncwarp();
    const int g = owned[size_t(box) * Mpad + row0 + m];
    if (g >= 0) {
      const float* yr = Ys + m * ys;
      for (int a = 0; a < P; ++a) {
        float v;
        if (transform) {
          v = 0.f;
          const float* ma = Ms + a * P;
#pragma unroll 5
          for (int b = 0; b < P; ++b) v = fmaf(ma[b], yr[b], v);
        } else {
          v = yr[a];
        }
        Z[int64_t(a) * ld + g] = v;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(tcols) : "memory");
}

// unit right-hand sides of one colour class: R[j][idx_b[j]] = 1 for the
// boxes b of that class (their overlapped sets are disjoint)
__global__ void k_inv_unit_rhs(double* __restrict__ R, int64_t ld, const int* __restrict__ idx, const int* __restrict__ nov,
                               const int* __restrict__ color, int cls, int Kp, int nbox) {
  const int64_t total = int64_t(nbox) * Kp;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
    const int b = int(t / Kp), j = int(t % Kp);
    if (color[b] != cls || j >= nov[b]) continue;
    R[int64_t(j) * ld + idx[size_t(b) * Kp + j]] = 1.0;
  }
}

// Ainv_b[m][j] = Z[j][owned_b[m]] for the boxes of one colour class
__global__ void k_inv_extract(const double* __restrict__ Zs, int64_t ld, float* __restrict__ ainv,
                              const int* __restrict__ owned, const int* __restrict__ nov,
                              const int* __restrict__ color, int cls, int Mpad, int Kp, int nbox) {
  const int64_t total = int64_t(nbox) * Mpad * Kp;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
    const int b = int(t / (int64_t(Mpad) * Kp));
    if (color[b] != cls) continue;
    const int64_t rem = t - int64_t(b) * Mpad * Kp;
    const int m = int(rem / Kp), j = int(rem % Kp);
    const int g = owned[size_t(b) * Mpad + m];
    ainv[t] = (g >= 0 && j < nov[b]) ? float(Zs[int64_t(j) * ld + g]) : 0.f;
  }
}

size_t inv_smem(int P, int N, int Kp) {
  const size_t stage = 2 * size_t(128) * kInvKC * 4 + 2 * size_t(N) * kInvKC * 4;
  return kInvStages * stage + ((size_t(P) * P * 4 + 15) & ~size_t(15)) + size_t(Kp) * 4 + kInvStages * 8 + 16;
}

}  // namespace

// the index list of the widest supported box: 48 x 48 overlapped nodes
constexpr int kInvMaxKp = 48 * 48;
bool ras_inverse_supported(int P) {
  return P >= 1 && P <= 96 && inv_smem(P, (P + 15) / 16 * 16, kInvMaxKp) <= 227 * 1024;
}

sg_status ras_inverse_build(sg_problem* pr, Precond& pc, cudaStream_t st) {
  RasData& D = pc.ras;
  if (!ras_inverse_supported(pr->P)) {
    set_error("RAS explicit inverses on tensor cores: P must be in [1, 96]");
    return SG_ERR_UNSUPPORTED;
  }
  const int nbox = D.nbox;
  int nmax = 0, omax = 0;
  std::vector<int> nov(nbox), color(nbox);
  for (int b = 0; b < nbox; ++b) {
    nov[b] = int(D.idx[b].size());
    nmax = std::max(nmax, nov[b]);
    int o = 0;
    for (int32_t f : D.owned[b]) o += f ? 1 : 0;
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
  const int Kp = (nmax + 31) / 32 * 32;
  if (Kp > kInvMaxKp) {
    set_error("RAS explicit inverses: overlapped boxes of at most 2,304 nodes");
    return SG_ERR_UNSUPPORTED;
  }
  const int Mpad = (omax + 127) / 128 * 128;
  std::vector<int32_t> hidx(size_t(nbox) * Kp, 0), hown(size_t(nbox) * Mpad, -1);
  std::vector<int2> items;
  for (int b = 0; b < nbox; ++b) {
    int o = 0;
    for (int j = 0; j < nov[b]; ++j) {
      hidx[size_t(b) * Kp + j] = D.idx[b][j];
      if (D.owned[b][j]) hown[size_t(b) * Mpad + o++] = D.idx[b][j];
    }
    for (int t = 0; t * 128 < o; ++t) items.push_back(make_int2(b, t));
  }
  DevBuf didx, down, dnov, dcol, ditems, dainv;
  SG_TRY(didx.alloc(hidx.size() * 4));
  SG_TRY(down.alloc(hown.size() * 4));
  SG_TRY(dnov.alloc(nov.size() * 4));
  SG_TRY(dcol.alloc(color.size() * 4));
  SG_TRY(ditems.alloc(items.size() * sizeof(int2)));
  SG_CUDA(cudaMemcpy(didx.ptr, hidx.data(), hidx.size() * 4, cudaMemcpyHostToDevice));
  SG_CUDA(cudaMemcpy(down.ptr, hown.data(), hown.size() * 4, cudaMemcpyHostToDevice));
  SG_CUDA(cudaMemcpy(dnov.ptr, nov.data(), nov.size() * 4, cudaMemcpyHostToDevice));
  SG_CUDA(cudaMemcpy(dcol.ptr, color.data(), color.size() * 4, cudaMemcpyHostToDevice));
  SG_CUDA(cudaMemcpy(ditems.ptr, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice));
  SG_TRY(dainv.alloc(size_t(nbox) * Mpad * Kp * 4));
  // the local solves (FP64, no Kronecker factor) of the unit right-hand sides
  const int64_t ld = pr->ld;
  DevBuf Rs, Zs;
  SG_TRY(Rs.alloc(size_t(nmax) * ld * 8));
  SG_TRY(Zs.alloc(size_t(nmax) * ld * 8));
  for (int cls = 0; cls < 4; ++cls) {
    SG_CUDA(cudaMemsetAsync(Rs.ptr, 0, Rs.bytes, st));
    SG_CUDA(cudaMemsetAsync(Zs.ptr, 0, Zs.bytes, st));
    k_inv_unit_rhs<<<4 * 152, 256, 0, st>>>(dp<double>(Rs), ld, dp<int>(didx), dp<int>(dnov), dp<int>(dcol), cls, Kp,
                                            nbox);
    note_launch();
    SG_CUDA(cudaGetLastError());
    SG_TRY(ras_apply<double>(pc, pr->n, nmax, dp<double>(Rs), ld, dp<double>(Zs), st, false));
    k_inv_extract<<<4 * 152, 256, 0, st>>>(dp<double>(Zs), ld, dp<float>(dainv), dp<int>(down), dp<int>(dnov),
                                           dp<int>(dcol), cls, Mpad, Kp, nbox);
    note_launch();
    SG_CUDA(cudaGetLastError());
  }
  SG_CUDA(cudaStreamSynchronize(st));
  D.inv_kp = Kp;
  D.inv_mpad = Mpad;
  D.inv_items = int(items.size());
  D.d_inv = std::move(dainv);
  D.d_inv_idx = std::move(didx);
  D.d_inv_owned = std::move(down);
  D.d_inv_nov = std::move(dnov);
  D.d_inv_items = std::move(ditems);
  if (!D.d_inv_err.ptr) SG_TRY(D.d_inv_err.alloc(16));
  SG_CUDA(cudaMemset(D.d_inv_err.ptr, 0, 16));
  static bool attr = false;
  if (!attr) {
    SG_CUDA(cudaFuncSetAttribute(k_ras_inv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    attr = true;
  }
  return SG_OK;
}

sg_status ras_inverse_apply(const Precond& pc, int P, const float* R, int64_t ld, float* Z, const float* M,
                            bool transform, int wait_limit, cudaStream_t st) {
  const RasData& D = pc.ras;
  if (transform && !M) {
    set_error("ras_inverse_apply: the Kronecker factor is not on the device yet");
    return SG_ERR_ARG;
  }
  const int N = (P + 15) / 16 * 16;
  const int tcols = N <= 32 ? 32 : (N <= 64 ? 64 : 128);
  k_ras_inv_tc<<<unsigned(D.inv_items), 128, inv_smem(P, N, D.inv_kp), st>>>(
      R, ld, Z, P, N, D.inv_kp, D.inv_mpad, dp<int2>(D.d_inv_items), dp<float>(D.d_inv), dp<int>(D.d_inv_owned),
      dp<int>(D.d_inv_idx), dp<int>(D.d_inv_nov), M, transform ? 1 : 0, tcols, dp<int>(D.d_inv_err), wait_limit);
  note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
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
