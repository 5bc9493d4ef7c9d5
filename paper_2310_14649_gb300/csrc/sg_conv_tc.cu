// Forward 3x3 convolution of the learned smoother on the fifth-generation
// tensor cores (tcgen05): one CTA computes 128 consecutive pixels of kRows
// image rows for all output channels as implicit GEMMs
//     D_r[pixel][co] = sum_tap sum_ci A_{r,tap}[pixel][ci] W_tap[co][ci],
// M = 128 pixels, N = C_out, K = 9 taps x C_in in steps of 16, BF16 operands
// in shared memory, one FP32 accumulator per row in tensor memory (TMEM).
// One thread issues the kRows x 9 x C_in / 16 MMAs; their completion arrives
// on an mbarrier; each warp then reads its 32 pixels of every accumulator
// and applies bias, ReLU and the BF16 (or FP32) store.
//
// Shared-memory operand layout (K-major, no swizzle, the canonical layout of
// 8-row x 16-byte core matrices): a "plane" holds 8 channels of every row
// (16 bytes per row, rows 16 bytes apart).  The activation tile is
// kRows + 2 image rows x 130 pixels (the output rows with their one-pixel
// halo) per plane, so the A operand of output row r and tap (dy, dx) is the
// same planes started (r + dy) * 130 + dx rows later: M-adjacent core
// matrices are 128 bytes apart (SBO) and K-adjacent ones a plane apart
// (LBO).  Weights are packed the same way, C_out rows per plane, C_in / 8
// planes per tap.
#include <cuda_bf16.h>

#include <algorithm>

#include "sg_cnn.h"

namespace sg {

namespace {

using bf16 = __nv_bfloat16;

constexpr int kHalo = 130;  // halo pixels per row: 128 outputs + 2
constexpr int kRows = 4;    // output rows per CTA (TMEM: 32 columns each)
constexpr int kDrainLimit = 1 << 24;  // polls of the wait that follows a timed-out one

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: start, LBO (K-adjacent core matrices),
// SBO (M/N-adjacent core matrices), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t mat_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return uint64_t((saddr >> 4) & 0x3FFFu) | (uint64_t((lbo >> 4) & 0x3FFFu) << 16) |
         (uint64_t((sbo >> 4) & 0x3FFFu) << 32) | (uint64_t(1) << 46);
}

// kind::f16 instruction descriptor: D FP32, A and B BF16, both K-major
__host__ __device__ constexpr uint32_t inst_desc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t pack_bf2(float lo, float hi) {
  return uint32_t(__bfloat16_as_ushort(__float2bfloat16(lo))) |
         (uint32_t(__bfloat16_as_ushort(__float2bfloat16(hi))) << 16);
}

__device__ __forceinline__ float relu_nan(float x) { return (x > 0.f || x != x) ? x : 0.f; }

// 16-byte global -> shared copy; src_bytes < 16 zero-fills the rest
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}

template <int CI, int CO>
struct TcShape {
  static constexpr int NPA = CI / 8;            // activation planes
  static constexpr int PLA = (kRows + 2) * kHalo * 16;  // bytes per activation plane
  static constexpr int NPB = CI / 8;            // weight planes per tap
  static constexpr int PLB = CO * 16;           // bytes per weight plane
  static constexpr int SB = 9 * NPB * PLB;      // weight bytes
  static constexpr int SA = NPA * PLA;          // activation bytes
  static constexpr int SMEM = SB + SA + 16;
};

// EPI 0: bias + ReLU, BF16 out (CO = 32 channels); EPI 1: bias, FP32 out of
// channel 0 (CO = 16); EPI 2: times (mask > 0), the derivative of the ReLU
// that produced the layer input, BF16 out (CO = 32): the input gradient
// (the same convolution of the output gradient with the flipped,
// transposed weights)
template <int CI, int CO, int EPI>
__global__ void __launch_bounds__(128) k_conv_tc(const bf16* __restrict__ X, const bf16* __restrict__ Wp,
                                                 const float* __restrict__ bias, const bf16* __restrict__ mask,
                                                 bf16* __restrict__ Yb,
                                                 float* __restrict__ Yf, int H, int W, int* __restrict__ err,
                                                 int wait_limit) {
  using S = TcShape<CI, CO>;
  extern __shared__ __align__(128) uint8_t sm[];
  uint8_t* sB = sm;
  uint8_t* sA = sm + S::SB;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sA + S::SA);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int img = blockIdx.z, y0 = blockIdx.y * kRows, x0 = blockIdx.x * 128;

  // all tile copies in flight at once (cp.async, 16 bytes each; outside the
  // image the source size is 0 and the destination is zero-filled)
  for (int e = tid; e < S::SB / 16; e += 128) cp_async16(sB + 16 * e, Wp + 8 * e, 16);
  const bf16* Ximg = X + size_t(img) * H * W * CI;
  for (int e = tid; e < (kRows + 2) * kHalo * S::NPA; e += 128) {
    const int c8 = e % S::NPA, pos = e / S::NPA;
    const int hr = pos / kHalo, hc = pos - hr * kHalo;
    const int gy = y0 + hr - 1, gx = x0 + hc - 1;
    const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
    const bf16* src = in ? Ximg + (size_t(gy) * W + gx) * CI + c8 * 8 : Ximg;
    cp_async16(sA + c8 * S::PLA + pos * 16, src, in ? 16 : 0);
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                 "n"(32 * kRows)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  // the tiles written by ordinary stores become visible to the tensor core
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tslot;
  if (tid == 0) {
    const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
    constexpr uint32_t idesc = inst_desc(128, CO);
#pragma unroll 1
    for (int r = 0; r < kRows; ++r) {
      uint32_t acc = 0;
#pragma unroll 1
      for (int t = 0; t < 9; ++t) {
        const int p0 = (r + t / 3) * kHalo + (t % 3);
#pragma unroll
        for (int kc = 0; kc < CI / 16; ++kc) {
          const uint64_t ad = mat_desc(a0 + uint32_t(2 * kc * S::PLA + p0 * 16), S::PLA, 128);
          const uint64_t bd = mat_desc(b0 + uint32_t((t * S::NPB + 2 * kc) * S::PLB), S::PLB, 128);
          asm volatile(
              "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + uint32_t(32 * r)),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
              : "memory");
          acc = 1;
        }
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                     smem_u32(mbar))
                 : "memory");
  }
  // accumulator complete (bounded wait of wait_limit polls; on a timeout
  // the error flag is set and nothing is stored, and a second bounded wait
  // lets the MMAs already issued finish before their tensor memory is freed)
  auto poll = [&](int limit, uint32_t done) {
    for (int it = 0; it < limit && !done; ++it)
      asm volatile(
          "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\nselp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(done)
          : "r"(smem_u32(mbar))
          : "memory");
    return done;
  };
  uint32_t done = poll(wait_limit, 0u);
  const bool ok = __all_sync(0xffffffffu, done != 0);
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (!ok) {
    if (lane == 0) atomicExch(err, 1);
    poll(kDrainLimit, done);
  } else {
    const int x = x0 + warp * 32 + lane;
#pragma unroll 1
    for (int rr = 0; rr < kRows; ++rr) {
      const uint32_t taddr = tmem + (uint32_t(warp * 32) << 16) + uint32_t(32 * rr);
      const int y = y0 + rr;
      const size_t pix = (size_t(img) * H + y) * W + x;
      const bool store = x < W && y < H;
      if (CO == 32) {
        uint32_t r[32];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
              "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
              "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
              "=r"(r[30]), "=r"(r[31])
            : "r"(taddr)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        if (store) {
          uint32_t o[16];
          if (EPI == 0) {
#pragma unroll
            for (int c = 0; c < 16; ++c)
              o[c] = pack_bf2(relu_nan(__uint_as_float(r[2 * c]) + bias[2 * c]),
                              relu_nan(__uint_as_float(r[2 * c + 1]) + bias[2 * c + 1]));
          } else {
            const uint4* mk = reinterpret_cast<const uint4*>(mask + pix * 32);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const uint4 mv = mk[q];
              const uint32_t mw[4] = {mv.x, mv.y, mv.z, mv.w};
#pragma unroll
              for (int h = 0; h < 4; ++h) {
                const int c = 4 * q + h;
                const float m0 = __bfloat162float(__ushort_as_bfloat16(uint16_t(mw[h] & 0xffffu)));
                const float m1 = __bfloat162float(__ushort_as_bfloat16(uint16_t(mw[h] >> 16)));
                o[c] = pack_bf2(m0 > 0.f ? __uint_as_float(r[2 * c]) : 0.f,
                                m1 > 0.f ? __uint_as_float(r[2 * c + 1]) : 0.f);
              }
            }
          }
          uint4* dst = reinterpret_cast<uint4*>(Yb + pix * 32);
#pragma unroll
          for (int q = 0; q < 4; ++q) dst[q] = make_uint4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
        }
      } else {
        uint32_t r[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15}, [%16];\n"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        if (store && EPI == 1) Yf[pix] = __uint_as_float(r[0]) + bias[0];
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "n"(32 * kRows) : "memory");
}

// Weight gradient of a 3x3 convolution on the tensor cores:
//     dW[dy dx][co][ci] = sum_pixels G[y][x][co] X[y + dy - 1][x + dx - 1][ci],
//     db[co] = sum_pixels G[y][x][co],
// as one implicit GEMM per tap row dy: D_dy[(dx, ci)][co] = sum_x A[(dx, ci)][x]
// B[co][x], M = 3 C_in shifted input channels (+ a row of ones that yields
// the bias gradient, the rest zero) padded to 128, N = C_out, K = the 128
// pixels of one image-row segment.  A CTA walks down a strip of rows of one
// 128-pixel column segment: input row y + 1 is transposed into one of three
// rolling shared-memory slots (pixels along K, three copies shifted by dx),
// so the rows y - 1, y and y + 1 that output row y needs are resident, and
// the output-gradient row y is transposed into B.  The three accumulators
// (one per dy) stay in tensor memory over the whole strip; the epilogue adds
// them to the FP32 gradient with atomics.  Shared-memory operands are
// K-major in the canonical layout (8-row x 16-byte core matrices; planes of
// 8 pixels, rows 16 bytes apart).
constexpr int kWgRows = 128;       // M rows of the A operand (padded)
constexpr int kWgPix = 128;        // pixels per chunk (K)

template <int CI, int CO>
struct WgShape {
  static constexpr int PLANE_A = kWgRows * 16;            // bytes per 8-pixel plane of A
  static constexpr int SLOT = (kWgPix / 8) * PLANE_A;     // bytes per rolling input slot
  static constexpr int PLANE_B = CO * 16;
  static constexpr int SB = (kWgPix / 8) * PLANE_B;
  static constexpr int ONES = 3 * CI;                     // the row of ones (bias gradient)
  static constexpr int SMEM = 3 * SLOT + SB + 16;
};

template <int CI, int CO>
__global__ void __launch_bounds__(128) k_wgrad_tc(const bf16* __restrict__ X, const bf16* __restrict__ G,
                                                  float* __restrict__ dW, float* __restrict__ db, int H, int W,
                                                  int rows_per_cta, int* __restrict__ err, int wait_limit) {
  using S = WgShape<CI, CO>;
  extern __shared__ __align__(128) uint8_t sm[];
  uint8_t* sA = sm;
  uint8_t* sB = sm + 3 * S::SLOT;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sB + S::SB);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int x0 = blockIdx.x * kWgPix, img = blockIdx.z;
  const int ya = blockIdx.y * rows_per_cta, yb = min(H, ya + rows_per_cta);
  const bf16* Ximg = X + size_t(img) * H * W * CI;
  const bf16* Gimg = G + size_t(img) * H * W * CO;
  // element (row m, pixel k) of slot s / of B (row co, pixel k)
  auto a_off = [&](int s, int m, int k) { return s * S::SLOT + (k >> 3) * S::PLANE_A + (m >> 3) * 128 + (m & 7) * 16 + (k & 7) * 2; };
  auto b_off = [&](int co, int k) { return (k >> 3) * S::PLANE_B + (co >> 3) * 128 + (co & 7) * 16 + (k & 7) * 2; };
  // zero every slot, then the row of ones
  for (int e = tid; e < 3 * S::SLOT / 16; e += 128) reinterpret_cast<uint4*>(sA)[e] = make_uint4(0, 0, 0, 0);
  __syncthreads();
  const bf16 one = __float2bfloat16(1.0f);
  for (int e = tid; e < 3 * kWgPix; e += 128)
    *reinterpret_cast<bf16*>(sA + a_off(e / kWgPix, S::ONES, e % kWgPix)) = one;
  // input row r (zero outside the image) into slot (r + 3) % 3: position q
  // (x = x0 + q - 1) feeds copies dx with pixel k = q - dx
  auto stage_x = [&](int r) {
    const int s = (r + 3) % 3;
    for (int e = tid; e < (kWgPix + 2) * (CI / 8); e += 128) {
      const int q = e / (CI / 8), c8 = e % (CI / 8);
      const int x = x0 + q - 1;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (r >= 0 && r < H && x >= 0 && x < W) v = *reinterpret_cast<const uint4*>(Ximg + (size_t(r) * W + x) * CI + 8 * c8);
      const bf16* hv = reinterpret_cast<const bf16*>(&v);
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) {
        const int k = q - dx;
        if (k < 0 || k >= kWgPix) continue;
#pragma unroll
        for (int c = 0; c < 8; ++c) *reinterpret_cast<bf16*>(sA + a_off(s, dx * CI + 8 * c8 + c, k)) = hv[c];
      }
    }
  };
  auto stage_g = [&](int y) {
    for (int e = tid; e < kWgPix * (CO / 8); e += 128) {
      const int k = e / (CO / 8), c8 = e % (CO / 8);
      const int x = x0 + k;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (x < W) v = *reinterpret_cast<const uint4*>(Gimg + (size_t(y) * W + x) * CO + 8 * c8);
      const bf16* hv = reinterpret_cast<const bf16*>(&v);
#pragma unroll
      for (int c = 0; c < 8; ++c) *reinterpret_cast<bf16*>(sB + b_off(8 * c8 + c, k)) = hv[c];
    }
  };
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                 "n"(128)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (ya < yb) {
    stage_x(ya - 1);
    stage_x(ya);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
  constexpr uint32_t idesc = inst_desc(128, CO);
  auto poll = [&](int limit, uint32_t parity) {
    uint32_t done = 0;
    for (int it = 0; it < limit && !done; ++it)
      asm volatile(
          "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(done)
          : "r"(smem_u32(mbar)), "r"(parity)
          : "memory");
    return done;
  };
  bool ok = true;
  uint32_t phase = 0;
  for (int y = ya; y < yb; ++y) {
    stage_x(y + 1);
    stage_g(y);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (tid == 0) {
#pragma unroll 1
      for (int dy = 0; dy < 3; ++dy) {
        const int s = (y + dy - 1 + 3) % 3;
#pragma unroll
        for (int kc = 0; kc < kWgPix / 16; ++kc) {
          const uint64_t ad = mat_desc(a0 + uint32_t(s * S::SLOT + 2 * kc * S::PLANE_A), S::PLANE_A, 128);
          const uint64_t bd = mat_desc(b0 + uint32_t(2 * kc * S::PLANE_B), S::PLANE_B, 128);
          const uint32_t acc = (y > ya || kc > 0) ? 1u : 0u;
          asm volatile(
              "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + uint32_t(dy * CO)),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
              : "memory");
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       smem_u32(mbar))
                   : "memory");
    }
    // the MMAs read the slots and B: wait before the next staging
    const uint32_t done = poll(wait_limit, phase);
    ok = __syncthreads_and(done != 0) != 0;
    phase ^= 1u;
    if (!ok) {
      if (tid == 0) atomicExch(err, 1);
      poll(kDrainLimit, phase ^ 1u);   // the MMAs of this chunk, before tensor memory is freed
      break;
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (ok && ya < yb) {
    // lanes = A rows m = dx C_in + ci (and the row of ones), columns = co
    const int m = warp * 32 + lane;
#pragma unroll 1
    for (int dy = 0; dy < 3; ++dy) {
      uint32_t r[CO];
      const uint32_t taddr = tmem + (uint32_t(warp * 32) << 16) + uint32_t(dy * CO);
      if (CO == 32) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
              "=r"(r[16 % CO]), "=r"(r[17 % CO]), "=r"(r[18 % CO]), "=r"(r[19 % CO]), "=r"(r[20 % CO]),
              "=r"(r[21 % CO]), "=r"(r[22 % CO]), "=r"(r[23 % CO]), "=r"(r[24 % CO]), "=r"(r[25 % CO]),
              "=r"(r[26 % CO]), "=r"(r[27 % CO]), "=r"(r[28 % CO]), "=r"(r[29 % CO]), "=r"(r[30 % CO]),
              "=r"(r[31 % CO])
            : "r"(taddr)
            : "memory");
      } else {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15}, [%16];\n"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr)
            : "memory");
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (m < 3 * CI) {
        const int dx = m / CI, ci = m % CI, t = dy * 3 + dx;
#pragma unroll
        for (int co = 0; co < CO; ++co) atomicAdd(dW + (size_t(t) * CO + co) * CI + ci, __uint_as_float(r[co]));
      } else if (m == S::ONES && dy == 1) {
#pragma unroll
        for (int co = 0; co < CO; ++co) atomicAdd(db + co, __uint_as_float(r[co]));
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "n"(128) : "memory");
}

// FP32 padded weights [tap][co][ci] -> BF16 planes [tap][ci / 8][co][8];
// with rev, the flipped, transposed weights of the input gradient,
// W'[8 - tap][ci][co] = W[tap][co][ci], as planes [tap'][co / 8][ci][8]
__global__ void k_pack_planes(const float* __restrict__ Wsrc, int ci_pad, int co_pad, bf16* __restrict__ out,
                              int rev) {
  const int total = 9 * co_pad * ci_pad;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int t = e / (co_pad * ci_pad), rem = e - t * co_pad * ci_pad;
    const int co = rem / ci_pad, ci = rem - co * ci_pad;
    const size_t dst = rev ? ((size_t(8 - t) * (co_pad / 8) + co / 8) * ci_pad + ci) * 8 + (co % 8)
                           : ((size_t(t) * (ci_pad / 8) + ci / 8) * co_pad + co) * 8 + (ci % 8);
    out[dst] = __float2bfloat16(Wsrc[e]);
  }
}

template <int CI, int CO, int EPI>
sg_status launch_tc(const bf16* X, const bf16* Wp, const float* b, const bf16* mask, bf16* Yb, float* Yf, int H,
                    int W, int nimg, int* err, int wait_limit, cudaStream_t st) {
  dim3 grid(unsigned((W + 127) / 128), unsigned((H + kRows - 1) / kRows), unsigned(nimg));
  k_conv_tc<CI, CO, EPI><<<grid, 128, TcShape<CI, CO>::SMEM, st>>>(X, Wp, b, mask, Yb, Yf, H, W, err, wait_limit);
  note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

}  // namespace

sg_status conv_tc_attrs() {
  static bool done = false;
  if (done) return SG_OK;
  SG_CUDA(cudaFuncSetAttribute(k_conv_tc<16, 32, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               TcShape<16, 32>::SMEM));
  SG_CUDA(cudaFuncSetAttribute(k_conv_tc<32, 32, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               TcShape<32, 32>::SMEM));
  SG_CUDA(cudaFuncSetAttribute(k_conv_tc<32, 16, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               TcShape<32, 16>::SMEM));
  SG_CUDA(cudaFuncSetAttribute(k_conv_tc<16, 32, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               TcShape<16, 32>::SMEM));
  SG_CUDA(cudaFuncSetAttribute(k_conv_tc<32, 32, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               TcShape<32, 32>::SMEM));
  SG_CUDA(cudaFuncSetAttribute(k_wgrad_tc<16, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               WgShape<16, 32>::SMEM));
  SG_CUDA(cudaFuncSetAttribute(k_wgrad_tc<32, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               WgShape<32, 32>::SMEM));
  SG_CUDA(cudaFuncSetAttribute(k_wgrad_tc<32, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               WgShape<32, 16>::SMEM));
  done = true;
  return SG_OK;
}

sg_status conv_tc_pack(const float* Wsrc, int ci_pad, int co_pad, void* out, bool rev, cudaStream_t st) {
  k_pack_planes<<<64, 256, 0, st>>>(Wsrc, ci_pad, co_pad, static_cast<bf16*>(out), rev ? 1 : 0);
  note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

// layer l of the network: 0 (16 -> 32), 1..3 (32 -> 32), 4 (32 -> 16, FP32 out)
sg_status conv_tc_layer(int l, const void* X, const void* Wp, const float* b, void* Yb, float* Yf, int H, int W,
                        int nimg, int* err, int wait_limit, cudaStream_t st) {
  const bf16* x = static_cast<const bf16*>(X);
  const bf16* w = static_cast<const bf16*>(Wp);
  if (l == 0)
    return launch_tc<16, 32, 0>(x, w, b, nullptr, static_cast<bf16*>(Yb), nullptr, H, W, nimg, err, wait_limit, st);
  if (l == 4) return launch_tc<32, 16, 1>(x, w, b, nullptr, nullptr, Yf, H, W, nimg, err, wait_limit, st);
  return launch_tc<32, 32, 0>(x, w, b, nullptr, static_cast<bf16*>(Yb), nullptr, H, W, nimg, err, wait_limit, st);
}

template <int CI, int CO>
sg_status launch_wgrad(const bf16* X, const bf16* G, float* dW, float* db, int H, int W, int nimg, int* err,
                       int wait_limit, cudaStream_t st) {
  const int xs = (W + kWgPix - 1) / kWgPix;
  // about two CTAs per SM over the (column segment, row strip, image) grid
  const int64_t strips = int64_t(xs) * nimg;
  int rows = int(std::max<int64_t>(4, (int64_t(H) * strips + 2 * 152 - 1) / (2 * 152)));
  rows = std::min(rows, H);
  dim3 grid(unsigned(xs), unsigned((H + rows - 1) / rows), unsigned(nimg));
  k_wgrad_tc<CI, CO><<<grid, 128, WgShape<CI, CO>::SMEM, st>>>(X, G, dW, db, H, W, rows, err, wait_limit);
  note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

// weight and bias gradients of layer l, added to dW [tap][C_out][C_in] and
// db (FP32, padded channel counts): X the layer input, G its output gradient
sg_status conv_tc_wgrad(int l, const void* X, const void* G, float* dW, float* db, int H, int W, int nimg, int* err,
                        int wait_limit, cudaStream_t st) {
  const bf16* x = static_cast<const bf16*>(X);
  const bf16* g = static_cast<const bf16*>(G);
  if (l == 0) return launch_wgrad<16, 32>(x, g, dW, db, H, W, nimg, err, wait_limit, st);
  if (l == 4) return launch_wgrad<32, 16>(x, g, dW, db, H, W, nimg, err, wait_limit, st);
  return launch_wgrad<32, 32>(x, g, dW, db, H, W, nimg, err, wait_limit, st);
}

// input gradient of layer l (1..4): G (the output gradient, C_out(l)
// channels) convolved with the flipped, transposed weights Wr, times the
// ReLU derivative of the layer input (mask), into Yb (C_in(l) = 32 channels)
sg_status conv_tc_dgrad(int l, const void* G, const void* Wr, const void* mask, void* Yb, int H, int W, int nimg,
                        int* err, int wait_limit, cudaStream_t st) {
  const bf16* g = static_cast<const bf16*>(G);
  const bf16* w = static_cast<const bf16*>(Wr);
  const bf16* mk = static_cast<const bf16*>(mask);
  if (l == 4)
    return launch_tc<16, 32, 2>(g, w, nullptr, mk, static_cast<bf16*>(Yb), nullptr, H, W, nimg, err, wait_limit, st);
  return launch_tc<32, 32, 2>(g, w, nullptr, mk, static_cast<bf16*>(Yb), nullptr, H, W, nimg, err, wait_limit, st);
}

}  // namespace sg
