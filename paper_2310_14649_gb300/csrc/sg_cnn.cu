// Learned smoother: a 5-layer 3x3 convolutional network (channels 2 -> 32
// -> 32 -> 32 -> 32 -> 1, ReLU between layers) applied to the P mode images
// of a residual, trained with Adam on (residual, A_0^{-1} residual) pairs.
// The method statement adds it in place of the mean-based block solve; the
// paper has no counterpart.
//
// Layout: activations are BF16, channels last ([image][y][x][C], C padded
// to 16 or 32); weights are [tap][Cout][Cin] (Cin contiguous), FP32 master
// copies with BF16 copies for the tensor cores; accumulation is FP32.
//
// With the tcgen05 kernels selected (default), the forward convolutions,
// the input gradients and the weight gradients run on the fifth-generation
// tensor cores (sg_conv_tc.cu); with the legacy kernels selected they run on
// the kernels below.
// Convolutions are implicit GEMMs on the tensor cores (BF16 mma.sync
// m16n8k16, FP32 accumulators): a CTA of 4 warps owns an 8 x 16 pixel tile,
// the input tile with its 1-pixel halo and all 9 taps of the weights sit in
// shared memory (rows padded by 8 elements so fragment loads are
// bank-conflict free).  Forward: M = pixels, N = Cout, K = 9 Cin.  The
// gradient with respect to the input is the same kernel run on the output
// gradient with the flipped, transposed weights; the weight gradient is a
// GEMM with M = Cout, N = Cin, K = pixels, accumulated per CTA and added to
// the global FP32 gradient once.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "sg_cnn.h"
#include "sg_kernels.h"

namespace sg {

namespace {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t ld32(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }
__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
  return uint32_t(__bfloat16_as_ushort(lo)) | (uint32_t(__bfloat16_as_ushort(hi)) << 16);
}

constexpr int TH = 8, TW = 16;  // pixel tile of one CTA

// ReLU that keeps NaN (as max(x, 0) of IEEE arithmetic without fmax's
// NaN suppression), so a corrupted network shows as a non-finite output
__device__ __forceinline__ float relu(float x) { return (x > 0.f || x != x) ? x : 0.f; }

// EPI 0: + bias, ReLU, BF16 out.  EPI 1: + bias, FP32 out of channel 0.
// EPI 2: multiply by (mask > 0) (ReLU of the layer input), BF16 out.
template <int CI, int CO, int EPI>
__global__ void __launch_bounds__(128) k_conv(const bf16* __restrict__ X, const bf16* __restrict__ Wt,
                                              const float* __restrict__ bias, const bf16* __restrict__ mask,
                                              bf16* __restrict__ Yb, float* __restrict__ Yf, int H, int W) {
  constexpr int CIS = CI + 8, COS = CI + 8;
  __shared__ __align__(16) bf16 xs[(TH + 2) * (TW + 2) * CIS];
  __shared__ __align__(16) bf16 ws[9 * CO * COS];
  const int img = blockIdx.z, y0 = blockIdx.y * TH, x0 = blockIdx.x * TW;
  const int tid = threadIdx.x;
  for (int e = tid; e < 9 * CO * (CI / 2); e += 128) {
    const int row = e / (CI / 2), c2 = e - row * (CI / 2);
    *reinterpret_cast<uint32_t*>(&ws[row * COS + 2 * c2]) = ld32(Wt + size_t(row) * CI + 2 * c2);
  }
  const bf16* Ximg = X + size_t(img) * H * W * CI;
  for (int e = tid; e < (TH + 2) * (TW + 2) * (CI / 2); e += 128) {
    const int pos = e / (CI / 2), c2 = e - pos * (CI / 2);
    const int hy = pos / (TW + 2), hx = pos - hy * (TW + 2);
    const int gy = y0 + hy - 1, gx = x0 + hx - 1;
    uint32_t v = 0u;
    if (gy >= 0 && gy < H && gx >= 0 && gx < W) v = ld32(Ximg + (size_t(gy) * W + gx) * CI + 2 * c2);
    *reinterpret_cast<uint32_t*>(&xs[pos * CIS + 2 * c2]) = v;
  }
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31, gid = lane >> 2, tig = lane & 3;
  constexpr int NT = CO / 8;
  float acc[2][NT][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[mt][nt][q] = 0.f;
#pragma unroll
  for (int tap = 0; tap < 9; ++tap) {
    const int dy = tap / 3, dx = tap % 3;
#pragma unroll
    for (int kc = 0; kc < CI / 16; ++kc) {
      uint32_t a[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const int r = 2 * warp + mt + dy;
        const bf16* base = xs + (r * (TW + 2) + dx) * CIS + kc * 16 + tig * 2;
        a[mt][0] = ld32(base + gid * CIS);
        a[mt][1] = ld32(base + (gid + 8) * CIS);
        a[mt][2] = ld32(base + gid * CIS + 8);
        a[mt][3] = ld32(base + (gid + 8) * CIS + 8);
      }
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const bf16* wb = ws + (tap * CO + nt * 8 + gid) * COS + kc * 16 + tig * 2;
        const uint32_t b0 = ld32(wb), b1 = ld32(wb + 8);
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) mma_bf16(acc[mt][nt], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b0, b1);
      }
    }
  }
  // epilogue: c0, c1 = (pixel gid, channels 2 tig, 2 tig + 1); c2, c3 = pixel gid + 8
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    const int y = y0 + 2 * warp + mt;
    if (y >= H) continue;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int x = x0 + gid + 8 * half;
      if (x >= W) continue;
      const size_t pix = (size_t(img) * H + y) * W + x;
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const int co = nt * 8 + tig * 2;
        float v0 = acc[mt][nt][2 * half], v1 = acc[mt][nt][2 * half + 1];
        if (EPI == 1) {
          if (co == 0) Yf[pix] = v0 + bias[0];
          continue;
        }
        if (EPI == 0) {
          v0 = relu(v0 + bias[co]);
          v1 = relu(v1 + bias[co + 1]);
        } else {
          const uint32_t m = ld32(mask + pix * CO + co);
          if (!(__bfloat162float(__ushort_as_bfloat16(uint16_t(m & 0xffffu))) > 0.f)) v0 = 0.f;
          if (!(__bfloat162float(__ushort_as_bfloat16(uint16_t(m >> 16))) > 0.f)) v1 = 0.f;
        }
        *reinterpret_cast<uint32_t*>(Yb + pix * CO + co) = pack2(__float2bfloat16(v0), __float2bfloat16(v1));
      }
    }
  }
}

// Weight and bias gradients of one layer: dW[tap][co][ci] += sum_p dY[p][co]
// X[p + off_tap][ci], db[co] += sum_p dY[p][co].  Grid-stride over 8 x 16
// pixel tiles; warp w owns taps w, w + 4, w + 8.
template <int CI, int CO>
__global__ void __launch_bounds__(128) k_conv_wgrad(const bf16* __restrict__ X, const bf16* __restrict__ dY,
                                                    float* __restrict__ dW, float* __restrict__ db, int H, int W,
                                                    int nimg) {
  constexpr int CIS = CI + 8, COS = CO + 8;
  __shared__ __align__(16) bf16 xs[(TH + 2) * (TW + 2) * CIS];
  __shared__ __align__(16) bf16 ys[TH * TW * COS];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, gid = lane >> 2, tig = lane & 3;
  constexpr int MT = CO / 16, NT = CI / 8;
  float acc[3][MT][NT][4];
#pragma unroll
  for (int t = 0; t < 3; ++t)
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[t][mt][nt][q] = 0.f;
  float bacc = 0.f;
  const int tx = (W + TW - 1) / TW, ty = (H + TH - 1) / TH;
  const long long ntiles = (long long)tx * ty * nimg;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int img = int(tile / (tx * ty));
    const int rem = int(tile - (long long)img * tx * ty);
    const int y0 = (rem / tx) * TH, x0 = (rem % tx) * TW;
    const bf16* Ximg = X + size_t(img) * H * W * CI;
    const bf16* Yimg = dY + size_t(img) * H * W * CO;
    __syncthreads();
    for (int e = tid; e < (TH + 2) * (TW + 2) * (CI / 2); e += 128) {
      const int pos = e / (CI / 2), c2 = e - pos * (CI / 2);
      const int hy = pos / (TW + 2), hx = pos - hy * (TW + 2);
      const int gy = y0 + hy - 1, gx = x0 + hx - 1;
      uint32_t v = 0u;
      if (gy >= 0 && gy < H && gx >= 0 && gx < W) v = ld32(Ximg + (size_t(gy) * W + gx) * CI + 2 * c2);
      *reinterpret_cast<uint32_t*>(&xs[pos * CIS + 2 * c2]) = v;
    }
    for (int e = tid; e < TH * TW * (CO / 2); e += 128) {
      const int pos = e / (CO / 2), c2 = e - pos * (CO / 2);
      const int gy = y0 + pos / TW, gx = x0 + pos % TW;
      uint32_t v = 0u;
      if (gy < H && gx < W) v = ld32(Yimg + (size_t(gy) * W + gx) * CO + 2 * c2);
      *reinterpret_cast<uint32_t*>(&ys[pos * COS + 2 * c2]) = v;
    }
    __syncthreads();
    // bias gradient: thread t < CO sums channel t over the tile
    if (tid < CO)
      for (int p = 0; p < TH * TW; ++p) bacc += __bfloat162float(ys[p * COS + tid]);
#pragma unroll
    for (int ti = 0; ti < 3; ++ti) {
      const int tap = warp + 4 * ti;
      if (tap >= 9) break;
      const int dy = tap / 3, dx = tap % 3;
#pragma unroll
      for (int kc = 0; kc < TH; ++kc) {  // 16 pixels of tile row kc per k step
        uint32_t a[MT][4], b[NT][2];
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
          const int c0 = mt * 16 + gid;
          const bf16* yr = ys + (kc * TW) * COS;
          a[mt][0] = pack2(yr[(tig * 2) * COS + c0], yr[(tig * 2 + 1) * COS + c0]);
          a[mt][1] = pack2(yr[(tig * 2) * COS + c0 + 8], yr[(tig * 2 + 1) * COS + c0 + 8]);
          a[mt][2] = pack2(yr[(tig * 2 + 8) * COS + c0], yr[(tig * 2 + 9) * COS + c0]);
          a[mt][3] = pack2(yr[(tig * 2 + 8) * COS + c0 + 8], yr[(tig * 2 + 9) * COS + c0 + 8]);
        }
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
          const int ci = nt * 8 + gid;
          const bf16* xr = xs + ((kc + dy) * (TW + 2) + dx) * CIS + ci;
          b[nt][0] = pack2(xr[(tig * 2) * CIS], xr[(tig * 2 + 1) * CIS]);
          b[nt][1] = pack2(xr[(tig * 2 + 8) * CIS], xr[(tig * 2 + 9) * CIS]);
        }
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
          for (int nt = 0; nt < NT; ++nt)
            mma_bf16(acc[ti][mt][nt], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b[nt][0], b[nt][1]);
      }
    }
  }
  // c0, c1 = (co gid, ci 2 tig, 2 tig + 1); c2, c3 = co gid + 8
#pragma unroll
  for (int ti = 0; ti < 3; ++ti) {
    const int tap = warp + 4 * ti;
    if (tap >= 9) break;
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const int co = mt * 16 + gid, ci = nt * 8 + tig * 2;
        float* d = dW + (size_t(tap) * CO + co) * CI + ci;
        atomicAdd(d, acc[ti][mt][nt][0]);
        atomicAdd(d + 1, acc[ti][mt][nt][1]);
        atomicAdd(d + size_t(8) * CI, acc[ti][mt][nt][2]);
        atomicAdd(d + size_t(8) * CI + 1, acc[ti][mt][nt][3]);
      }
  }
  if (tid < CO) atomicAdd(db + tid, bacc);
}

// Network input of the mode images: ch0 = r / rms(r), ch1 = log(diag / 4),
// channels 2..15 zero.
template <typename T>
__global__ void k_pack_input(const T* __restrict__ R, int64_t ld, int64_t n, const double* __restrict__ sumsq,
                             const float* __restrict__ logd, bf16* __restrict__ X) {
  const int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int a = blockIdx.y;
  if (r >= n) return;
  const double ms = sumsq[a] / double(n);
  const double inv = ms > 0.0 ? 1.0 / sqrt(ms) : 0.0;
  uint4* x = reinterpret_cast<uint4*>(X + (size_t(a) * n + r) * 16);
  const uint32_t c01 = pack2(__double2bfloat16(double(R[int64_t(a) * ld + r]) * inv), __float2bfloat16(logd[r]));
  x[0] = make_uint4(c01, 0u, 0u, 0u);
  x[1] = make_uint4(0u, 0u, 0u, 0u);
}

template <typename T>
__global__ void k_col_sumsq(const T* __restrict__ R, int64_t ld, int64_t n, double* __restrict__ out) {
  const int a = blockIdx.y;
  double s = 0.0;
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < n; r += int64_t(gridDim.x) * blockDim.x) {
    const double v = double(R[int64_t(a) * ld + r]);
    s += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out + a, s);
}

// Z[a][r] = Y[a][r] * rms_a (the network output back in residual units);
// rows n..ld-1 of Z are cleared
template <typename T>
__global__ void k_unpack_output(const float* __restrict__ Y, int64_t n, const double* __restrict__ sumsq,
                                T* __restrict__ Z, int64_t ld) {
  const int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int a = blockIdx.y;
  if (r >= ld) return;
  if (r >= n) {
    Z[int64_t(a) * ld + r] = T(0);
    return;
  }
  const double rms = sqrt(sumsq[a] / double(n));
  Z[int64_t(a) * ld + r] = T(double(Y[size_t(a) * n + r]) * rms);
}

// training target in network units: Zs[a][r] = Z*[a][r] / rms(r_a)
__global__ void k_scale_targets(const float* __restrict__ Z, int64_t ld, int64_t n, const double* __restrict__ sumsq,
                                float* __restrict__ Zs) {
  const int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int a = blockIdx.y;
  if (r >= n) return;
  const double ms = sumsq[a] / double(n);
  Zs[size_t(a) * n + r] = ms > 0.0 ? float(double(Z[int64_t(a) * ld + r]) / sqrt(ms)) : 0.f;
}

// loss: per image sum (zhat - z*)^2 and sum z*^2 (z* in network units)
__global__ void k_loss_parts(const float* __restrict__ Yf, const float* __restrict__ Zs, int64_t npix,
                             double* __restrict__ num, double* __restrict__ den) {
  const int img = blockIdx.y;
  double a = 0.0, b = 0.0;
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < npix; p += int64_t(gridDim.x) * blockDim.x) {
    const double y = Yf[size_t(img) * npix + p], z = Zs[size_t(img) * npix + p];
    a += (y - z) * (y - z);
    b += z * z;
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(num + img, a);
    atomicAdd(den + img, b);
  }
}

// dL/dy = 2 (zhat - z*) / ||z*||^2, written as channel 0 of a 16-channel
// BF16 gradient image
__global__ void k_loss_grad(const float* __restrict__ Yf, const float* __restrict__ Zs, int64_t npix,
                            const double* __restrict__ den, bf16* __restrict__ dY) {
  const int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int img = blockIdx.y;
  if (p >= npix) return;
  const double d = den[img];
  const float g = d > 0.0 ? float(2.0 * (double(Yf[size_t(img) * npix + p]) - Zs[size_t(img) * npix + p]) / d) : 0.f;
  uint32_t* o = reinterpret_cast<uint32_t*>(dY + (size_t(img) * npix + p) * 16);
  o[0] = pack2(__float2bfloat16(g), __float2bfloat16(0.f));
#pragma unroll
  for (int q = 1; q < 8; ++q) o[q] = 0u;
}

// energy-norm loss: E = Y - Z*, then (with AE = A_0 E, AZ = A_0 Z* from the
// sparse product) per image e.AE and z.AZ, and the gradient 2 AE / (z.AZ)
__global__ void k_diff(const float* __restrict__ Y, const float* __restrict__ Z, float* __restrict__ E, int64_t cnt) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < cnt; i += int64_t(gridDim.x) * blockDim.x)
    E[i] = Y[i] - Z[i];
}

__global__ void k_energy_parts(const float* __restrict__ E, const float* __restrict__ AE, const float* __restrict__ Z,
                               const float* __restrict__ AZ, int64_t npix, double* __restrict__ num,
                               double* __restrict__ den) {
  const int img = blockIdx.y;
  const size_t o = size_t(img) * npix;
  double a = 0.0, b = 0.0;
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < npix; p += int64_t(gridDim.x) * blockDim.x) {
    a += double(E[o + p]) * double(AE[o + p]);
    b += double(Z[o + p]) * double(AZ[o + p]);
  }
  for (int w = 16; w > 0; w >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, w);
    b += __shfl_xor_sync(0xffffffffu, b, w);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(num + img, a);
    atomicAdd(den + img, b);
  }
}

__global__ void k_energy_grad(const float* __restrict__ AE, int64_t npix, const double* __restrict__ den,
                              bf16* __restrict__ dY) {
  const int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int img = blockIdx.y;
  if (p >= npix) return;
  const double d = den[img];
  const float g = d > 0.0 ? float(2.0 * double(AE[size_t(img) * npix + p]) / d) : 0.f;
  uint32_t* o = reinterpret_cast<uint32_t*>(dY + (size_t(img) * npix + p) * 16);
  o[0] = pack2(__float2bfloat16(g), __float2bfloat16(0.f));
#pragma unroll
  for (int q = 1; q < 8; ++q) o[q] = 0u;
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t cnt, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < cnt; i += int64_t(gridDim.x) * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// BF16 forward weights [tap][co][ci] and the flipped, transposed weights of
// the input gradient [tap][ci][co]: Wr[t][ci][co] = W[8 - t][co][ci]
__global__ void k_pack_weights(const float* __restrict__ W, int ci_pad, int co_pad, bf16* __restrict__ Wf,
                               bf16* __restrict__ Wr) {
  const int total = 9 * co_pad * ci_pad;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int t = e / (co_pad * ci_pad), rem = e - t * co_pad * ci_pad;
    const int co = rem / ci_pad, ci = rem - co * ci_pad;
    const bf16 w = __float2bfloat16(W[e]);
    Wf[e] = w;
    if (Wr) Wr[(size_t(8 - t) * ci_pad + ci) * co_pad + co] = w;
  }
}

}  // namespace

// --------------------------------------------------------------------------
// host side
// --------------------------------------------------------------------------
static const int kCi[5] = {2, 32, 32, 32, 32}, kCo[5] = {32, 32, 32, 32, 1};
static const int kCiPad[5] = {16, 32, 32, 32, 32}, kCoPad[5] = {32, 32, 32, 32, 16};

int64_t cnn_param_count_padded() {
  int64_t c = 0;
  for (int l = 0; l < 5; ++l) c += 9LL * kCoPad[l] * kCiPad[l] + kCoPad[l];
  return c;
}

int64_t cnn_param_count() {
  int64_t c = 0;
  for (int l = 0; l < 5; ++l) c += 9LL * kCo[l] * kCi[l] + kCo[l];
  return c;
}

sg_status Cnn::init(const std::vector<double>& logdiag, int H_, int W_, const std::vector<int32_t>& rowptr,
                    const std::vector<int32_t>& colidx, const std::vector<double>& a0) {
  H = H_;
  W = W_;
  SG_TRY(A0.upload(int64_t(H_) * W_, int64_t(H_) * W_, rowptr, colidx, a0));
  const int64_t np = cnn_param_count_padded();
  SG_TRY(params.alloc(np * 4));
  SG_TRY(grads.alloc(np * 4));
  SG_TRY(adam_m.alloc(np * 4));
  SG_TRY(adam_v.alloc(np * 4));
  int64_t off = 0;
  for (int l = 0; l < 5; ++l) {
    woff[l] = off;
    off += 9LL * kCoPad[l] * kCiPad[l];
    boff[l] = off;
    off += kCoPad[l];
    SG_TRY(wf[l].alloc(size_t(9) * kCoPad[l] * kCiPad[l] * 2));
    SG_TRY(wr[l].alloc(size_t(9) * kCoPad[l] * kCiPad[l] * 2));
    SG_TRY(wtc[l].alloc(size_t(9) * kCoPad[l] * kCiPad[l] * 2));
    SG_TRY(wtcr[l].alloc(size_t(9) * kCoPad[l] * kCiPad[l] * 2));
  }
  std::vector<float> ld(logdiag.begin(), logdiag.end());
  SG_TRY(logd.alloc(ld.size() * 4));
  SG_CUDA(cudaMemcpy(logd.ptr, ld.data(), ld.size() * 4, cudaMemcpyHostToDevice));
  SG_TRY(sumsq.alloc(4096 * 8));
  SG_TRY(lossbuf.alloc(2 * 4096 * 8));
  SG_TRY(tcerr.alloc(16));
  SG_TRY(conv_tc_attrs());
  ready = true;
  return SG_OK;
}

sg_status Cnn::reserve(int nimg) {
  if (nimg <= cap) return SG_OK;
  const size_t npix = size_t(H) * W;
  SG_TRY(act[0].alloc(size_t(nimg) * npix * 16 * 2));
  for (int l = 1; l < 5; ++l) SG_TRY(act[l].alloc(size_t(nimg) * npix * 32 * 2));
  SG_TRY(gbuf[0].alloc(size_t(nimg) * npix * 32 * 2));
  SG_TRY(gbuf[1].alloc(size_t(nimg) * npix * 32 * 2));
  SG_TRY(out.alloc(size_t(nimg) * npix * 4));
  SG_TRY(ztgt.alloc(size_t(nimg) * npix * 4));
  for (DevBuf* b : {&ebuf, &aebuf, &azbuf}) SG_TRY(b->alloc(size_t(nimg) * npix * 4));
  if (nimg > 4096) {
    SG_TRY(sumsq.alloc(size_t(nimg) * 8));
    SG_TRY(lossbuf.alloc(size_t(2) * nimg * 8));
  }
  cap = nimg;
  return SG_OK;
}

// oracle layout [l]: W [3][3][ci][co], b [co]  <->  padded [tap][co][ci]
sg_status Cnn::set_weights(const float* host, cudaStream_t st) {
  std::vector<float> pad(cnn_param_count_padded(), 0.f);
  int64_t src = 0;
  for (int l = 0; l < 5; ++l) {
    for (int t = 0; t < 9; ++t)
      for (int ci = 0; ci < kCi[l]; ++ci)
        for (int co = 0; co < kCo[l]; ++co)
          pad[woff[l] + (int64_t(t) * kCoPad[l] + co) * kCiPad[l] + ci] = host[src + (int64_t(t) * kCi[l] + ci) * kCo[l] + co];
    src += 9LL * kCi[l] * kCo[l];
    for (int co = 0; co < kCo[l]; ++co) pad[boff[l] + co] = host[src + co];
    src += kCo[l];
  }
  SG_CUDA(cudaMemcpyAsync(params.ptr, pad.data(), pad.size() * 4, cudaMemcpyHostToDevice, st));
  SG_CUDA(cudaMemsetAsync(adam_m.ptr, 0, adam_m.bytes, st));
  SG_CUDA(cudaMemsetAsync(adam_v.ptr, 0, adam_v.bytes, st));
  adam_t = 0;
  trained = true;
  return pack(st);
}

sg_status Cnn::get_weights(float* host, bool grad, cudaStream_t st) {
  std::vector<float> pad(cnn_param_count_padded());
  SG_CUDA(cudaMemcpyAsync(pad.data(), grad ? grads.ptr : params.ptr, pad.size() * 4, cudaMemcpyDeviceToHost, st));
  SG_CUDA(cudaStreamSynchronize(st));
  int64_t dst = 0;
  for (int l = 0; l < 5; ++l) {
    for (int t = 0; t < 9; ++t)
      for (int ci = 0; ci < kCi[l]; ++ci)
        for (int co = 0; co < kCo[l]; ++co)
          host[dst + (int64_t(t) * kCi[l] + ci) * kCo[l] + co] = pad[woff[l] + (int64_t(t) * kCoPad[l] + co) * kCiPad[l] + ci];
    dst += 9LL * kCi[l] * kCo[l];
    for (int co = 0; co < kCo[l]; ++co) host[dst + co] = pad[boff[l] + co];
    dst += kCo[l];
  }
  return SG_OK;
}

sg_status Cnn::pack(cudaStream_t st) {
  for (int l = 0; l < 5; ++l) {
    k_pack_weights<<<64, 256, 0, st>>>(dp<float>(params) + woff[l], kCiPad[l], kCoPad[l], dp<bf16>(wf[l]),
                                      dp<bf16>(wr[l])); note_launch();
    SG_CUDA(cudaGetLastError());
    SG_TRY(conv_tc_pack(dp<float>(params) + woff[l], kCiPad[l], kCoPad[l], wtc[l].ptr, false, st));
    if (l > 0) SG_TRY(conv_tc_pack(dp<float>(params) + woff[l], kCiPad[l], kCoPad[l], wtcr[l].ptr, true, st));
  }
  return SG_OK;
}

// forward over nimg images already packed in act[0]; FP32 output in out
sg_status Cnn::forward(int nimg, cudaStream_t st) {
  dim3 grid(unsigned((W + TW - 1) / TW), unsigned((H + TH - 1) / TH), unsigned(nimg));
  const float* b[5];
  for (int l = 0; l < 5; ++l) b[l] = dp<float>(params) + boff[l];
  if (use_tc) {
    for (int l = 0; l < 5; ++l)
      SG_TRY(conv_tc_layer(l, act[l].ptr, wtc[l].ptr, b[l], l < 4 ? act[l + 1].ptr : nullptr,
                           l == 4 ? dp<float>(out) : nullptr, H, W, nimg, dp<int>(tcerr), wait_limit, st));
    return SG_OK;
  }
  k_conv<16, 32, 0><<<grid, 128, 0, st>>>(dp<bf16>(act[0]), dp<bf16>(wf[0]), b[0], nullptr, dp<bf16>(act[1]), nullptr, H,
                                          W); note_launch();
  for (int l = 1; l < 4; ++l) {
    k_conv<32, 32, 0><<<grid, 128, 0, st>>>(dp<bf16>(act[l]), dp<bf16>(wf[l]), b[l], nullptr, dp<bf16>(act[l + 1]),
                                            nullptr, H, W); note_launch();
  }
  k_conv<32, 16, 1><<<grid, 128, 0, st>>>(dp<bf16>(act[4]), dp<bf16>(wf[4]), b[4], nullptr, nullptr, dp<float>(out), H,
                                          W); note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

// gradients of all weights given dL/dy (16-channel BF16 image in gbuf[0])
sg_status Cnn::backward(int nimg, cudaStream_t st) {
  SG_CUDA(cudaMemsetAsync(grads.ptr, 0, grads.bytes, st));
  dim3 grid(unsigned((W + TW - 1) / TW), unsigned((H + TH - 1) / TH), unsigned(nimg));
  const unsigned wg_blocks = 4 * 152;
  int cur = 0;  // gbuf[cur] holds dL/d(output of layer l)
  for (int l = 4; l >= 0; --l) {
    float* dW = dp<float>(grads) + woff[l];
    float* db = dp<float>(grads) + boff[l];
    const bf16* X = dp<bf16>(act[l]);
    const bf16* G = dp<bf16>(gbuf[cur]);
    if (use_tc)
      SG_TRY(conv_tc_wgrad(l, X, G, dW, db, H, W, nimg, dp<int>(tcerr), wait_limit, st));
    else if (l == 4)
      k_conv_wgrad<32, 16><<<wg_blocks, 128, 0, st>>>(X, G, dW, db, H, W, nimg);
    else if (l == 0)
      k_conv_wgrad<16, 32><<<wg_blocks, 128, 0, st>>>(X, G, dW, db, H, W, nimg);
    else
      k_conv_wgrad<32, 32><<<wg_blocks, 128, 0, st>>>(X, G, dW, db, H, W, nimg);
    if (!use_tc) note_launch();
    SG_CUDA(cudaGetLastError());
    if (l == 0) break;
    // dL/d(input of layer l) masked by the ReLU that produced it
    bf16* Gn = dp<bf16>(gbuf[cur ^ 1]);
    if (use_tc) {
      SG_TRY(conv_tc_dgrad(l, G, wtcr[l].ptr, X, Gn, H, W, nimg, dp<int>(tcerr), wait_limit, st));
      cur ^= 1;
      continue;
    }
    if (l == 4)
      k_conv<16, 32, 2><<<grid, 128, 0, st>>>(G, dp<bf16>(wr[l]), nullptr, X, Gn, nullptr, H, W);
    else
      k_conv<32, 32, 2><<<grid, 128, 0, st>>>(G, dp<bf16>(wr[l]), nullptr, X, Gn, nullptr, H, W);
    note_launch();
    SG_CUDA(cudaGetLastError());
    cur ^= 1;
  }
  return SG_OK;
}

template <typename T>
sg_status Cnn::pack_input(const T* R, int64_t ld, int nimg, cudaStream_t st) {
  const int64_t n = int64_t(H) * W;
  SG_CUDA(cudaMemsetAsync(sumsq.ptr, 0, size_t(nimg) * 8, st));
  k_col_sumsq<T><<<dim3(64, unsigned(nimg)), 256, 0, st>>>(R, ld, n, dp<double>(sumsq)); note_launch();
  k_pack_input<T><<<dim3(unsigned((n + 255) / 256), unsigned(nimg)), 256, 0, st>>>(
      R, ld, n, dp<double>(sumsq), dp<float>(logd), dp<bf16>(act[0])); note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

sg_status Cnn::scale_targets(const float* Z, int64_t ld, int nimg, cudaStream_t st) {
  const int64_t n = int64_t(H) * W;
  k_scale_targets<<<dim3(unsigned((n + 255) / 256), unsigned(nimg)), 256, 0, st>>>(Z, ld, n, dp<double>(sumsq),
                                                                                  dp<float>(ztgt)); note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

template <typename T>
sg_status Cnn::unpack_output(T* Z, int64_t ld, int nimg, cudaStream_t st) {
  const int64_t n = int64_t(H) * W;
  k_unpack_output<T><<<dim3(unsigned((ld + 255) / 256), unsigned(nimg)), 256, 0, st>>>(dp<float>(out), n,
                                                                                      dp<double>(sumsq), Z, ld); note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

sg_status Cnn::loss_and_grad(int nimg, double* host_loss, cudaStream_t st) {
  const float* Zs = dp<float>(ztgt);
  const int64_t npix = int64_t(H) * W;
  double* num = dp<double>(lossbuf);
  double* den = num + nimg;
  SG_CUDA(cudaMemsetAsync(num, 0, size_t(2) * nimg * 8, st));
  const dim3 gimg(unsigned((npix + 255) / 256), unsigned(nimg));
  if (loss_kind == 0) {
    const int64_t cnt = int64_t(nimg) * npix;
    k_diff<<<4 * 152, 256, 0, st>>>(dp<float>(out), Zs, dp<float>(ebuf), cnt); note_launch();
    SG_TRY(spmm<float>(A0, dp<float>(ebuf), npix, nullptr, 0, dp<float>(aebuf), npix, nimg, 0, st));
    SG_TRY(spmm<float>(A0, Zs, npix, nullptr, 0, dp<float>(azbuf), npix, nimg, 0, st));
    k_energy_parts<<<dim3(64, unsigned(nimg)), 256, 0, st>>>(dp<float>(ebuf), dp<float>(aebuf), Zs, dp<float>(azbuf),
                                                             npix, num, den); note_launch();
    k_energy_grad<<<gimg, 256, 0, st>>>(dp<float>(aebuf), npix, den, dp<bf16>(gbuf[0])); note_launch();
  } else {
    k_loss_parts<<<dim3(64, unsigned(nimg)), 256, 0, st>>>(dp<float>(out), Zs, npix, num, den); note_launch();
    k_loss_grad<<<gimg, 256, 0, st>>>(dp<float>(out), Zs, npix, den, dp<bf16>(gbuf[0])); note_launch();
  }
  SG_CUDA(cudaGetLastError());
  if (host_loss) {
    std::vector<double> h(size_t(2) * nimg);
    SG_CUDA(cudaMemcpyAsync(h.data(), num, h.size() * 8, cudaMemcpyDeviceToHost, st));
    SG_CUDA(cudaStreamSynchronize(st));
    double L = 0.0;
    for (int i = 0; i < nimg; ++i) L += h[nimg + i] > 0 ? h[i] / h[nimg + i] : 0.0;
    *host_loss = L;
  }
  return SG_OK;
}

sg_status Cnn::adam(float lr, cudaStream_t st) {
  ++adam_t;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, float(adam_t)), c2 = 1.f - std::pow(b2, float(adam_t));
  k_adam<<<4 * 152, 256, 0, st>>>(dp<float>(params), dp<float>(grads), dp<float>(adam_m), dp<float>(adam_v),
                                  cnn_param_count_padded(), lr, b1, b2, 1e-8f, c1, c2); note_launch();
  SG_CUDA(cudaGetLastError());
  return pack(st);
}

template <typename T>
sg_status cnn_smooth(sg_problem* pr, const Precond& pc, const T* R, int64_t ld, T* Z, bool transform,
                     cudaStream_t st) {
  if (!pr->cnn || !pr->cnn->trained) {
    set_error("learned smoother: no weights");
    return SG_ERR_ARG;
  }
  Cnn& c = *pr->cnn;
  SG_TRY(c.reserve(pr->P));
  SG_TRY(c.pack_input<T>(R, ld, pr->P, st));
  SG_TRY(c.forward(pr->P, st));
  SG_TRY(c.unpack_output<T>(Z, ld, pr->P, st));
  if (transform) {
    const T* M = sizeof(T) == 8 ? reinterpret_cast<const T*>(pc.gtcnn64.ptr) : reinterpret_cast<const T*>(pc.gtcnn32.ptr);
    SG_TRY(node_transform<T>(Z, ld, pr->n, pr->P, M, st));
  }
  return SG_OK;
}

static uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

std::vector<float> cnn_he_init(uint64_t seed) {
  std::vector<float> w(cnn_param_count(), 0.f);
  uint64_t s = seed;
  auto uni = [&]() { return (double(splitmix64(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0); };
  int64_t off = 0;
  for (int l = 0; l < 5; ++l) {
    const int64_t nw = 9LL * kCi[l] * kCo[l];
    const double sd = std::sqrt(2.0 / (9.0 * kCi[l]));
    for (int64_t i = 0; i < nw; ++i) {
      const double u1 = uni(), u2 = uni();
      w[off + i] = float(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
    }
    off += nw + kCo[l];
  }
  return w;
}

void cnn_free(sg_problem* pr) {
  delete pr->cnn;
  pr->cnn = nullptr;
}

template sg_status cnn_smooth<float>(sg_problem*, const Precond&, const float*, int64_t, float*, bool, cudaStream_t);
template sg_status cnn_smooth<double>(sg_problem*, const Precond&, const double*, int64_t, double*, bool,
                                      cudaStream_t);
template sg_status Cnn::pack_input<float>(const float*, int64_t, int, cudaStream_t);
template sg_status Cnn::pack_input<double>(const double*, int64_t, int, cudaStream_t);
template sg_status Cnn::unpack_output<float>(float*, int64_t, int, cudaStream_t);
template sg_status Cnn::unpack_output<double>(double*, int64_t, int, cudaStream_t);

}  // namespace sg
