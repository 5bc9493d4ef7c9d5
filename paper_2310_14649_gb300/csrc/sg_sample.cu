// Batched deterministic solves for Monte Carlo verification of the SG
// solution (Sec. 4.1, Fig. mcs_verify_poisson: the paper compares the SG
// mean, standard deviation and pdf with 40,000 Monte Carlo samples).
//
// Sample s draws xi_s in R^L and solves the deterministic problem
//     -div( c_s grad u_s ) = 1,  u_s = 0 on the boundary,
//     c_s(e) = exp( g0 + sum_i g_i(e) xi_{s,i} )      (the exact lognormal
// field of Eq. KLE at the element centroids, not its chaos expansion) with
// the same P1 discretisation as the SG system.  One CTA solves one sample
// entirely in shared memory by Jacobi-preconditioned conjugate gradients
// in FP32: the search direction, the edge conductances and the inverse
// diagonal live in shared memory, the iterate and the residual in registers
// (nodes r = tid + k * 1024 of the thread).
#include <algorithm>
#include <cmath>

#include "sg_internal.h"

namespace sg {
namespace {

constexpr int kSampThreads = 1024;
constexpr int kSampNodes = 10;   // nodes per thread: n <= 10240 (meshes up to N = 102)

// block-wide sums of two values (every thread receives them)
__device__ inline void block_sum2(float a, float b, double* red, double& sa, double& sb) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double x = a, y = b;
  for (int o = 16; o > 0; o >>= 1) {
    x += __shfl_xor_sync(0xffffffffu, x, o);
    y += __shfl_xor_sync(0xffffffffu, y, o);
  }
  __syncthreads();  // red is free again
  if (lane == 0) {
    red[warp] = x;
    red[32 + warp] = y;
  }
  __syncthreads();
  double u = 0.0, v = 0.0;
  for (int w = 0; w < kSampThreads / 32; ++w) {
    u += red[w];
    v += red[32 + w];
  }
  sa = u;
  sb = v;
}

// Edge conductances of the P1 stencil (Sec. 2.1): the horizontal edge
// (i,j)-(i+1,j) couples the lower triangle of cell (i,j) and the upper one
// of cell (i,j-1), wx = (c_lo(i,j) + c_up(i,j-1)) / 2; the vertical edge
// (i,j)-(i,j+1) couples the upper triangle of cell (i,j) and the lower one
// of cell (i-1,j), wy = (c_up(i,j) + c_lo(i-1,j)) / 2.  Row (i,j) of A(c):
// diagonal = the four conductances around the node, off-diagonals = minus
// the conductance of the edge (edges to boundary nodes are dropped).
// Shared memory: p [n], wx [m N], wy [N m], the inverse diagonal [n] and
// the reduction slots; x, r and A p of the thread's nodes in registers.
template <typename To>
__global__ void __launch_bounds__(kSampThreads, 1)
    k_sample_pcg(int N, int L, const double* __restrict__ gfield, double g0, const double* __restrict__ xi,
                 double h2, double rtol, int max_it, To* __restrict__ U, int64_t ldu, int* __restrict__ its_max) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = N - 1;
  const int n = m * m;
  const int64_t E = 2LL * N * N;
  float* p = reinterpret_cast<float*>(smem_raw);       // [n]
  float* wx = p + n;                                    // [m][N]: (i = 0..N-1, j = 1..m)
  float* wy = wx + int64_t(m) * N;                      // [N][m]: (i = 1..m, j = 0..m)
  float* dinv = wy + int64_t(N) * m;                    // [n]
  double* red = reinterpret_cast<double*>(dinv + n + 2);  // [64], 8-byte aligned below
  red = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(red) + 7) & ~uintptr_t(7));
  __shared__ double sxi[16];
  const int64_t s = blockIdx.x;
  if (threadIdx.x < L) sxi[threadIdx.x] = xi[s * L + threadIdx.x];
  __syncthreads();
  auto coef = [&](int ci, int cj, int upper) -> float {
    if (ci < 0 || cj < 0 || ci >= N || cj >= N) return 0.0f;
    const int64_t e = 2LL * (int64_t(cj) * N + ci) + upper;
    double a = g0;
    for (int i = 0; i < L; ++i) a += gfield[int64_t(i) * E + e] * sxi[i];
    return float(exp(a));
  };
  for (int t = threadIdx.x; t < m * N; t += kSampThreads) {
    const int i = t % N, j = t / N + 1;  // edge (i,j)-(i+1,j)
    wx[t] = 0.5f * (coef(i, j, 0) + coef(i, j - 1, 1));
  }
  for (int t = threadIdx.x; t < N * m; t += kSampThreads) {
    const int i = t % m + 1, j = t / m;  // edge (i,j)-(i,j+1)
    wy[t] = 0.5f * (coef(i, j, 1) + coef(i - 1, j, 0));
  }
  __syncthreads();
  float x[kSampNodes], r[kSampNodes];
  float rz_loc = 0.0f, bb_loc = 0.0f;
#pragma unroll
  for (int k = 0; k < kSampNodes; ++k) {
    const int node = threadIdx.x + k * kSampThreads;
    x[k] = 0.0f;
    r[k] = 0.0f;
    if (node < n) {
      const int i = node % m + 1, j = node / m + 1;
      const float d = wx[(j - 1) * N + i] + wx[(j - 1) * N + i - 1] + wy[j * m + i - 1] + wy[(j - 1) * m + i - 1];
      const float di = 1.0f / d;
      dinv[node] = di;
      r[k] = float(h2);
      p[node] = r[k] * di;
      rz_loc += r[k] * r[k] * di;
      bb_loc += r[k] * r[k];
    }
  }
  double rz, bb;
  block_sum2(rz_loc, bb_loc, red, rz, bb);
  const double tol2 = rtol * rtol * bb;
  int it = 0;
  for (; it < max_it; ++it) {
    __syncthreads();  // p complete
    float q[kSampNodes];
    float pq_loc = 0.0f;
#pragma unroll
    for (int k = 0; k < kSampNodes; ++k) {
      const int node = threadIdx.x + k * kSampThreads;
      q[k] = 0.0f;
      if (node < n) {
        const int i = node % m + 1, j = node / m + 1;
        const float we = wx[(j - 1) * N + i], ww = wx[(j - 1) * N + i - 1];
        const float wn = wy[j * m + i - 1], ws = wy[(j - 1) * m + i - 1];
        const float pc = p[node];
        float v = (we + ww + wn + ws) * pc;
        if (i > 1) v -= ww * p[node - 1];
        if (i < m) v -= we * p[node + 1];
        if (j > 1) v -= ws * p[node - m];
        if (j < m) v -= wn * p[node + m];
        q[k] = v;
        pq_loc += pc * v;
      }
    }
    double pq, dummy;
    block_sum2(pq_loc, 0.0f, red, pq, dummy);
    if (!(pq > 0.0)) break;
    const float alpha = float(rz / pq);
    float rr_loc = 0.0f, rzn_loc = 0.0f;
#pragma unroll
    for (int k = 0; k < kSampNodes; ++k) {
      const int node = threadIdx.x + k * kSampThreads;
      if (node < n) {
        x[k] += alpha * p[node];
        r[k] -= alpha * q[k];
        rr_loc += r[k] * r[k];
        rzn_loc += r[k] * r[k] * dinv[node];
      }
    }
    double rr, rzn;
    block_sum2(rr_loc, rzn_loc, red, rr, rzn);
    if (rr <= tol2) {
      ++it;
      break;
    }
    const float beta = float(rzn / rz);
    rz = rzn;
    __syncthreads();  // every thread has read p for x
#pragma unroll
    for (int k = 0; k < kSampNodes; ++k) {
      const int node = threadIdx.x + k * kSampThreads;
      if (node < n) p[node] = r[k] * dinv[node] + beta * p[node];
    }
  }
#pragma unroll
  for (int k = 0; k < kSampNodes; ++k) {
    const int node = threadIdx.x + k * kSampThreads;
    if (node < n) U[s * ldu + node] = To(x[k]);
  }
  if (threadIdx.x == 0) atomicMax(its_max, it);
}

size_t sample_smem(int N) {
  const int64_t m = N - 1;
  return size_t(2 * m * m + 2 * m * N + 2) * 4 + 64 * 8 + 8;
}

}  // namespace
}  // namespace sg

using namespace sg;

extern "C" sg_status sg_sample_solve(sg_problem* pr, const double* xi, int64_t S, sg_dtype dtype, void* U,
                                     int64_t ldu, double rtol, int max_it, int* its_max, void* stream) {
  SG_ARG(pr && xi && U, "sg_sample_solve: NULL argument");
  SG_ARG(dtype == SG_F64 || dtype == SG_F32, "sg_sample_solve: bad dtype");
  SG_ARG(S >= 0 && S <= 0x7fffffff, "sg_sample_solve: sample count out of range");
  SG_ARG(ldu >= pr->n, "sg_sample_solve: leading dimension < n");
  SG_ARG(rtol > 0 && max_it > 0, "sg_sample_solve: rtol and max_it must be > 0");
  SG_ARG(pr->L >= 1 && pr->L <= 16, "sg_sample_solve: needs 1 <= L <= 16 KL modes");
  SG_ARG(pr->n <= int64_t(kSampThreads) * kSampNodes && sample_smem(pr->N) <= 227 * 1024,
         "sg_sample_solve: the mesh is too large for one CTA per sample (N <= 102)");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the KL modes at the element centroids, once per problem
  DevBuf& g = pr->gfield_dev;
  if (!g.ptr) {
    SG_TRY(g.alloc(pr->gfield.size() * 8));
    SG_CUDA(cudaMemcpy(g.ptr, pr->gfield.data(), pr->gfield.size() * 8, cudaMemcpyHostToDevice));
  }
  DevBuf itsd;
  SG_TRY(itsd.alloc(sizeof(int)));
  SG_CUDA(cudaMemsetAsync(itsd.ptr, 0, sizeof(int), st));
  const double h = 1.0 / pr->N;
  const size_t smem = sample_smem(pr->N);
  if (S > 0) {
    if (dtype == SG_F32) {
      SG_CUDA(cudaFuncSetAttribute(k_sample_pcg<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
      k_sample_pcg<float><<<unsigned(S), kSampThreads, smem, st>>>(pr->N, pr->L, dp<double>(g), pr->g0, xi, h * h,
                                                                   rtol, max_it, static_cast<float*>(U), ldu,
                                                                   dp<int>(itsd));
    } else {
      SG_CUDA(cudaFuncSetAttribute(k_sample_pcg<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
      k_sample_pcg<double><<<unsigned(S), kSampThreads, smem, st>>>(pr->N, pr->L, dp<double>(g), pr->g0, xi, h * h,
                                                                    rtol, max_it, static_cast<double*>(U), ldu,
                                                                    dp<int>(itsd));
    }
    note_launch();
    SG_CUDA(cudaGetLastError());
  }
  int its = 0;
  SG_CUDA(cudaMemcpyAsync(&its, itsd.ptr, sizeof(int), cudaMemcpyDeviceToHost, st));
  SG_CUDA(cudaStreamSynchronize(st));
  if (its_max) *its_max = its;
  if (S > 0 && its >= max_it) {
    set_error("sg_sample_solve: a sample reached max_it before rtol");
    return SG_NOT_CONVERGED;
  }
  return SG_OK;
}
