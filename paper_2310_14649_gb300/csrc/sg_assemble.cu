// Device assembly of the stiffness matrices A_k of every input PCE term
// (Sec. 2.1, Eqs. inputlogn and Galerkin_L_exp) on the shared 5-point
// pattern, stored slot-major (ELL) for the operator apply.
//
// c_bar_k(e) = c_0(e) prod_i g_i(e)^{alpha_ki} / sqrt(alpha_ki!),
// c_0(e) = exp(g0 + 1/2 sum_i g_i(e)^2)       (lognormal input PCE)
// A_k[r][c] = sum_{triangles e containing edge rc} c_bar_k(e) K_e[r][c]
// with the unit P1 element matrices of the two right triangles of a cell.
#include <algorithm>
#include <cmath>

#include "sg_internal.h"
#include "sg_stencil.h"

namespace sg {

sg_status DevBuf::alloc(size_t nbytes) {
  free_();
  if (nbytes == 0) nbytes = 16;
  cudaError_t e = cudaMalloc(&ptr, nbytes);
  if (e != cudaSuccess) {
    ptr = nullptr;
    set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    return SG_ERR_NOMEM;
  }
  bytes = nbytes;
  cudaMemset(ptr, 0, nbytes);
  return SG_OK;
}

void DevBuf::free_() {
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
  bytes = 0;
}

namespace {

// c_bar for input terms [k0, k0 + kn) on every triangle: out[(k - k0) * E + e]
__global__ void k_cbar(const double* __restrict__ gfield, const int* __restrict__ mi_in,
                       const double* __restrict__ inv_sqrt_fact, int L, int64_t E, double g0,
                       int k0, int kn, double* __restrict__ out) {
  int64_t total = int64_t(kn) * E;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    int kl = int(t / E);
    int64_t e = t - int64_t(kl) * E;
    int k = k0 + kl;
    double s2 = 0.0, prod = 1.0;
    for (int i = 0; i < L; ++i) {
      double gi = gfield[int64_t(i) * E + e];
      s2 += gi * gi;
      int d = mi_in[k * L + i];
      for (int j = 0; j < d; ++j) prod *= gi;
    }
    out[t] = exp(g0 + 0.5 * s2) * prod * inv_sqrt_fact[k];
  }
}

// Five-slot ELL values for input terms [k0, k0 + kn).  Slot order (ascending
// column): south, west, centre, east, north.  Thread per (row, term).
__global__ void k_fine_ell(const double* __restrict__ cb, int N, int64_t n, int64_t ldr, int k0,
                           int kn, double* __restrict__ v64, float* __restrict__ v32) {
  const int m = N - 1;
  const int64_t E = 2LL * N * N;
  int64_t total = int64_t(kn) * n;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    int kl = int(t / n);
    int64_t r = t - int64_t(kl) * n;
    int i = int(r % m) + 1, j = int(r / m) + 1;
    const double* c = cb + int64_t(kl) * E;
    double v[5];
    p1_stencil<double>(c, N, i, j, v);
    int k = k0 + kl;
    for (int s = 0; s < 5; ++s) {
      int64_t idx = (int64_t(k) * 5 + s) * ldr + r;
      v64[idx] = v[s];
      v32[idx] = float(v[s]);
    }
  }
}

// Conductances of the edge-flux form for input terms [k0, k0 + kn): the
// horizontal edge (i,j)-(i+1,j) (i = 0..N-1, j = 1..N-1) at (j-1) N + i,
// half the sum of the lower triangle of cell (i,j) and the upper one of
// cell (i,j-1); the vertical edge (i,j)-(i,j+1) (i = 1..N-1, j = 0..N-1) at
// N (N-1) + j (N-1) + i - 1, half the sum of the upper triangle of cell
// (i,j) and the lower one of cell (i-1,j).  A row of A_k is then the sum
// over its four edges of w (x_r - x_neighbour) (the rows of the P1 element
// matrices sum to zero).  Thread per (term, edge).
template <typename T>
__global__ void k_flux_values(const double* __restrict__ cb, int N, int64_t vkst, int k0, int kn,
                              T* __restrict__ v32) {
  const int m = N - 1;
  const int64_t E = 2LL * N * N, ne = 2LL * N * m, total = int64_t(kn) * ne;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int kl = int(t / ne);
    const int64_t e = t - int64_t(kl) * ne;
    const double* c = cb + int64_t(kl) * E;
    auto lo = [&](int ci, int cj) { return c[2LL * (int64_t(cj) * N + ci)]; };
    auto up = [&](int ci, int cj) { return c[2LL * (int64_t(cj) * N + ci) + 1]; };
    double v;
    if (e < int64_t(N) * m) {
      const int i = int(e % N), j = int(e / N) + 1;
      v = 0.5 * (lo(i, j) + up(i, j - 1));
    } else {
      const int64_t e2 = e - int64_t(N) * m;
      const int i = int(e2 % m) + 1, j = int(e2 / m);
      v = 0.5 * (up(i, j) + lo(i - 1, j));
    }
    v32[int64_t(k0 + kl) * vkst + e] = T(v);
  }
}

}  // namespace

sg_status flux_build(sg_problem* pr) {
  Ell& A = pr->flux;
  if (A.v32.ptr) return SG_OK;
  const int S = 4, K = pr->K, N = pr->N, m = N - 1;
  const int64_t n = pr->n, E = pr->E, ldr = pr->fine.ldr, ne = 2LL * N * m;
  A.S = S;
  A.n = n;
  A.ldr = ldr;
  A.vkst = round_up(ne, 64);
  std::vector<int32_t> col(size_t(S) * ldr, -1), vidx(size_t(S) * ldr, 0);
  for (int64_t r = 0; r < n; ++r) {
    const int i = int(r % m) + 1, j = int(r / m) + 1;
    col[0 * ldr + r] = int32_t(i < m ? r + 1 : -1);
    vidx[0 * ldr + r] = int32_t(int64_t(j - 1) * N + i);
    col[1 * ldr + r] = int32_t(i > 1 ? r - 1 : -1);
    vidx[1 * ldr + r] = int32_t(int64_t(j - 1) * N + i - 1);
    col[2 * ldr + r] = int32_t(j < m ? r + m : -1);
    vidx[2 * ldr + r] = int32_t(int64_t(N) * m + int64_t(j) * m + i - 1);
    col[3 * ldr + r] = int32_t(j > 1 ? r - m : -1);
    vidx[3 * ldr + r] = int32_t(int64_t(N) * m + int64_t(j - 1) * m + i - 1);
  }
  SG_TRY(A.col.alloc(col.size() * 4));
  SG_TRY(A.vidx.alloc(vidx.size() * 4));
  SG_CUDA(cudaMemcpy(A.col.ptr, col.data(), col.size() * 4, cudaMemcpyHostToDevice));
  SG_CUDA(cudaMemcpy(A.vidx.ptr, vidx.data(), vidx.size() * 4, cudaMemcpyHostToDevice));
  DevBuf v;
  SG_TRY(v.alloc(size_t(K) * A.vkst * 4));
  SG_CUDA(cudaMemset(v.ptr, 0, size_t(K) * A.vkst * 4));
  const int KC = 32;
  DevBuf dcb;
  SG_TRY(dcb.alloc(size_t(KC) * E * sizeof(double)));
  for (int k0 = 0; k0 < K; k0 += KC) {
    const int kn = std::min(KC, K - k0);
    SG_TRY(element_coefficients(pr, k0, kn, dcb.as<double>(), nullptr));
    k_flux_values<float><<<4 * 152, 256>>>(dcb.as<double>(), N, A.vkst, k0, kn, v.as<float>());
    note_launch();
    SG_CUDA(cudaGetLastError());
  }
  SG_CUDA(cudaDeviceSynchronize());
  A.v32 = std::move(v);
  return SG_OK;
}

sg_status flux_values64(sg_problem* pr, double* w, int64_t vkst) {
  const int K = pr->K, N = pr->N, KC = 32;
  DevBuf dcb;
  SG_TRY(dcb.alloc(size_t(KC) * pr->E * sizeof(double)));
  for (int k0 = 0; k0 < K; k0 += KC) {
    const int kn = std::min(KC, K - k0);
    SG_TRY(element_coefficients(pr, k0, kn, dcb.as<double>(), nullptr));
    k_flux_values<double><<<4 * 152, 256>>>(dcb.as<double>(), N, vkst, k0, kn, w);
    note_launch();
    SG_CUDA(cudaGetLastError());
  }
  SG_CUDA(cudaDeviceSynchronize());
  return SG_OK;
}

sg_status assemble_fine(sg_problem* pr) {
  const int S = 5, K = pr->K, L = pr->L, N = pr->N;
  const int64_t n = pr->n, E = pr->E, ldr = round_up(n, 64);
  Ell& A = pr->fine;
  A.S = S;
  A.n = n;
  A.ldr = ldr;
  // column indices: neighbour or the row itself for padding slots
  std::vector<int32_t> col(size_t(S) * ldr, 0);
  const int m = N - 1;
  for (int64_t r = 0; r < ldr; ++r) {
    if (r >= n) {
      for (int s = 0; s < S; ++s) col[s * ldr + r] = 0;
      continue;
    }
    int i = int(r % m) + 1, j = int(r / m) + 1;
    col[0 * ldr + r] = int32_t(j > 1 ? r - m : r);
    col[1 * ldr + r] = int32_t(i > 1 ? r - 1 : r);
    col[2 * ldr + r] = int32_t(r);
    col[3 * ldr + r] = int32_t(i < m ? r + 1 : r);
    col[4 * ldr + r] = int32_t(j < m ? r + m : r);
  }
  SG_TRY(A.col.alloc(col.size() * sizeof(int32_t)));
  SG_CUDA(cudaMemcpy(A.col.ptr, col.data(), col.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  SG_TRY(A.v64.alloc(size_t(K) * S * ldr * sizeof(double)));
  SG_TRY(A.v32.alloc(size_t(K) * S * ldr * sizeof(float)));

  const int KC = 32;
  DevBuf dcb;
  SG_TRY(dcb.alloc(size_t(KC) * E * sizeof(double)));
  for (int k0 = 0; k0 < K; k0 += KC) {
    int kn = std::min(KC, K - k0);
    SG_TRY(element_coefficients(pr, k0, kn, dcb.as<double>(), nullptr));
    k_fine_ell<<<4 * 152, 256>>>(dcb.as<double>(), N, n, ldr, k0, kn, A.v64.as<double>(),
                                 A.v32.as<float>()); note_launch();
    SG_CUDA(cudaGetLastError());
  }
  SG_CUDA(cudaDeviceSynchronize());
  return SG_OK;
}

sg_status element_coefficients(sg_problem* pr, int k0, int kn, double* out, cudaStream_t st) {
  const int K = pr->K, L = pr->L;
  const int64_t E = pr->E;
  DevBuf dg, dmi, disf;
  std::vector<double> isf(K, 1.0);
  std::vector<int32_t> mi = pr->mi_in;
  if (L == 0) mi.assign(1, 0);
  for (int k = 0; k < K; ++k) {
    double f = 1.0;
    for (int i = 0; i < L; ++i)
      for (int v = 2; v <= mi[size_t(k) * L + i]; ++v) f *= v;
    isf[k] = 1.0 / std::sqrt(f);
  }
  SG_TRY(dg.alloc(std::max<size_t>(1, pr->gfield.size()) * sizeof(double)));
  if (!pr->gfield.empty())
    SG_CUDA(cudaMemcpy(dg.ptr, pr->gfield.data(), pr->gfield.size() * sizeof(double),
                       cudaMemcpyHostToDevice));
  SG_TRY(dmi.alloc(mi.size() * sizeof(int32_t)));
  SG_CUDA(cudaMemcpy(dmi.ptr, mi.data(), mi.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  SG_TRY(disf.alloc(isf.size() * sizeof(double)));
  SG_CUDA(cudaMemcpy(disf.ptr, isf.data(), isf.size() * sizeof(double), cudaMemcpyHostToDevice));
  k_cbar<<<4 * 152, 256, 0, st>>>(dg.as<double>(), dmi.as<int>(), disf.as<double>(), L, E, pr->g0, k0, kn, out);
  note_launch();
  SG_CUDA(cudaGetLastError());
  SG_CUDA(cudaStreamSynchronize(st));
  return SG_OK;
}

// Triples re-ordered by (a, k, b) and split into input-term chunks of kc for
// the shared-memory apply; off[a * (nchunk + 1) + c] is the first triple of
// output a with k >= c * kc.
sg_status build_triple_tables(sg_problem* pr, TripleTables& t, int S) {
  const int P = pr->P, K = pr->K;
  const int64_t T = pr->T;
  // chunk of input terms: the FP64 tile of 32 rows must fit in shared memory
  const size_t budget = 200 * 1024;
  const size_t fixed = size_t(S * P + P) * 32 * sizeof(double);
  int kc = 1;
  if (fixed < budget) kc = int((budget - fixed) / (size_t(S) * 32 * sizeof(double)));
  kc = std::max(1, std::min(kc, K));
  if (kc >= 8) kc = kc / 8 * 8;
  t.kc = kc;
  t.nchunk = (K + kc - 1) / kc;
  std::vector<int64_t> order(T);
  for (int64_t i = 0; i < T; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int64_t x, int64_t y) {
    const int32_t* a = &pr->kab[3 * x];
    const int32_t* b = &pr->kab[3 * y];
    if (a[1] != b[1]) return a[1] < b[1];
    if (a[0] != b[0]) return a[0] < b[0];
    return a[2] < b[2];
  });
  std::vector<int32_t> tk(T), tb(T), off(size_t(P) * (t.nchunk + 1));
  std::vector<double> g64(T);
  std::vector<float> g32(T);
  for (int64_t i = 0; i < T; ++i) {
    tk[i] = pr->kab[3 * order[i] + 0];
    tb[i] = pr->kab[3 * order[i] + 2];
    g64[i] = pr->g[order[i]];
    g32[i] = float(g64[i]);
  }
  int64_t pos = 0;
  for (int a = 0; a < P; ++a) {
    for (int c = 0; c <= t.nchunk; ++c) {
      int kstart = std::min(c * kc, K);
      while (pos < T && pr->kab[3 * order[pos] + 1] == a && tk[pos] < kstart) ++pos;
      off[size_t(a) * (t.nchunk + 1) + c] = int32_t(pos);
    }
    while (pos < T && pr->kab[3 * order[pos] + 1] == a) ++pos;
  }
  SG_TRY(t.tk.alloc(T * sizeof(int32_t)));
  SG_TRY(t.tb.alloc(T * sizeof(int32_t)));
  SG_TRY(t.g64.alloc(T * sizeof(double)));
  SG_TRY(t.g32.alloc(T * sizeof(float)));
  SG_TRY(t.off.alloc(off.size() * sizeof(int32_t)));
  SG_CUDA(cudaMemcpy(t.tk.ptr, tk.data(), T * sizeof(int32_t), cudaMemcpyHostToDevice));
  SG_CUDA(cudaMemcpy(t.tb.ptr, tb.data(), T * sizeof(int32_t), cudaMemcpyHostToDevice));
  SG_CUDA(cudaMemcpy(t.g64.ptr, g64.data(), T * sizeof(double), cudaMemcpyHostToDevice));
  SG_CUDA(cudaMemcpy(t.g32.ptr, g32.data(), T * sizeof(float), cudaMemcpyHostToDevice));
  SG_CUDA(cudaMemcpy(t.off.ptr, off.data(), off.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  return SG_OK;
}

}  // namespace sg
