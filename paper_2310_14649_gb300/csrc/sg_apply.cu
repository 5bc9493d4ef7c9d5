// Galerkin operator apply (Sec. 2.1, Eq. Galerkin_L_exp, Kronecker form):
//     Y = sum_k A_k X G_k^T,
//     y_r[a] = sum_{s} sum_{(k,a,b) in T} v_k^{r,s} g_kab x_{col(r,s)}[b],
// over an ELL family of K matrices with S slots per row.
//
// Shared-memory tile kernel: one CTA owns 32 consecutive rows (lane = row)
// and all P output modes; its warps split the output modes.  The 32-row
// tile of X gathered through the slot columns (S x P values per row) and a
// chunk of kc input terms of the matrix values (S x kc per row) are staged
// in shared memory, laid out [.][lane] so every access is bank-conflict
// free; the triple list of each output mode is walked warp-uniformly.
#include <algorithm>

#include "sg_solver.h"

namespace sg {

namespace {

template <typename T>
struct ApplyArgs {
  const int* col;
  const T* V;
  int64_t ldr, n;
  int S, K, P;
  const T* X;
  int64_t ldx;
  const T* F;  // optional: Y = F - A(X)
  int64_t ldf;
  T* Y;
  int64_t ldy;
  const int* tk;
  const int* tb;
  const T* tg;
  const int* off;
  int kc, nchunk;
};

template <typename T>
__global__ void __launch_bounds__(256) k_apply_tile(ApplyArgs<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* xs = reinterpret_cast<T*>(smem_raw);  // [S][P][32]
  T* vs = xs + size_t(p.S) * p.P * 32;     // [S][kc][32]
  T* ys = vs + size_t(p.S) * p.kc * 32;    // [P][32]
  const int lane = threadIdx.x, w = threadIdx.y, W = blockDim.y;
  const int64_t r = int64_t(blockIdx.x) * 32 + lane;
  const bool valid = r < p.n;
  const int S = p.S, P = p.P, kc = p.kc;

  for (int sb = w; sb < S * P; sb += W) {
    int s = sb / P, b = sb - s * P;
    T v = T(0);
    if (valid) v = p.X[int64_t(b) * p.ldx + p.col[int64_t(s) * p.ldr + r]];
    xs[sb * 32 + lane] = v;
  }
  for (int a = w; a < P; a += W) ys[a * 32 + lane] = T(0);

  for (int c = 0; c < p.nchunk; ++c) {
    const int k0 = c * kc;
    __syncthreads();
    for (int sk = w; sk < S * kc; sk += W) {
      int s = sk / kc, kk = sk - s * kc, k = k0 + kk;
      T v = T(0);
      if (valid && k < p.K) v = p.V[(int64_t(k) * S + s) * p.ldr + r];
      vs[sk * 32 + lane] = v;
    }
    __syncthreads();
    for (int a = w; a < P; a += W) {
      T acc = ys[a * 32 + lane];
      const int t0 = p.off[a * (p.nchunk + 1) + c], t1 = p.off[a * (p.nchunk + 1) + c + 1];
      for (int t = t0; t < t1; ++t) {
        const int kk = p.tk[t] - k0, b = p.tb[t];
        T sum = T(0);
        for (int s = 0; s < S; ++s) sum += vs[(s * kc + kk) * 32 + lane] * xs[(s * P + b) * 32 + lane];
        acc += p.tg[t] * sum;
      }
      ys[a * 32 + lane] = acc;
    }
  }
  __syncthreads();
  if (valid) {
    for (int a = w; a < P; a += W) {
      T y = ys[a * 32 + lane];
      if (p.F) y = p.F[int64_t(a) * p.ldf + r] - y;
      p.Y[int64_t(a) * p.ldy + r] = y;
    }
  }
}

template <typename T> const T* vals_of(const Ell& A);
template <> const double* vals_of<double>(const Ell& A) { return A.v64.as<double>(); }
template <> const float* vals_of<float>(const Ell& A) { return A.v32.as<float>(); }
template <typename T> const T* g_of(const TripleTables& t);
template <> const double* g_of<double>(const TripleTables& t) { return t.g64.as<double>(); }
template <> const float* g_of<float>(const TripleTables& t) { return t.g32.as<float>(); }

}  // namespace

template <typename T>
sg_status apply_ell(const Ell& A, const TripleTables& tri, int P, int K, const T* X, int64_t ldx,
                    const T* F, int64_t ldf, T* Y, int64_t ldy, cudaStream_t st) {
  ApplyArgs<T> a;
  a.col = A.col.as<int>();
  a.V = vals_of<T>(A);
  a.ldr = A.ldr;
  a.n = A.n;
  a.S = A.S;
  a.K = K;
  a.P = P;
  a.X = X;
  a.ldx = ldx;
  a.F = F;
  a.ldf = ldf;
  a.Y = Y;
  a.ldy = ldy;
  a.tk = tri.tk.as<int>();
  a.tb = tri.tb.as<int>();
  a.tg = g_of<T>(tri);
  a.off = tri.off.as<int>();
  a.kc = tri.kc;
  a.nchunk = tri.nchunk;
  const size_t smem = (size_t(A.S) * P + size_t(A.S) * tri.kc + P) * 32 * sizeof(T);
  static bool attr_set[2] = {false, false};
  bool& set = attr_set[sizeof(T) == 8 ? 1 : 0];
  if (!set) {
    SG_CUDA(cudaFuncSetAttribute(k_apply_tile<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 227 * 1024));
    set = true;
  }
  const int W = std::min(8, P);
  dim3 block(32, W);
  dim3 grid(unsigned((A.n + 31) / 32));
  if (A.n == 0) return SG_OK;
  k_apply_tile<T><<<grid, block, smem, st>>>(a); note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

sg_status apply_attrs_init() {
  SG_CUDA(cudaFuncSetAttribute(k_apply_tile<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  SG_CUDA(cudaFuncSetAttribute(k_apply_tile<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  return SG_OK;
}

Profiler::~Profiler() {
  for (auto& r : pool) {
    if (r.a) cudaEventDestroy(r.a);
    if (r.b) cudaEventDestroy(r.b);
  }
}

sg_status Profiler::begin(int kind, cudaStream_t st, size_t& slot) {
  if (used == pool.size()) {
    Rec r;
    SG_CUDA(cudaEventCreate(&r.a));
    SG_CUDA(cudaEventCreate(&r.b));
    pool.push_back(r);
  }
  slot = used++;
  pool[slot].kind = kind;
  SG_CUDA(cudaEventRecord(pool[slot].a, st));
  return SG_OK;
}

sg_status Profiler::end(size_t slot, cudaStream_t st) {
  SG_CUDA(cudaEventRecord(pool[slot].b, st));
  return SG_OK;
}

sg_status Profiler::read(int kind, int64_t* launches, double* ms) {
  int64_t cnt = 0;
  double tot = 0.0;
  for (size_t i = 0; i < used; ++i) {
    if (pool[i].kind != kind) continue;
    SG_CUDA(cudaEventSynchronize(pool[i].b));
    float t = 0.0f;
    SG_CUDA(cudaEventElapsedTime(&t, pool[i].a, pool[i].b));
    tot += t;
    ++cnt;
  }
  if (launches) *launches = cnt;
  if (ms) *ms = tot;
  return SG_OK;
}

template <typename T>
sg_status apply_op(sg_problem* pr, bool coarse, const T* X, int64_t ldx, const T* F, int64_t ldf, T* Y,
                   int64_t ldy, cudaStream_t st) {
  const Ell& A = coarse ? coarse_ell(pr) : pr->fine;
  const TripleTables& tri = coarse ? coarse_tri(pr) : pr->tri;
  size_t slot = 0;
  const bool on = pr->prof.on;
  if (on) SG_TRY(pr->prof.begin((coarse ? 2 : 0) + (sizeof(T) == 8 ? 1 : 0), st, slot));
  const bool spec = pr->apply_mode != 1 && jit_eligible(pr);
  if (spec) {
    SG_TRY(jit_apply_launch(pr, (coarse ? 1 : 0) + (sizeof(T) == 8 ? 2 : 0), A, X, ldx, F, ldf, Y, ldy, st));
  } else {
    SG_TRY(apply_ell<T>(A, tri, pr->P, pr->K, X, ldx, F, ldf, Y, ldy, st));
  }
  if (on) SG_TRY(pr->prof.end(slot, st));
  return SG_OK;
}

template sg_status apply_op<double>(sg_problem*, bool, const double*, int64_t, const double*, int64_t, double*,
                                    int64_t, cudaStream_t);
template sg_status apply_op<float>(sg_problem*, bool, const float*, int64_t, const float*, int64_t, float*,
                                   int64_t, cudaStream_t);

template sg_status apply_ell<double>(const Ell&, const TripleTables&, int, int, const double*, int64_t,
                                     const double*, int64_t, double*, int64_t, cudaStream_t);
template sg_status apply_ell<float>(const Ell&, const TripleTables&, int, int, const float*, int64_t,
                                    const float*, int64_t, float*, int64_t, cudaStream_t);

}  // namespace sg
