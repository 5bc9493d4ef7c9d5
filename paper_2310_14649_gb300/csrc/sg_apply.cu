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

// ---------------------------------------------------------------------------
// Assembled FP64 apply.  The generated FP64 kernel spends two FP64
// operations per triple and slot (2,395 triples at P = 35), and GB300's FP64
// units (about 1.2 TFLOP/s) bound it; summing the K values of each stencil
// edge into its symmetric P x P block once leaves P^2 FMAs per edge (3x
// fewer FP64 operations) for (S P (P+1) / 2) doubles per row of memory.
// Block build: thread per (row, packed pair), loop over the pair's (k, g)
// list and the slots.  Apply: lane = row of a 32-row tile, warps over the
// output modes; C_ab and C_ba are one stored value, read by two warps of
// the same CTA (the second from L1).
// ---------------------------------------------------------------------------
__global__ void k_asm_build(int64_t ldr, int S, int npair, const int* __restrict__ pptr, const int* __restrict__ pk,
                            const double* __restrict__ pg, const double* __restrict__ V, double* __restrict__ C) {
  const int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int p = blockIdx.y;
  if (r >= ldr) return;
  const int e0 = pptr[p], e1 = pptr[p + 1];
  for (int s = 0; s < S; ++s) {
    double c = 0.0;
    for (int e = e0; e < e1; ++e) c += pg[e] * V[(int64_t(pk[e]) * S + s) * ldr + r];
    C[(int64_t(s) * npair + p) * ldr + r] = c;
  }
}

__global__ void __launch_bounds__(256) k_apply_asm64(int64_t n, int64_t ldr, int S, int P, int npair,
                                                      const int* __restrict__ col, const double* __restrict__ C,
                                                      const double* __restrict__ X, int64_t ldx,
                                                      const double* __restrict__ F, int64_t ldf,
                                                      double* __restrict__ Y, int64_t ldy) {
  const int64_t r = int64_t(blockIdx.x) * 32 + threadIdx.x;
  if (r >= n) return;
  for (int a = threadIdx.y; a < P; a += blockDim.y) {
    // packed index of (lo, hi), lo <= hi: off(lo) + hi with
    // off(b) = b P - b (b - 1) / 2 - b
    const int off_a = a * P - a * (a - 1) / 2 - a;
    double acc = 0.0;
    for (int s = 0; s < S; ++s) {
      const int c = col[int64_t(s) * ldr + r];
      const double* Cs = C + int64_t(s) * npair * ldr + r;
      const double* xc = X + c;
      int off_b = 0;
      for (int b = 0; b < P; ++b) {
        const int pidx = b < a ? off_b + a : off_a + b;
        acc = fma(Cs[int64_t(pidx) * ldr], xc[int64_t(b) * ldx], acc);
        off_b += P - b - 1;
      }
    }
    Y[int64_t(a) * ldy + r] = F ? F[int64_t(a) * ldf + r] - acc : acc;
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

void pair_lists(const sg_problem* pr, std::vector<int>& pptr, std::vector<int>& pk, std::vector<double>& pg) {
  const int P = pr->P;
  const int npair = P * (P + 1) / 2;
  // (k, g) list of every packed pair a <= b
  std::vector<std::vector<std::pair<int, double>>> lst(npair);
  for (int64_t t = 0; t < pr->T; ++t) {
    const int k = pr->kab[3 * t], a = pr->kab[3 * t + 1], b = pr->kab[3 * t + 2];
    if (a > b) continue;
    lst[size_t(a) * P - size_t(a) * (a - 1) / 2 + (b - a)].push_back({k, pr->g[t]});
  }
  pptr.assign(npair + 1, 0);
  pk.clear();
  pg.clear();
  for (int q = 0; q < npair; ++q) {
    for (const auto& e : lst[q]) {
      pk.push_back(e.first);
      pg.push_back(e.second);
    }
    pptr[q + 1] = int(pk.size());
  }
}

sg_status asm_prepare(sg_problem* pr, const Ell& A, AsmBlocks& B, cudaStream_t st) {
  if (B.tried || pr->asm_mode == 1) return SG_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  SG_CUDA(cudaStreamIsCapturing(st, &cs));
  if (cs != cudaStreamCaptureStatusNone) return SG_OK;
  B.tried = true;
  const int P = pr->P, S = A.S;
  const int npair = P * (P + 1) / 2;
  const size_t bytes = size_t(S) * npair * A.ldr * sizeof(double);
  if (pr->asm_mode == 0) {
    // automatic: only while the blocks take at most a quarter of free memory
    size_t fr = 0, tot = 0;
    SG_CUDA(cudaMemGetInfo(&fr, &tot));
    if (bytes > fr / 4) return SG_OK;
  }
  std::vector<int> pptr, pk;
  std::vector<double> pg;
  pair_lists(pr, pptr, pk, pg);
  DevBuf dptr, dk, dg, c;
  SG_TRY(c.alloc(bytes));
  SG_TRY(dptr.alloc(pptr.size() * 4));
  SG_TRY(dk.alloc(std::max<size_t>(1, pk.size()) * 4));
  SG_TRY(dg.alloc(std::max<size_t>(1, pg.size()) * 8));
  SG_CUDA(cudaMemcpy(dptr.ptr, pptr.data(), pptr.size() * 4, cudaMemcpyHostToDevice));
  if (!pk.empty()) {
    SG_CUDA(cudaMemcpy(dk.ptr, pk.data(), pk.size() * 4, cudaMemcpyHostToDevice));
    SG_CUDA(cudaMemcpy(dg.ptr, pg.data(), pg.size() * 8, cudaMemcpyHostToDevice));
  }
  k_asm_build<<<dim3(unsigned((A.ldr + 127) / 128), unsigned(npair)), 128, 0, st>>>(
      A.ldr, S, npair, dptr.as<int>(), dk.as<int>(), dg.as<double>(), A.v64.as<double>(), c.as<double>());
  note_launch();
  SG_CUDA(cudaGetLastError());
  SG_CUDA(cudaStreamSynchronize(st));
  B.npair = npair;
  B.c = std::move(c);
  return SG_OK;
}

sg_status apply_asm64(const sg_problem* pr, const Ell& A, const AsmBlocks& B, const double* X, int64_t ldx,
                      const double* F, int64_t ldf, double* Y, int64_t ldy, cudaStream_t st) {
  if (A.n == 0) return SG_OK;
  const dim3 block(32, 8);
  k_apply_asm64<<<unsigned((A.n + 31) / 32), block, 0, st>>>(A.n, A.ldr, A.S, pr->P, B.npair, A.col.as<int>(),
                                                              B.c.as<double>(), X, ldx, F, ldf, Y, ldy);
  note_launch();
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

template <typename T>
sg_status apply_any(sg_problem* pr, bool coarse, const T* X, int64_t ldx, const T* F, int64_t ldf, T* Y,
                    int64_t ldy, cudaStream_t st) {
  const Ell& A = coarse ? coarse_ell(pr) : pr->fine;
  if (sizeof(T) == 8) {
    const AsmBlocks& B = coarse ? coarse_asm(pr) : pr->asm_fine;
    if (B.c.ptr)
      return apply_asm64(pr, A, B, reinterpret_cast<const double*>(X), ldx, reinterpret_cast<const double*>(F),
                         ldf, reinterpret_cast<double*>(Y), ldy, st);
  }
  if (pr->apply_mode != 1 && jit_eligible(pr)) {
    // the edge-flux form of the fine FP32 operator when the family is configured for it
    const bool flux = !coarse && sizeof(T) == 4 && pr->flux_on;
    return jit_apply_launch(pr, (coarse ? 1 : 0) + (sizeof(T) == 8 ? 2 : 0), flux ? pr->flux : A, X, ldx, F, ldf, Y,
                            ldy, st);
  }
  return apply_ell<T>(A, coarse ? coarse_tri(pr) : pr->tri, pr->P, pr->K, X, ldx, F, ldf, Y, ldy, st);
}

template sg_status apply_any<double>(sg_problem*, bool, const double*, int64_t, const double*, int64_t, double*,
                                     int64_t, cudaStream_t);
template sg_status apply_any<float>(sg_problem*, bool, const float*, int64_t, const float*, int64_t, float*,
                                    int64_t, cudaStream_t);

template <typename T>
sg_status apply_op(sg_problem* pr, bool coarse, const T* X, int64_t ldx, const T* F, int64_t ldf, T* Y,
                   int64_t ldy, cudaStream_t st) {
  if (sizeof(T) == 8) SG_TRY(asm_prepare(pr, coarse ? coarse_ell(pr) : pr->fine, coarse ? coarse_asm(pr) : pr->asm_fine, st));
  size_t slot = 0;
  const bool on = pr->prof.on;
  if (on) SG_TRY(pr->prof.begin((coarse ? 2 : 0) + (sizeof(T) == 8 ? 1 : 0), st, slot));
  SG_TRY(apply_any<T>(pr, coarse, X, ldx, F, ldf, Y, ldy, st));
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
