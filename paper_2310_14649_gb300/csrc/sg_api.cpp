#include <algorithm>
// C ABI of libsg: argument checking and dispatch (declared in sg.h).
#include <atomic>
#include <cstring>
#include <new>

#include "sg_kernels.h"

namespace sg {
namespace {
thread_local std::string g_last_error;
}
void set_error(const std::string& msg) { g_last_error = msg; }
namespace {
std::atomic<int64_t> g_launches{0};
}
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace sg

using namespace sg;

extern "C" {

const char* sg_last_error(void) { return g_last_error.c_str(); }

sg_status sg_launch_count(int64_t* count) {
  SG_ARG(count, "sg_launch_count: NULL argument");
  *count = launch_count();
  return SG_OK;
}

sg_status sg_setup(const sg_mesh_desc* mesh, const sg_kl_desc* kl, int p_out, int q_in,
                   sg_problem** out) {
  SG_ARG(mesh && kl && out, "sg_setup: NULL argument");
  *out = nullptr;
  SG_ARG(mesh->N >= 2, "sg_setup: N must be >= 2");
  SG_ARG(kl->L >= 0 && kl->L <= 16, "sg_setup: L must be in [0, 16]");
  SG_ARG(p_out >= 0 && q_in >= 0, "sg_setup: orders must be >= 0");
  SG_ARG(kl->L == 0 || kl->user_modes || (kl->bx > 0 && kl->by > 0 && kl->sigma2 >= 0),
         "sg_setup: correlation lengths must be > 0 and sigma2 >= 0");
  sg_problem* pr = new (std::nothrow) sg_problem();
  if (!pr) {
    set_error("sg_setup: out of host memory");
    return SG_ERR_NOMEM;
  }
  pr->N = mesh->N;
  pr->L = kl->L;
  pr->p = p_out;
  pr->q = q_in;
  pr->sigma2 = kl->sigma2;
  pr->bx = kl->bx;
  pr->by = kl->by;
  pr->g0 = kl->g0;
  cudaGetDevice(&pr->device);
  sg_status st = build_host(pr, kl);
  if (st == SG_OK) st = assemble_fine(pr);
  if (st == SG_OK) st = build_triple_tables(pr, pr->tri, pr->fine.S);
  if (st != SG_OK) {
    sg_destroy(pr);
    return st;
  }
  pr->ld = round_up(pr->n, 64);
  *out = pr;
  return SG_OK;
}

sg_status sg_destroy(sg_problem* pr) {
  if (!pr) return SG_OK;
  solver_free(pr);
  cnn_free(pr);
  newton_free(pr);
  for (int w = 0; w < kJitFamilies; ++w) jit_free(pr, w);
  pr->mdot_partial.free_();
  pr->mdot_counter.free_();
  pr->fine.col.free_();
  pr->fine.v64.free_();
  pr->fine.v32.free_();
  pr->tri.tk.free_();
  pr->tri.tb.free_();
  pr->tri.g64.free_();
  pr->tri.g32.free_();
  pr->tri.off.free_();
  delete pr;
  return SG_OK;
}

sg_status sg_set_apply_kernel(sg_problem* pr, int mode) {
  SG_ARG(pr && mode >= 0 && mode <= 2, "sg_set_apply_kernel: mode must be 0, 1 or 2");
  if (mode == 2 && !jit_eligible(pr)) {
    set_error("sg_set_apply_kernel: the specialised kernel needs P <= 128 and T <= 40000");
    return SG_ERR_UNSUPPORTED;
  }
  drop_recorded(pr);
  pr->apply_mode = mode;
  if (mode != 1 && jit_eligible(pr)) return jit_apply_build(pr, 0);
  return SG_OK;
}

sg_status sg_apply_config(sg_problem* pr, int which, int rows, int groups, int igroups, int sgroups, int prefetch,
                          int min_blocks, int stages, int cgroups, int warps) {
  SG_ARG(pr && which >= 0 && which < kJitFamilies, "sg_apply_config: NULL handle or which not in [0, 3]");
  drop_recorded(pr);
  JitConfig c;
  c.rows = rows;
  c.groups = groups;
  c.igroups = igroups;
  c.sgroups = sgroups;
  c.prefetch = prefetch;
  c.min_blocks = min_blocks;
  c.stages = stages;
  c.cgroups = cgroups;
  c.warps = warps;
  return jit_configure(pr, which, c);
}

sg_status sg_apply_flux(sg_problem* pr, int mode, int* on) {
  SG_ARG(pr && mode >= -1 && mode <= 2, "sg_apply_flux: NULL handle or mode not in [-1, 2]");
  if (mode >= 0) pr->flux_allowed = mode != 0;
  if (mode == 0 || mode == 1) {
    SG_ARG(jit_eligible(pr) || mode == 0, "sg_apply_flux: the edge-flux form needs the specialised kernel");
    JitConfig c = pr->jit_cfg_set[0] ? pr->jit_cfg[0] : jit_default_config(pr, 0);
    if (mode == 1 && (c.rows != 1 || c.stages != 0 || c.cgroups != 1)) {
      c.rows = 1;
      c.stages = 0;
      c.cgroups = 1;
      c.prefetch = std::max(c.prefetch, 8);
    }
    c.flux = mode;
    if (pr->flux_on != c.flux || !pr->jit_cfg_set[0]) SG_TRY(jit_configure(pr, 0, c));
  }
  if (on) *on = pr->flux_on;
  return SG_OK;
}

sg_status sg_apply_autotune(sg_problem* pr, int which, int force, double* best_ms) {
  SG_ARG(pr && which >= 0 && which < kJitFamilies, "sg_apply_autotune: NULL handle or which not in [0, 3]");
  return jit_autotune(pr, which, force, best_ms);
}

sg_status sg_apply_info(const sg_problem* pr, int which, int* cfg10, double* compile_s) {
  SG_ARG(pr && which >= 0 && which < kJitFamilies, "sg_apply_info: NULL handle or which not in [0, 3]");
  const JitConfig c = pr->jit_cfg_set[which] ? pr->jit_cfg[which] : jit_default_config(pr, which);
  if (cfg10) {
    cfg10[0] = c.rows;
    cfg10[1] = c.groups;
    cfg10[2] = c.igroups;
    cfg10[3] = c.sgroups;
    cfg10[4] = c.prefetch;
    cfg10[5] = c.min_blocks;
    cfg10[6] = c.stages;
    cfg10[7] = c.cgroups;
    cfg10[8] = c.warps;
    cfg10[9] = kJitGeneratorVersion;
  }
  if (compile_s) *compile_s = pr->jit[which] ? pr->jit[which]->compile_s : 0.0;
  return SG_OK;
}

sg_status sg_get_sizes(const sg_problem* pr, int64_t* n, int* P, int* K, int64_t* nnzA, int64_t* T) {
  SG_ARG(pr, "sg_get_sizes: NULL handle");
  if (n) *n = pr->n;
  if (P) *P = pr->P;
  if (K) *K = pr->K;
  if (nnzA) *nnzA = pr->nnzA;
  if (T) *T = pr->T;
  return SG_OK;
}

sg_status sg_get_multi_indices(const sg_problem* pr, int32_t* out, int which) {
  SG_ARG(pr && out, "sg_get_multi_indices: NULL argument");
  SG_ARG(which == 0 || which == 1, "sg_get_multi_indices: which must be 0 or 1");
  const auto& v = which == 0 ? pr->mi_out : pr->mi_in;
  if (!v.empty()) std::memcpy(out, v.data(), v.size() * sizeof(int32_t));
  return SG_OK;
}

sg_status sg_get_triples(const sg_problem* pr, int32_t* kab, int64_t* num, double* g) {
  SG_ARG(pr && kab, "sg_get_triples: NULL argument");
  std::memcpy(kab, pr->kab.data(), pr->kab.size() * sizeof(int32_t));
  if (num) std::memcpy(num, pr->num.data(), pr->num.size() * sizeof(int64_t));
  if (g) std::memcpy(g, pr->g.data(), pr->g.size() * sizeof(double));
  return SG_OK;
}

sg_status sg_get_csr(const sg_problem* pr, int32_t* rowptr, int32_t* colidx) {
  SG_ARG(pr && rowptr && colidx, "sg_get_csr: NULL argument");
  std::memcpy(rowptr, pr->rowptr.data(), pr->rowptr.size() * sizeof(int32_t));
  std::memcpy(colidx, pr->colidx.data(), pr->colidx.size() * sizeof(int32_t));
  return SG_OK;
}

sg_status sg_get_values(const sg_problem* pr, double* vals) {
  SG_ARG(pr && vals, "sg_get_values: NULL argument");
  const Ell& A = pr->fine;
  const size_t cnt = size_t(pr->K) * A.S * A.ldr;
  std::vector<double> v(cnt);
  std::vector<int32_t> col(size_t(A.S) * A.ldr);
  SG_CUDA(cudaMemcpy(v.data(), A.v64.ptr, cnt * sizeof(double), cudaMemcpyDeviceToHost));
  SG_CUDA(cudaMemcpy(col.data(), A.col.ptr, col.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
  for (int64_t r = 0; r < pr->n; ++r)
    for (int32_t t = pr->rowptr[r]; t < pr->rowptr[r + 1]; ++t) {
      int slot = -1;
      for (int s = 0; s < A.S; ++s)
        if (col[s * A.ldr + r] == pr->colidx[t] && (pr->colidx[t] != r || s == 2)) slot = s;
      if (slot < 0) {
        set_error("sg_get_values: pattern entry without a slot");
        return SG_ERR_ARG;
      }
      for (int k = 0; k < pr->K; ++k) vals[size_t(k) * pr->nnzA + t] = v[(size_t(k) * A.S + slot) * A.ldr + r];
    }
  return SG_OK;
}

sg_status sg_get_rhs(const sg_problem* pr, double* F, int64_t ld, void* stream) {
  SG_ARG(pr && F, "sg_get_rhs: NULL argument");
  SG_ARG(ld >= pr->n, "sg_get_rhs: ld < n");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SG_CUDA(cudaMemsetAsync(F, 0, sizeof(double) * size_t(ld) * pr->P, st));
  SG_CUDA(cudaMemcpyAsync(F, pr->b.data(), sizeof(double) * pr->n, cudaMemcpyHostToDevice, st));
  SG_CUDA(cudaStreamSynchronize(st));
  return SG_OK;
}

static bool overlaps(const void* a, size_t abytes, const void* b, size_t bbytes) {
  const char* x = static_cast<const char*>(a);
  const char* y = static_cast<const char*>(b);
  return x < y + bbytes && y < x + abytes;
}

sg_status sg_apply(sg_problem* pr, sg_dtype dtype, const void* X, int64_t ldx, void* Y, int64_t ldy,
                   void* stream) {
  SG_ARG(pr && X && Y, "sg_apply: NULL argument");
  SG_ARG(ldx >= pr->n && ldy >= pr->n, "sg_apply: leading dimension < n");
  SG_ARG(dtype == SG_F64 || dtype == SG_F32, "sg_apply: bad dtype");
  const size_t es = dtype == SG_F64 ? 8 : 4;
  SG_ARG(!overlaps(X, es * size_t(ldx) * pr->P, Y, es * size_t(ldy) * pr->P),
         "sg_apply: X and Y overlap");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (dtype == SG_F64)
    return apply_op<double>(pr, false, static_cast<const double*>(X), ldx, nullptr, 0, static_cast<double*>(Y),
                            ldy, st);
  return apply_op<float>(pr, false, static_cast<const float*>(X), ldx, nullptr, 0, static_cast<float*>(Y), ldy,
                         st);
}

sg_status sg_residual(sg_problem* pr, sg_dtype dtype, const void* F, int64_t ldf, const void* X,
                      int64_t ldx, void* R, int64_t ldr, void* stream) {
  SG_ARG(pr && F && X && R, "sg_residual: NULL argument");
  SG_ARG(ldx >= pr->n && ldr >= pr->n && ldf >= pr->n, "sg_residual: leading dimension < n");
  SG_ARG(dtype == SG_F64 || dtype == SG_F32, "sg_residual: bad dtype");
  const size_t es = dtype == SG_F64 ? 8 : 4;
  SG_ARG(!overlaps(X, es * size_t(ldx) * pr->P, R, es * size_t(ldr) * pr->P),
         "sg_residual: X and R overlap");
  SG_ARG(F == R ? ldf == ldr : !overlaps(F, es * size_t(ldf) * pr->P, R, es * size_t(ldr) * pr->P),
         "sg_residual: F and R overlap with different layouts");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (dtype == SG_F64)
    return apply_op<double>(pr, false, static_cast<const double*>(X), ldx, static_cast<const double*>(F), ldf,
                            static_cast<double*>(R), ldr, st);
  return apply_op<float>(pr, false, static_cast<const float*>(X), ldx, static_cast<const float*>(F), ldf,
                         static_cast<float*>(R), ldr, st);
}

sg_status sg_residual_refine(sg_problem* pr, const double* F, int64_t ldf, const double* X, int64_t ldx, double* R,
                             int64_t ldr, void* stream) {
  SG_ARG(pr && F && X && R, "sg_residual_refine: NULL argument");
  SG_ARG(ldx >= pr->n && ldr >= pr->n && ldf >= pr->n, "sg_residual_refine: leading dimension < n");
  SG_ARG(!overlaps(X, 8 * size_t(ldx) * pr->P, R, 8 * size_t(ldr) * pr->P), "sg_residual_refine: X and R overlap");
  SG_ARG(F == R ? ldf == ldr : !overlaps(F, 8 * size_t(ldf) * pr->P, R, 8 * size_t(ldr) * pr->P),
         "sg_residual_refine: F and R overlap with different layouts");
  return refine_residual(pr, F, ldf, X, ldx, R, ldr, static_cast<cudaStream_t>(stream));
}

sg_status sg_mdot(sg_problem* pr, sg_dtype dtype, const void* V, int64_t stride, int nv, const void* w, int64_t len,
                  double* out, void* stream) {
  SG_ARG(pr && V && w && out, "sg_mdot: NULL argument");
  SG_ARG(dtype == SG_F64 || dtype == SG_F32, "sg_mdot: bad dtype");
  SG_ARG(nv >= 1 && nv <= kMdotMaxVectors, "sg_mdot: nv must be in [1, 32]");
  SG_ARG(len >= 0 && (nv == 1 || stride >= len), "sg_mdot: len < 0 or stride < len");
  if (!pr->mdot_partial.ptr) {
    SG_TRY(pr->mdot_partial.alloc(size_t(kMdotBlocks) * kMdotMaxVectors * sizeof(double)));
    SG_TRY(pr->mdot_counter.alloc(256));
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (dtype == SG_F64)
    return vec_mdot<double>(static_cast<const double*>(V), stride, nv, static_cast<const double*>(w), len, out,
                            dp<double>(pr->mdot_partial), dp<unsigned>(pr->mdot_counter), st);
  return vec_mdot<float>(static_cast<const float*>(V), stride, nv, static_cast<const float*>(w), len, out,
                         dp<double>(pr->mdot_partial), dp<unsigned>(pr->mdot_counter), st);
}

}  // extern "C"
