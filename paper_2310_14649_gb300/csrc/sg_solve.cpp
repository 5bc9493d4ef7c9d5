// Solver orchestration: the two-level preconditioner of Sec. 3 (Eq. RAS_2L),
// flexible GMRES on the fine Galerkin system, GMRES + AMG on the coarse
// system (the 2GV3 variant), and mixed-precision iterative refinement
// (FP32 inner FGMRES inside an FP64 residual loop).
#include <chrono>
#include <cmath>
#include <cstring>
#include <algorithm>
#include <memory>

#include "sg_ctx.h"

namespace sg {

const Ell& coarse_ell(const sg_problem* pr) { return pr->solver->pc.co.ell; }
const TripleTables& coarse_tri(const sg_problem* pr) { return pr->solver->pc.co.tri; }
AsmBlocks& coarse_asm(sg_problem* pr) { return pr->solver->pc.co.asm_c; }

// Recorded graphs (the coarse-solve graphs of the solver contexts) hold the
// kernels and buffers of the applies they captured: a change of apply
// kernel drops the contexts, so they are rebuilt, and recorded batches of
// this problem refuse to run (their contexts no longer match).
void drop_recorded(sg_problem* pr) {
  if (!pr->solver) return;
  cudaDeviceSynchronize();
  pr->solver->c64.reset();
  pr->solver->c32.reset();
  ++pr->solver->ctx_gen;  // a new context may reuse a freed one's address
}


void solver_free(sg_problem* pr) {
  delete pr->solver;
  pr->solver = nullptr;
}

// d = omega * G~^{-1} in FP64 and FP32
static sg_status upload_scaled(const std::vector<double>& ginv, double omega, DevBuf& d64, DevBuf& d32) {
  std::vector<double> m64(ginv.size());
  std::vector<float> m32(ginv.size());
  for (size_t e = 0; e < m64.size(); ++e) {
    m64[e] = omega * ginv[e];
    m32[e] = float(m64[e]);
  }
  if (!d64.ptr) SG_TRY(d64.alloc(m64.size() * 8));
  if (!d32.ptr) SG_TRY(d32.alloc(m32.size() * 4));
  SG_CUDA(cudaMemcpy(d64.ptr, m64.data(), m64.size() * 8, cudaMemcpyHostToDevice));
  SG_CUDA(cudaMemcpy(d32.ptr, m32.data(), m32.size() * 4, cudaMemcpyHostToDevice));
  return SG_OK;
}

// upload omega * G~^{-1} (smoother) and G~^{-1} (coarse preconditioner)
static sg_status upload_gtinv(sg_problem*, Precond& pc, const std::vector<double>& ginv) {
  pc.ginv = ginv;
  if (!pc.gkron64.ptr) SG_TRY(upload_scaled(ginv, 1.0, pc.gkron64, pc.gkron32));
  return upload_scaled(ginv, pc.omega, pc.gtinv64, pc.gtinv32);
}

// Kronecker stochastic factor G~ = sum_k w_k G_k, w_k = <A_k, A_0>_F / <A_0, A_0>_F,
// and its inverse (SPD: Cholesky on the host).
static sg_status kronecker_factor(sg_problem* pr, Precond& pc, std::vector<double>& ginv) {
  std::vector<double> fw;
  SG_TRY(frobenius_weights(pr, fw));
  const int P = pr->P;
  pc.gt.assign(size_t(P) * P, 0.0);
  for (int64_t t = 0; t < pr->T; ++t) {
    int k = pr->kab[3 * t], a = pr->kab[3 * t + 1], b = pr->kab[3 * t + 2];
    pc.gt[size_t(a) * P + b] += fw[k] / fw[0] * pr->g[t];
  }
  // Gauss-Jordan inverse with partial pivoting
  std::vector<double> A = pc.gt;
  ginv.assign(size_t(P) * P, 0.0);
  for (int i = 0; i < P; ++i) ginv[size_t(i) * P + i] = 1.0;
  for (int c = 0; c < P; ++c) {
    int piv = c;
    for (int r = c + 1; r < P; ++r)
      if (std::fabs(A[size_t(r) * P + c]) > std::fabs(A[size_t(piv) * P + c])) piv = r;
    if (A[size_t(piv) * P + c] == 0.0) {
      set_error("Kronecker factor is singular");
      return SG_ERR_BREAKDOWN;
    }
    for (int k = 0; k < P; ++k) {
      std::swap(A[size_t(c) * P + k], A[size_t(piv) * P + k]);
      std::swap(ginv[size_t(c) * P + k], ginv[size_t(piv) * P + k]);
    }
    const double d = A[size_t(c) * P + c];
    for (int k = 0; k < P; ++k) {
      A[size_t(c) * P + k] /= d;
      ginv[size_t(c) * P + k] /= d;
    }
    for (int r = 0; r < P; ++r) {
      if (r == c) continue;
      const double f = A[size_t(r) * P + c];
      if (f == 0.0) continue;
      for (int k = 0; k < P; ++k) {
        A[size_t(r) * P + k] -= f * A[size_t(c) * P + k];
        ginv[size_t(r) * P + k] -= f * ginv[size_t(c) * P + k];
      }
    }
  }
  return SG_OK;
}

// rho(S A) by 20 power iterations (FP32) from the seed-free start
// X[a][r] = 1 + (r + a) mod 3, with the smoother currently selected
static sg_status estimate_rho(sg_problem* pr, cudaStream_t st, double& rho) {
  SolverCtx<float>* c = nullptr;
  SG_TRY(get_ctx<float>(pr, c));
  const int P = pr->P;
  const int64_t ld = pr->ld, len = c->len;
  std::vector<float> x0(len, 0.0f);
  for (int a = 0; a < P; ++a)
    for (int64_t r = 0; r < pr->n; ++r) x0[size_t(a) * ld + r] = float(1 + (r + a) % 3);
  float* X = dp<float>(c->fine.tmp);
  float* Y = dp<float>(c->fine.tmp2);
  float* AX = dp<float>(c->fine.w);
  SG_CUDA(cudaMemcpyAsync(X, x0.data(), len * 4, cudaMemcpyHostToDevice, st));
  double* nrm = c->fine.s.scal + 6;
  SG_TRY(vec_norm2<float>(X, len, nrm, dp<double>(c->fine.partial), dp<unsigned>(c->fine.counter), st));
  SG_TRY(vec_scale_by<float>(X, X, len, nrm, true, st));
  for (int it = 0; it < 20; ++it) {
    SG_TRY(c->apply_fine(X, AX, nullptr, st));
    SG_TRY(c->smooth(AX, Y, st));
    SG_TRY(vec_norm2<float>(Y, len, nrm, dp<double>(c->fine.partial), dp<unsigned>(c->fine.counter), st));
    SG_TRY(vec_scale_by<float>(Y, X, len, nrm, true, st));
  }
  SG_CUDA(cudaMemcpyAsync(c->fine.host + 6, nrm, 8, cudaMemcpyDeviceToHost, st));
  SG_CUDA(cudaStreamSynchronize(st));
  rho = std::sqrt(c->fine.host[6]);
  if (!(rho > 0.0) || !std::isfinite(rho)) {
    set_error("omega estimate failed");
    return SG_ERR_BREAKDOWN;
  }
  return SG_OK;
}

// omega = 1 / rho(S A) for the RAS smoother
static sg_status estimate_omega(sg_problem* pr, SolverState& S, cudaStream_t st) {
  double rho = 0.0;
  SG_TRY(estimate_rho(pr, st, rho));
  S.pc.omega = 1.0 / rho;
  return SG_OK;
}

Precond& precond_of(sg_problem* pr) { return pr->solver->pc; }

// ras_kernel 3: build the explicit local inverses when they are available
// and keep them when one FP32 application (median of 5, CUDA events, after
// a warm-up) is faster than the line kernel's; otherwise the line kernel.
sg_status ras_kernel_choose(sg_problem* pr, Precond& pc, cudaStream_t st) {
  pc.ras_kernel = 0;
  if (!ras_inverse_supported(pr->P)) return SG_OK;
  const sg_status b = ras_inverse_build(pr, pc, st);
  if (b == SG_ERR_UNSUPPORTED) return SG_OK;
  SG_TRY(b);
  const int64_t len = int64_t(pr->P) * pr->ld;
  DevBuf R, Z;
  SG_TRY(R.alloc(len * 4));
  SG_TRY(Z.alloc(len * 4));
  std::vector<float> h(len);
  for (int64_t e = 0; e < len; ++e) h[e] = float(1 + (e * 7) % 13) * 0.125f;
  SG_CUDA(cudaMemcpy(R.ptr, h.data(), len * 4, cudaMemcpyHostToDevice));
  cudaEvent_t e0, e1;
  SG_CUDA(cudaEventCreate(&e0));
  SG_CUDA(cudaEventCreate(&e1));
  double t[2] = {0, 0};
  for (int k : {0, 2}) {
    pc.ras_kernel = k;
    std::vector<float> ts;
    for (int rep = 0; rep < 6; ++rep) {
      SG_CUDA(cudaEventRecord(e0, st));
      SG_TRY(ras_apply<float>(pc, pr->n, pr->P, dp<float>(R), pr->ld, dp<float>(Z), st, true));
      SG_CUDA(cudaEventRecord(e1, st));
      SG_CUDA(cudaEventSynchronize(e1));
      float ms = 0;
      SG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (rep) ts.push_back(ms);
    }
    std::sort(ts.begin(), ts.end());
    t[k == 2] = ts[ts.size() / 2];
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  SG_TRY(ras_inverse_check(pc, st));
  pc.ras_kernel = t[1] < t[0] ? 2 : 0;
  if (pc.ras_kernel == 0) {
    pc.ras.inv_free();
  }
  return SG_OK;
}

// Selects the learned smoother for later solves with damping omega_cnn
// (= 1 / rho(S_cnn A) by the same power iteration when omega <= 0).
sg_status learned_smoother_enable(sg_problem* pr, double omega, cudaStream_t st) {
  Precond& pc = pr->solver->pc;
  pc.omega_cnn = 1.0;
  SG_TRY(upload_scaled(pc.ginv, 1.0, pc.gtcnn64, pc.gtcnn32));
  if (omega <= 0) {
    const bool prev = pc.use_cnn;
    pc.use_cnn = true;
    double rho = 0.0;
    sg_status s = estimate_rho(pr, st, rho);
    pc.use_cnn = prev;
    SG_TRY(s);
    omega = 1.0 / rho;
  }
  pc.omega_cnn = omega;
  SG_TRY(upload_scaled(pc.ginv, omega, pc.gtcnn64, pc.gtcnn32));
  pc.smoother = 1;
  return SG_OK;
}

}  // namespace sg

using namespace sg;

template <typename T>
static sg_status precond_apply_t(sg_problem* pr, int which, const T* Rin, int64_t ldr, T* Zout, int64_t ldz,
                                 cudaStream_t st) {
  SolverCtx<T>* c = nullptr;
  SG_TRY(get_ctx<T>(pr, c));
  SolverState& S = *pr->solver;
  const int P = pr->P;
  const bool coarse_in = which == 3 || which == 4 || which == 6;
  const bool coarse_out = which == 3 || which == 4 || which == 5;
  const int64_t nin = coarse_in ? S.pc.co.nc : pr->n, ldin = coarse_in ? c->ldc : c->ld;
  const int64_t nout = coarse_out ? S.pc.co.nc : pr->n, ldout = coarse_out ? c->ldc : c->ld;
  SG_ARG(ldr >= nin && ldz >= nout, "sg_precond_apply: leading dimension too small");
  const bool learned = which == 8 || which == 9;
  if (learned) {
    SG_ARG(pr->cnn && pr->cnn->trained, "sg_precond_apply: the learned smoother has no weights");
    SG_ARG(which == 9 || S.pc.gtcnn64.ptr, "sg_precond_apply: learned smoother not enabled");
  }
  const bool prev_cnn = S.pc.use_cnn;
  S.pc.use_cnn = learned || (S.pc.smoother == 1 && pr->cnn && pr->cnn->trained);
  struct Restore {
    Precond& pc;
    bool v;
    ~Restore() { pc.use_cnn = v; }
  } restore{S.pc, prev_cnn};
  T* in = coarse_in ? dp<T>(c->coarse.tmp) : dp<T>(c->fine.tmp);
  T* out = coarse_out ? dp<T>(c->coarse.tmp2) : dp<T>(c->fine.tmp2);
  SG_CUDA(cudaMemsetAsync(in, 0, size_t(P) * ldin * sizeof(T), st));
  SG_CUDA(cudaMemsetAsync(out, 0, size_t(P) * ldout * sizeof(T), st));
  SG_CUDA(cudaMemcpy2DAsync(in, ldin * sizeof(T), Rin, ldr * sizeof(T), nin * sizeof(T), P,
                            cudaMemcpyDeviceToDevice, st));
  switch (which) {
    case 0: SG_TRY(c->twolevel(in, out, st)); break;
    case 1: SG_TRY(c->smooth(in, out, st)); break;
    case 2: SG_TRY(c->coarse_correction(in, out, false, st)); break;
    case 3: SG_TRY(c->amg(in, out, st)); break;
    case 4: SG_TRY(c->apply_coarse(in, out, st)); break;
    case 5: SG_TRY(spmm<T>(S.pc.co.R, in, c->ld, nullptr, 0, out, c->ldc, P, 0, st)); break;
    case 6: SG_TRY(spmm<T>(S.pc.co.RT, in, c->ldc, nullptr, 0, out, c->ld, P, 0, st)); break;
    case 7: SG_TRY(ras_apply<T>(S.pc, pr->n, P, in, c->ld, out, st, false)); break;
    case 8: SG_TRY(c->smooth(in, out, st)); break;
    case 9: SG_TRY(cnn_smooth<T>(pr, S.pc, in, c->ld, out, false, st)); break;
    default: set_error("sg_precond_apply: unknown operator"); return SG_ERR_ARG;
  }
  SG_CUDA(cudaMemcpy2DAsync(Zout, ldz * sizeof(T), out, ldout * sizeof(T), nout * sizeof(T), P,
                            cudaMemcpyDeviceToDevice, st));
  return SG_OK;
}


extern "C" {

sg_status sg_precond_setup(sg_problem* pr, const sg_precond_opts* o, void* stream) {
  SG_ARG(pr && o, "sg_precond_setup: NULL argument");
  SG_ARG(pr->N % 2 == 0 && pr->N >= 4, "sg_precond_setup: the 2h coarse grid needs an even N >= 4");
  SG_ARG(o->sx >= 1 && o->sy >= 1 && o->sx <= pr->N - 1 && o->sy <= pr->N - 1,
         "sg_precond_setup: subdomain counts must be in [1, N-1]");
  SG_ARG(o->overlap >= 0 && o->overlap <= 8, "sg_precond_setup: overlap must be in [0, 8]");
  SG_ARG(o->amg_kernel == 0 || o->amg_kernel == 1, "sg_precond_setup: amg_kernel must be 0 or 1");
  SG_ARG(o->ras_kernel >= 0 && o->ras_kernel <= 3, "sg_precond_setup: ras_kernel must be 0, 1, 2 or 3");
  SG_ARG(o->ras_kernel != 2 || ras_inverse_supported(pr->P),
         "sg_precond_setup: ras_kernel 2 (explicit local inverses) needs P <= 96");
  SG_ARG(o->ras_stages == 0 || (o->ras_stages >= 2 && o->ras_stages <= 8),
         "sg_precond_setup: ras_stages must be 0 (automatic) or in [2, 8]");
  SG_ARG(o->inner_orth_passes >= 0 && o->inner_orth_passes <= 2,
         "sg_precond_setup: inner_orth_passes must be 0 (default), 1 or 2");
  SG_ARG(o->smoother == 0 || o->smoother == 1, "sg_precond_setup: smoother must be 0 (RAS) or 1 (learned)");
  SG_ARG(o->smoother == 0 || (pr->cnn && pr->cnn->trained),
         "sg_precond_setup: the learned smoother needs trained or loaded weights");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  solver_free(pr);
  pr->solver = new SolverState();
  SolverState& S = *pr->solver;
  Precond& pc = S.pc;
  pc.sx = o->sx;
  pc.sy = o->sy;
  pc.overlap = o->overlap;
  pc.inner_rtol = o->inner_rtol > 0 ? o->inner_rtol : 1e-5;
  pc.inner_max = o->inner_max > 0 ? o->inner_max : 100;
  pc.inner_restart = 30;
  pc.device_loops = o->host_loops == 0;
  pc.ras_modes = o->ras_modes > 0 ? o->ras_modes : 0;
  pc.ras_stages = o->ras_stages;
  pc.ras_kernel = o->ras_kernel;
  pc.inner_passes = o->inner_orth_passes > 0 ? o->inner_orth_passes : 1;
  SG_TRY(kernel_attrs_init());
  sg_status s = precond_setup_host(pr, pc);
  pc.amg.fused = o->amg_kernel == 0;
  pc.wait_limit = pr->wait_limit;
  if (s == SG_OK && pc.ras_kernel == 2) s = ras_inverse_build(pr, pc, st);
  std::vector<double> ginv;
  if (s == SG_OK) s = kronecker_factor(pr, pc, ginv);
  pc.omega = 1.0;
  if (s == SG_OK) s = upload_gtinv(pr, pc, ginv);
  // the choice times the full local step (with the Kronecker factor), so
  // it runs once that factor is on the device
  if (s == SG_OK && pc.ras_kernel == 3) s = ras_kernel_choose(pr, pc, st);
  if (s == SG_OK && o->omega <= 0) s = estimate_omega(pr, S, st);
  if (s == SG_OK && o->omega > 0) pc.omega = o->omega;
  if (s == SG_OK) s = upload_gtinv(pr, pc, ginv);
  if (s == SG_OK && o->smoother == 1) s = learned_smoother_enable(pr, 0.0, st);
  if (s != SG_OK) {
    solver_free(pr);
    return s;
  }
  pc.ready = true;
  return SG_OK;
}

sg_status sg_set_apply_fp64(sg_problem* pr, int mode) {
  SG_ARG(pr && mode >= 0 && mode <= 2, "sg_set_apply_fp64: mode must be 0, 1 or 2");
  drop_recorded(pr);
  pr->asm_mode = mode;
  pr->asm_fine = AsmBlocks();
  if (pr->solver) pr->solver->pc.co.asm_c = AsmBlocks();
  if (mode == 2) {
    SG_TRY(asm_prepare(pr, pr->fine, pr->asm_fine, nullptr));
    if (pr->solver && pr->solver->pc.ready) SG_TRY(asm_prepare(pr, coarse_ell(pr), coarse_asm(pr), nullptr));
  }
  return SG_OK;
}

sg_status sg_set_refine_residual(sg_problem* pr, int mode) {
  SG_ARG(pr && mode >= 0 && mode <= 2, "sg_set_refine_residual: mode must be 0, 1 or 2");
  drop_recorded(pr);
  pr->res_mode = mode;
  pr->fdf = FluxDf();
  if (mode == 2) SG_TRY(resid_prepare(pr, nullptr));
  return SG_OK;
}

sg_status sg_refine_residual_info(const sg_problem* pr, int* built, int64_t* bytes) {
  SG_ARG(pr, "sg_refine_residual_info: NULL handle");
  const bool b = pr->fdf.b.ptr != nullptr && pr->res_mode != 1;
  if (built) *built = b;
  if (bytes) *bytes = b ? int64_t(pr->fdf.b.bytes + pr->fdf.xs.bytes) : 0;
  return SG_OK;
}

sg_status sg_apply_fp64_info(const sg_problem* pr, int* fine, int* coarse, int64_t* bytes) {
  SG_ARG(pr, "sg_apply_fp64_info: NULL handle");
  const bool f = pr->asm_fine.c.ptr != nullptr;
  const bool c = pr->solver && pr->solver->pc.co.asm_c.c.ptr != nullptr;
  if (fine) *fine = f;
  if (coarse) *coarse = c;
  if (bytes) *bytes = int64_t((f ? pr->asm_fine.c.bytes : 0) + (c ? pr->solver->pc.co.asm_c.c.bytes : 0));
  return SG_OK;
}

sg_status sg_profile(sg_problem* pr, int enable) {
  SG_ARG(pr, "sg_profile: NULL handle");
  pr->prof.on = enable != 0;
  pr->prof.reset();
  return SG_OK;
}

sg_status sg_profile_read(sg_problem* pr, int kind, int64_t* launches, double* ms) {
  SG_ARG(pr && kind >= 0 && kind < kProfKinds, "sg_profile_read: bad argument");
  return pr->prof.read(kind, launches, ms);
}

sg_status sg_precond_info(const sg_problem* pr, double* omega, int* amg_levels, int64_t* nc, int* inner_its_last) {
  SG_ARG(pr && pr->solver && pr->solver->pc.ready, "sg_precond_info: no preconditioner set up");
  const Precond& pc = pr->solver->pc;
  if (omega) *omega = pc.omega;
  if (amg_levels) *amg_levels = int(pc.amg.size());
  if (nc) *nc = pc.co.nc;
  if (inner_its_last) {
    *inner_its_last = pc.inner_its_last;
    if (pc.device_loops && pc.last_coarse_dtype >= 0) {
      // iterations of the last device-driven coarse solve (device counter)
      const int* iv = pc.last_coarse_dtype == 0 ? pr->solver->c64->dg.iv : pr->solver->c32->dg.iv;
      SG_CUDA(cudaDeviceSynchronize());
      SG_CUDA(cudaMemcpy(inner_its_last, iv + 1, sizeof(int), cudaMemcpyDeviceToHost));
    }
  }
  return SG_OK;
}

sg_status sg_precond_stats(const sg_problem* pr, double* ras_flops, int* ras_boxes, int* ras_wmax, int* ras_kernel) {
  SG_ARG(pr && pr->solver && pr->solver->pc.ready, "sg_precond_stats: no preconditioner set up");
  const RasData& R = pr->solver->pc.ras;
  if (ras_flops) *ras_flops = R.flops_per_mode * pr->P;
  if (ras_boxes) *ras_boxes = R.nbox;
  if (ras_wmax) *ras_wmax = R.wmax;
  if (ras_kernel) *ras_kernel = pr->solver->pc.ras_kernel;
  return SG_OK;
}

sg_status sg_get_partition(const sg_problem* pr, int sub, int32_t* idx, int64_t* count, int32_t* owned) {
  SG_ARG(pr && pr->solver && pr->solver->pc.ready && count, "sg_get_partition: no preconditioner set up");
  const RasData& R = pr->solver->pc.ras;
  SG_ARG(sub >= 0 && sub < R.nbox, "sg_get_partition: subdomain out of range");
  *count = int64_t(R.idx[sub].size());
  if (idx) std::memcpy(idx, R.idx[sub].data(), R.idx[sub].size() * 4);
  if (owned) std::memcpy(owned, R.owned[sub].data(), R.owned[sub].size() * 4);
  return SG_OK;
}

sg_status sg_get_coarse_csr(const sg_problem* pr, int64_t* nc, int64_t* nnz, int32_t* rowptr, int32_t* colidx) {
  SG_ARG(pr && pr->solver && pr->solver->pc.ready, "sg_get_coarse_csr: no preconditioner set up");
  const CoarseData& C = pr->solver->pc.co;
  if (nc) *nc = C.nc;
  if (nnz) *nnz = int64_t(C.colidx.size());
  if (rowptr) std::memcpy(rowptr, C.rowptr.data(), C.rowptr.size() * 4);
  if (colidx) std::memcpy(colidx, C.colidx.data(), C.colidx.size() * 4);
  return SG_OK;
}

sg_status sg_get_amg_level(const sg_problem* pr, int level, int64_t* n, int32_t* agg) {
  SG_ARG(pr && pr->solver && pr->solver->pc.ready, "sg_get_amg_level: no preconditioner set up");
  const auto& L = pr->solver->pc.amg;
  SG_ARG(level >= 0 && level < int(L.size()), "sg_get_amg_level: level out of range");
  if (n) *n = L[level].n;
  if (agg && !L[level].agg.empty()) std::memcpy(agg, L[level].agg.data(), L[level].agg.size() * 4);
  return SG_OK;
}

sg_status sg_precond_apply(sg_problem* pr, sg_dtype dtype, int which, const void* R, int64_t ldr, void* Z,
                           int64_t ldz, void* stream) {
  SG_ARG(pr && R && Z, "sg_precond_apply: NULL argument");
  SG_ARG(pr->solver && pr->solver->pc.ready, "sg_precond_apply: call sg_precond_setup first");
  SG_ARG(dtype == SG_F64 || dtype == SG_F32, "sg_precond_apply: bad dtype");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const sg_status s =
      dtype == SG_F64
          ? precond_apply_t<double>(pr, which, static_cast<const double*>(R), ldr, static_cast<double*>(Z), ldz, st)
          : precond_apply_t<float>(pr, which, static_cast<const float*>(R), ldr, static_cast<float*>(Z), ldz, st);
  if (s < 0) pr->solver->dirty = true;
  if (s == SG_OK && pr->solver->pc.ras_kernel == 2) return ras_inverse_check(pr->solver->pc, st);
  return s;
}

static sg_status solve_impl(sg_problem* pr, const double* F, int64_t ldf, double* X, int64_t ldx,
                            const sg_solve_opts* o, sg_solve_info* info, void* stream);

sg_status sg_solve(sg_problem* pr, const double* F, int64_t ldf, double* X, int64_t ldx, const sg_solve_opts* o,
                   sg_solve_info* info, void* stream) {
  const sg_status s = solve_impl(pr, F, ldf, X, ldx, o, info, stream);
  if (s < 0 && pr && pr->solver) pr->solver->dirty = true;
  return s;
}

}  // extern "C"

static sg_status solve_impl(sg_problem* pr, const double* F, int64_t ldf, double* X, int64_t ldx,
                            const sg_solve_opts* o, sg_solve_info* info, void* stream) {
  SG_ARG(pr && X && o, "sg_solve: NULL argument");
  SG_ARG(pr->solver && pr->solver->pc.ready, "sg_solve: call sg_precond_setup first");
  SG_ARG(ldx >= pr->n && (!F || ldf >= pr->n), "sg_solve: leading dimension < n");
  SG_ARG(o->rtol > 0 && o->max_it > 0, "sg_solve: rtol and max_it must be > 0");
  SG_ARG(o->mode == 0 || o->mode == 1, "sg_solve: mode must be 0 (FP64) or 1 (FP32 in FP64 refinement)");
  SG_ARG(o->orth_passes >= 0 && o->orth_passes <= 2, "sg_solve: orth_passes must be 0 (default), 1 or 2");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SolverState& S = *pr->solver;
  S.restart = o->restart > 0 ? std::min(o->restart, 31) : 30;
  const int P = pr->P;
  const int64_t ld = pr->ld, len = int64_t(P) * ld;
  auto t0 = std::chrono::steady_clock::now();
  if (!S.host) SG_CUDA(cudaHostAlloc(&S.host, 16 * sizeof(double), cudaHostAllocDefault));
  if (!S.x64.ptr) SG_TRY(S.x64.alloc(len * 8));
  if (!S.r64.ptr) SG_TRY(S.r64.alloc(len * 8));
  if (!S.io.ptr) SG_TRY(S.io.alloc(len * 8));
  if (!S.scal.ptr) SG_TRY(S.scal.alloc(64 * 8));
  double* x64 = dp<double>(S.x64);
  double* F64 = dp<double>(S.io);
  // internal copies with the library's leading dimension (padding zero)
  SG_CUDA(cudaMemsetAsync(F64, 0, len * 8, st));
  SG_CUDA(cudaMemsetAsync(x64, 0, len * 8, st));
  if (F) {
    SG_CUDA(cudaMemcpy2DAsync(F64, ld * 8, F, ldf * 8, pr->n * 8, P, cudaMemcpyDeviceToDevice, st));
  } else {
    SG_CUDA(cudaMemcpyAsync(F64, pr->b.data(), pr->n * 8, cudaMemcpyHostToDevice, st));
  }
  SG_CUDA(cudaMemcpy2DAsync(x64, ld * 8, X, ldx * 8, pr->n * 8, P, cudaMemcpyDeviceToDevice, st));
  SolverCtx<double>* c64 = nullptr;
  SG_TRY(get_ctx<double>(pr, c64));
  c64->fine.passes = fine_orth_passes(*o);
  double* scal = dp<double>(S.scal);
  SG_TRY(vec_norm2<double>(F64, len, scal, dp<double>(c64->fine.partial), dp<unsigned>(c64->fine.counter), st));
  SG_CUDA(cudaMemcpyAsync(S.host, scal, 8, cudaMemcpyDeviceToHost, st));
  SG_CUDA(cudaStreamSynchronize(st));
  const double nF = std::sqrt(S.host[0]);
  sg_solve_info inf{};
  std::vector<double> hist;
  if (S.dirty) {
    SG_TRY(c64->scrub(st));
    if (S.c32) SG_TRY(S.c32->scrub(st));
    S.dirty = false;
  }
  S.pc.use_cnn = S.pc.smoother == 1 && pr->cnn && pr->cnn->trained;
  const bool stall_test = S.pc.use_cnn && !o->no_fallback;
  struct ClearCnn {
    Precond& pc;
    ~ClearCnn() { pc.use_cnn = false; }
  } clear_cnn{S.pc};
  S.pc.inner_its_total = 0;
  S.pc.inner_calls = 0;
  SG_TRY(c64->clear_counters(st));
  if (S.c32) SG_TRY(S.c32->clear_counters(st));
  sg_status status = SG_OK;
  // squared norm of F - A x for the returned x when a solve path already
  // computed it in FP64 (it then needs no extra residual apply)
  double final_r2 = -1.0;
  if (nF == 0.0) {
    SG_CUDA(cudaMemsetAsync(x64, 0, len * 8, st));
    final_r2 = 0.0;
  } else if (o->mode == 0) {
    Op<double> A = [&](const double* x, double* y) { return c64->apply_fine(x, y, nullptr, st); };
    Op<double> M = [&](const double* r, double* z) { return c64->twolevel(r, z, st); };
    for (;;) {
      GmresResult res;
      const sg_status gs = gmres_run<double>(c64->fine, A, M, F64, x64, false, o->rtol * nF, o->max_it - inf.outer_it,
                                             res, &hist, 1.0 / nF, st, false, stall_test && S.pc.use_cnn);
      inf.outer_it += res.its;
      // learned smoother: non-finite values or stagnation switch to RAS
      if (stall_test && S.pc.use_cnn && (gs == SG_ERR_BREAKDOWN || res.stalled) && inf.outer_it < o->max_it) {
        S.pc.use_cnn = false;
        inf.fallback_used = 1;
        SG_TRY(c64->scrub(st));
        continue;
      }
      SG_TRY(gs);
      // without a stagnation stop the last estimate is the true FP64
      // residual of the final x (computed at the closing restart)
      if (!res.stalled) final_r2 = res.est * res.est;
      break;
    }
  } else {
    SolverCtx<float>* c32 = nullptr;
    SG_TRY(get_ctx<float>(pr, c32));
    c32->fine.passes = fine_orth_passes(*o);
    if (!S.r32.ptr) SG_TRY(S.r32.alloc(len * 4));
    if (!S.d32.ptr) SG_TRY(S.d32.alloc(len * 4));
    float* r32 = dp<float>(S.r32);
    float* d32 = dp<float>(S.d32);
    Op<float> A = [&](const float* x, float* y) { return c32->apply_fine(x, y, nullptr, st); };
    Op<float> M = [&](const float* r, float* z) { return c32->twolevel(r, z, st); };
    // the FP32 correction's true FP64 progress stalls near 1e-3 per step
    // (1.5e-3 at 256^2, 1e-2 at 512^2, whatever the Arnoldi estimate
    // reaches), so a default below that only adds iterations
    const double inner = o->inner_rtol > 0 ? o->inner_rtol : 3e-4;
    const int max_ir = o->max_ir > 0 ? o->max_ir : 20;
    double rr_prev = 0.0;
    // a zero initial guess has residual F: no apply for the first step
    SG_TRY(vec_norm2<double>(x64, len, scal + 3, dp<double>(c64->fine.partial), dp<unsigned>(c64->fine.counter), st));
    SG_CUDA(cudaMemcpyAsync(S.host + 3, scal + 3, 8, cudaMemcpyDeviceToHost, st));
    SG_CUDA(cudaStreamSynchronize(st));
    bool x_is_zero = S.host[3] == 0.0;
    for (int ir = 0;; ++ir) {
      if (x_is_zero)
        SG_CUDA(cudaMemcpyAsync(dp<double>(S.r64), F64, len * 8, cudaMemcpyDeviceToDevice, st));
      else
        SG_TRY(refine_residual(pr, F64, ld, x64, ld, dp<double>(S.r64), ld, st));
      x_is_zero = false;
      {
        ProfScope phase(&pr->prof, 9, st);
        SG_TRY(vec_norm2<double>(dp<double>(S.r64), len, scal + 1, dp<double>(c64->fine.partial),
                                 dp<unsigned>(c64->fine.counter), st));
        SG_CUDA(cudaMemcpyAsync(S.host + 1, scal + 1, 8, cudaMemcpyDeviceToHost, st));
      }
      SG_CUDA(cudaStreamSynchronize(st));
      const double rr = std::sqrt(S.host[1]) / nF;
      if (!std::isfinite(rr)) {
        set_error("sg_solve: non-finite residual");
        return SG_ERR_BREAKDOWN;
      }
      hist.push_back(rr);
      if (rr <= o->rtol || ir >= max_ir || inf.outer_it >= o->max_it) {
        final_r2 = S.host[1];  // the residual of the returned x
        break;
      }
      // learned smoother: a refinement step that did not halve the residual
      // switches to RAS
      if (stall_test && S.pc.use_cnn && ir > 0 && rr > 0.5 * rr_prev) {
        S.pc.use_cnn = false;
        inf.fallback_used = 1;
      }
      rr_prev = rr;
      inf.ir_steps++;
      {
        ProfScope phase(&pr->prof, 9, st);
        SG_TRY((vec_convert<double, float>(dp<double>(S.r64), r32, len, nullptr, scal + 1, st)));
        SG_CUDA(cudaMemsetAsync(d32, 0, len * 4, st));
      }
      GmresResult res;
      // the FP32 correction solve stops on its Arnoldi estimate: its true FP32
      // residual cannot fall much below u_32 * cond(A), the FP64 loop
      // measures the real progress.  It needs to reduce the residual only by
      // the factor left to the target: at most `inner`, at least half of
      // rtol / rr (capped at 0.5), so a last step just above the target is
      // one or two iterations instead of a full `inner` reduction.
      const double inner_k = std::max(inner, std::min(0.5, 0.5 * o->rtol / rr));
      const sg_status gs = gmres_run<float>(c32->fine, A, M, r32, d32, true, inner_k, o->max_it - inf.outer_it, res,
                                            nullptr, 1.0, st, true, stall_test && S.pc.use_cnn);
      inf.outer_it += res.its;
      if (stall_test && S.pc.use_cnn && (gs == SG_ERR_BREAKDOWN || res.stalled)) {
        S.pc.use_cnn = false;
        inf.fallback_used = 1;
        SG_TRY(c32->scrub(st));
        if (gs != SG_OK) continue;  // the correction is not usable
      }
      SG_TRY(gs);
      ProfScope phase(&pr->prof, 9, st);
      SG_TRY(vec_add_scaled_f32(x64, d32, len, scal + 1, st));
    }
  }
  // true FP64 residual of the returned iterate
  if (final_r2 < 0.0) {
    if (o->mode == 1)
      SG_TRY(refine_residual(pr, F64, ld, x64, ld, dp<double>(S.r64), ld, st));
    else
      SG_TRY(apply_op<double>(pr, false, x64, ld, F64, ld, dp<double>(S.r64), ld, st));
    SG_TRY(vec_norm2<double>(dp<double>(S.r64), len, scal + 2, dp<double>(c64->fine.partial),
                             dp<unsigned>(c64->fine.counter), st));
    SG_CUDA(cudaMemcpyAsync(S.host + 2, scal + 2, 8, cudaMemcpyDeviceToHost, st));
  }
  SG_CUDA(cudaMemcpy2DAsync(X, ldx * 8, x64, ld * 8, pr->n * 8, P, cudaMemcpyDeviceToDevice, st));
  SG_CUDA(cudaStreamSynchronize(st));
  const double r2 = final_r2 >= 0.0 ? final_r2 : S.host[2];
  inf.relres = nF > 0 ? std::sqrt(r2) / nF : 0.0;
  inf.inner_it = S.pc.inner_its_total;
  if (S.pc.device_loops) {
    // coarse iterations and the kernels the coarse-solve graphs ran (the
    // launch count sees each graph launch only on the host)
    int64_t graph_kernels = 0;
    for (int which = 0; which < 2; ++which) {
      int fits = 0, cits = 0;
      int64_t k = 0;
      if (which == 0) {
        SG_TRY(c64->read_counters(&fits, &cits));
        SG_TRY(c64->coarse_graph_kernels(&k));
      } else if (S.c32) {
        SG_TRY(S.c32->read_counters(&fits, &cits));
        SG_TRY(S.c32->coarse_graph_kernels(&k));
      }
      inf.inner_it += cits;
      graph_kernels += k;
    }
    note_launches(graph_kernels);
  }
  inf.t_solve = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (o->hist_host && o->hist_cap > 0) {
    int cnt = std::min<int>(o->hist_cap, int(hist.size()));
    std::memcpy(o->hist_host, hist.data(), cnt * sizeof(double));
    inf.hist_len = cnt;
  }
  if (info) *info = inf;
  if (S.pc.ras_kernel == 2) SG_TRY(ras_inverse_check(S.pc, st));
  status = inf.relres <= o->rtol ? SG_OK : SG_NOT_CONVERGED;
  if (status == SG_NOT_CONVERGED) set_error("sg_solve: max_it reached before rtol");
  return status;
}


