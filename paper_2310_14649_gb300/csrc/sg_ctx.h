// Solver contexts shared by the solver entry points (sg_solve.cpp) and the
// graph-captured solves (sg_graph.cpp): Krylov workspaces, the host-driven
// (F)GMRES driver, the per-precision two-level preconditioner context and
// the solver state attached to a problem handle.
#pragma once

#include <chrono>
#include <cmath>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <memory>

#include "sg_cnn.h"
#include "sg_kernels.h"

namespace sg {

// --------------------------------------------------------------------------
// (F)GMRES workspace and driver
// --------------------------------------------------------------------------
template <typename T>
struct KrylovWork {
  int64_t len = 0;
  int m = 0;
  bool flexible = false;
  int passes = 1;  // Gram-Schmidt passes per Arnoldi step: 1 (CGS) or 2 (CGS2)
  DevBuf V, Z, w, tmp, tmp2, state, partial, counter;
  GmresState s{};
  double* host = nullptr;  // pinned: [0] est, [1] h_{j+1,j}, [2] bad, [4..] scalars
  Profiler* prof = nullptr;  // times the Arnoldi steps (phase kind 8) when on

  sg_status init(int64_t len_, int m_, bool flexible_) {
    len = len_;
    m = m_;
    flexible = flexible_;
    SG_TRY(V.alloc(size_t(m + 1) * len * sizeof(T)));
    if (flexible) SG_TRY(Z.alloc(size_t(m) * len * sizeof(T)));
    SG_TRY(w.alloc(size_t(len) * sizeof(T)));
    SG_TRY(tmp.alloc(size_t(len) * sizeof(T)));
    SG_TRY(tmp2.alloc(size_t(len) * sizeof(T)));
    const size_t nst = size_t(m + 1) * m + 2 * m + (m + 1) + m + 2 * (m + 1) + 8;
    SG_TRY(state.alloc(nst * sizeof(double)));
    SG_TRY(partial.alloc(size_t(2 * 152) * 32 * sizeof(double)));
    SG_TRY(counter.alloc(64));
    double* p = dp<double>(state);
    s.H = p;
    p += size_t(m + 1) * m;
    s.cs = p;
    p += m;
    s.sn = p;
    p += m;
    s.g = p;
    p += m + 1;
    s.y = p;
    p += m;
    s.hsum = p;
    p += 2 * (m + 1);
    s.scal = p;
    SG_CUDA(cudaHostAlloc(&host, 16 * sizeof(double), cudaHostAllocMapped));
    std::memset(host, 0, 16 * sizeof(double));
    return SG_OK;
  }
  ~KrylovWork() {
    if (host) cudaFreeHost(host);
  }
  T* Vj(int j) { return dp<T>(V) + int64_t(j) * len; }
  T* Zj(int j) { return dp<T>(Z) + int64_t(j) * len; }
};

template <typename T>
using Op = std::function<sg_status(const T*, T*)>;

template <typename T> const T* dp_sel(const DevBuf& b64, const DevBuf& b32);
template <> inline const double* dp_sel<double>(const DevBuf& b64, const DevBuf&) { return dp<double>(b64); }
template <> inline const float* dp_sel<float>(const DevBuf&, const DevBuf& b32) { return dp<float>(b32); }

// y = a - b (elementwise), used for r = F - A x
template <typename T>
inline sg_status sub_into(const T* a, const T* b, T* y, int64_t len, KrylovWork<T>& W, cudaStream_t st) {
  // y = a; y -= 1 * b  (axpy with a device coefficient -1)
  SG_CUDA(cudaMemcpyAsync(y, a, len * sizeof(T), cudaMemcpyDeviceToDevice, st));
  static thread_local double* minus_one = nullptr;
  if (!minus_one) {
    SG_CUDA(cudaMalloc(&minus_one, sizeof(double)));
    const double v = -1.0;
    SG_CUDA(cudaMemcpy(minus_one, &v, sizeof(double), cudaMemcpyHostToDevice));
  }
  return vec_axpy_multi<T>(b, 0, 1, minus_one, y, len, st);
}

struct GmresResult {
  int its = 0;
  double est = 0.0;     // last residual estimate (absolute)
  bool converged = false;
  bool stalled = false; // stopped by the stagnation test
};

// stagnation test of a solve with the learned smoother: after kStallIts
// iterations the residual estimate must have dropped below kStallRatio
// times its value kStallIts iterations earlier
constexpr int kStallIts = 10;
constexpr double kStallRatio = 0.7;

// Right-preconditioned restarted GMRES (flexible when W.flexible: the
// preconditioned vectors are kept and x += Z y).  Stops when the residual
// estimate drops below tol_abs; at each restart the true residual is used.
template <typename T>
inline sg_status gmres_run(KrylovWork<T>& W, const Op<T>& A, const Op<T>& M, const T* F, T* x, bool x_zero,
                           double tol_abs, int max_it, GmresResult& res, std::vector<double>* hist, double hist_scale,
                           cudaStream_t st, bool trust_estimate, bool stall_test = false) {
  const int64_t len = W.len;
  res = GmresResult{};
  std::vector<double> ests;
  bool first = true;
  if (W.passes == 1) SG_CUDA(cudaMemsetAsync(W.s.hsum + (W.m + 1), 0, (W.m + 1) * sizeof(double), st));
  for (;;) {
    // r0 = F - A x
    if (first && x_zero) {
      SG_CUDA(cudaMemcpyAsync(W.Vj(0), F, len * sizeof(T), cudaMemcpyDeviceToDevice, st));
    } else {
      SG_TRY(A(x, dp<T>(W.w)));
      SG_TRY(sub_into<T>(F, dp<T>(W.w), W.Vj(0), len, W, st));
    }
    first = false;
    SG_TRY(vec_norm2<T>(W.Vj(0), len, W.s.scal + 3, dp<double>(W.partial), dp<unsigned>(W.counter), st));
    SG_CUDA(cudaMemcpyAsync(W.host + 4, W.s.scal + 3, sizeof(double), cudaMemcpyDeviceToHost, st));
    SG_CUDA(cudaStreamSynchronize(st));
    const double beta = std::sqrt(W.host[4]);
    if (!std::isfinite(beta)) {
      set_error("GMRES: non-finite residual");
      return SG_ERR_BREAKDOWN;
    }
    res.est = beta;
    if (beta <= tol_abs) {
      res.converged = true;
      return SG_OK;
    }
    if (res.its >= max_it) return SG_OK;
    SG_TRY(vec_scale_by<T>(W.Vj(0), W.Vj(0), len, W.s.scal + 3, true, st));
    SG_TRY(gmres_init(W.s, W.m, W.s.scal + 3, st));
    int k = 0;
    bool stop = false;
    for (int j = 0; j < W.m; ++j) {
      T* zj = W.flexible ? W.Zj(j) : dp<T>(W.tmp);
      SG_TRY(M(W.Vj(j), zj));
      SG_TRY(A(zj, dp<T>(W.w)));
      ProfScope arnoldi(W.prof, 8, st);
      double* h1 = W.s.hsum;
      double* h2 = W.s.hsum + (W.m + 1);
      SG_TRY(vec_mdot<T>(dp<T>(W.V), len, j + 1, dp<T>(W.w), len, h1, dp<double>(W.partial),
                         dp<unsigned>(W.counter), st));
      if (W.passes == 1) {
        // one classical pass; the second coefficient column stays zero
        SG_TRY(vec_maxpy_norm<T>(dp<T>(W.V), len, j + 1, h1, dp<T>(W.w), len, W.s.scal, dp<double>(W.partial),
                                 dp<unsigned>(W.counter), st));
      } else {
        SG_TRY(vec_maxpy_mdot<T>(dp<T>(W.V), len, j + 1, h1, dp<T>(W.w), len, h2, dp<double>(W.partial),
                                 dp<unsigned>(W.counter), st));
        SG_TRY(vec_maxpy_norm<T>(dp<T>(W.V), len, j + 1, h2, dp<T>(W.w), len, W.s.scal, dp<double>(W.partial),
                                 dp<unsigned>(W.counter), st));
      }
      SG_TRY(gmres_givens(W.s, W.m, j, W.host, st));
      SG_TRY(vec_scale_by<T>(dp<T>(W.w), W.Vj(j + 1), len, W.s.scal + 1, false, st));
      arnoldi.stop();
      SG_CUDA(cudaStreamSynchronize(st));
      res.its++;
      k = j + 1;
      const double est = W.host[0], hn = W.host[1];
      if (W.host[2] != 0.0) {
        set_error("GMRES: non-finite value in the Arnoldi process");
        return SG_ERR_BREAKDOWN;
      }
      res.est = est;
      if (hist) hist->push_back(est * hist_scale);
      if (est <= tol_abs || hn == 0.0) {
        stop = true;
        break;
      }
      if (stall_test) {
        ests.push_back(est);
        const size_t q = ests.size();
        if (q > size_t(kStallIts) && est > kStallRatio * ests[q - 1 - kStallIts]) {
          res.stalled = true;
          break;
        }
      }
      if (res.its >= max_it) break;
    }
    SG_TRY(gmres_backsolve(W.s, W.m, k, st));
    if (W.flexible) {
      SG_TRY(vec_axpy_multi<T>(dp<T>(W.Z), len, k, W.s.y, x, len, st));
    } else {
      SG_CUDA(cudaMemsetAsync(W.tmp2.ptr, 0, len * sizeof(T), st));
      SG_TRY(vec_axpy_multi<T>(dp<T>(W.V), len, k, W.s.y, dp<T>(W.tmp2), len, st));
      SG_TRY(M(dp<T>(W.tmp2), dp<T>(W.tmp)));
      static thread_local double* one = nullptr;
      if (!one) {
        SG_CUDA(cudaMalloc(&one, sizeof(double)));
        const double v = 1.0;
        SG_CUDA(cudaMemcpy(one, &v, sizeof(double), cudaMemcpyHostToDevice));
      }
      SG_TRY(vec_axpy_multi<T>(dp<T>(W.tmp), 0, 1, one, x, len, st));
    }
    if (stop && trust_estimate) {  // inner solves stop on the Arnoldi estimate
      res.converged = true;
      return SG_OK;
    }
    if (res.stalled) return SG_OK;
    if (res.its >= max_it && !stop) {
      // report the true residual of the final iterate
      SG_TRY(A(x, dp<T>(W.w)));
      SG_TRY(sub_into<T>(F, dp<T>(W.w), dp<T>(W.tmp), len, W, st));
      SG_TRY(vec_norm2<T>(dp<T>(W.tmp), len, W.s.scal + 3, dp<double>(W.partial), dp<unsigned>(W.counter), st));
      SG_CUDA(cudaMemcpyAsync(W.host + 4, W.s.scal + 3, sizeof(double), cudaMemcpyDeviceToHost, st));
      SG_CUDA(cudaStreamSynchronize(st));
      res.est = std::sqrt(W.host[4]);
      res.converged = res.est <= tol_abs;
      return SG_OK;
    }
  }
}

// --------------------------------------------------------------------------
// Per-precision solver context: operator, preconditioner and workspaces.
// --------------------------------------------------------------------------
// Kernel nodes of a recorded loop nest: outside the loops, per restart
// cycle, per Arnoldi iteration (nested loops excluded).  The launch count
// adds them for the executions the device counters report.
struct RegionCounts {
  int64_t fixed = 0, restart = 0, iter = 0;
  int64_t total(int64_t calls, int64_t restarts, int64_t iters) const {
    return calls * fixed + restarts * restart + iters * iter;
  }
};

template <typename T>
struct SolverCtx;
// Records a device-driven coarse GMRES solve r_c -> e_c (the 2GV3 inner
// solve, loops as conditional WHILE nodes) into the capture active on s1;
// s2 and s3 capture the loop bodies (sg_graph.cpp).
template <typename T>
sg_status capture_coarse(SolverCtx<T>& c, cudaStream_t s1, cudaStream_t s2, cudaStream_t s3);

template <typename T>
struct SolverCtx {
  sg_problem* pr = nullptr;
  Precond* pc = nullptr;
  int64_t ld = 0, len = 0, ldc = 0, lenc = 0;
  KrylovWork<T> fine, coarse;
  DevBuf r1, zt, rc, ec;          // two-level temporaries
  DevBuf consts;                  // device doubles {1, -1}
  // device-driven coarse solve, captured once into a CUDA graph
  DevBuf dg_iv, dg_tol;
  DevGmres dg{};
  // device-driven fine FGMRES (graph-captured solves)
  DevBuf fdg_iv, fdg_tol;
  DevGmres fdg{};
  RegionCounts cc_coarse, cc_fine;  // kernel nodes per region of the recorded loops
  int64_t coarse_graph_launches = 0;
  cudaGraphExec_t cexec = nullptr;
  cudaStream_t cap[3] = {nullptr, nullptr, nullptr};
  std::vector<DevBuf> amgbuf;     // b, x, t per level
  AmgWork<T> aw;
  bool ready = false;

  sg_status init(sg_problem* p, Precond* c, int restart) {
    pr = p;
    pc = c;
    ld = pr->ld;
    len = int64_t(pr->P) * ld;
    ldc = pc->co.ldc;
    lenc = int64_t(pr->P) * ldc;
    SG_TRY(fine.init(len, restart, true));
    fine.prof = &pr->prof;
    // flexible storage: the update x += M (V y) reuses Z_j = M V_j
    SG_TRY(coarse.init(lenc, pc->inner_restart, true));
    coarse.passes = pc->inner_passes;
    SG_TRY(r1.alloc(len * sizeof(T)));
    SG_TRY(zt.alloc(len * sizeof(T)));
    SG_TRY(consts.alloc(2 * sizeof(double)));
    {
      const double cv[2] = {1.0, -1.0};
      SG_CUDA(cudaMemcpy(consts.ptr, cv, sizeof cv, cudaMemcpyHostToDevice));
    }
    SG_TRY(dg_iv.alloc(16 * sizeof(int)));
    SG_TRY(dg_tol.alloc(4 * sizeof(double)));
    dg.iv = dp<int>(dg_iv);
    dg.dtol = dp<double>(dg_tol);
    SG_TRY(fdg_iv.alloc(16 * sizeof(int)));
    SG_TRY(fdg_tol.alloc(4 * sizeof(double)));
    fdg.iv = dp<int>(fdg_iv);
    fdg.dtol = dp<double>(fdg_tol);
    {
      const int cap_it = pc->inner_max;
      SG_CUDA(cudaMemcpy(dg.iv + 2, &cap_it, sizeof(int), cudaMemcpyHostToDevice));
    }
    SG_TRY(rc.alloc(lenc * sizeof(T)));
    SG_TRY(ec.alloc(lenc * sizeof(T)));
    amgbuf.resize(3 * pc->amg.size());
    aw.b.clear();
    aw.x.clear();
    aw.t.clear();
    for (size_t l = 0; l < pc->amg.size(); ++l) {
      const size_t sz = size_t(pr->P) * pc->amg[l].ld * sizeof(T);
      for (int q = 0; q < 3; ++q) SG_TRY(amgbuf[3 * l + q].alloc(sz));
      aw.b.push_back(amgbuf[3 * l].as<T>());
      aw.x.push_back(amgbuf[3 * l + 1].as<T>());
      aw.t.push_back(amgbuf[3 * l + 2].as<T>());
    }
    ready = true;
    return SG_OK;
  }

  ~SolverCtx() {
    if (cexec) cudaGraphExecDestroy(cexec);
    for (auto& c : cap)
      if (c) cudaStreamDestroy(c);
  }

  // Clears every work vector.  After a non-finite value the padding rows
  // (n..ld-1) of the Krylov vectors can hold NaN that later full-length
  // reductions would pick up; a solve that continues after such a value
  // (the fallback from the learned smoother) starts from clean buffers.
  sg_status scrub(cudaStream_t st) {
    for (DevBuf* b : {&fine.V, &fine.Z, &fine.w, &fine.tmp, &fine.tmp2, &coarse.V, &coarse.Z, &coarse.w, &coarse.tmp,
                      &coarse.tmp2, &r1, &zt, &rc, &ec})
      if (b->ptr) SG_CUDA(cudaMemsetAsync(b->ptr, 0, b->bytes, st));
    for (DevBuf& b : amgbuf)
      if (b.ptr) SG_CUDA(cudaMemsetAsync(b.ptr, 0, b.bytes, st));
    return SG_OK;
  }

  sg_status apply_fine(const T* X, T* Y, const T* F, cudaStream_t st) {
    return apply_op<T>(pr, false, X, ld, F, ld, Y, ld, st);
  }
  sg_status apply_coarse(const T* X, T* Y, cudaStream_t st) {
    return apply_op<T>(pr, true, X, ldc, nullptr, 0, Y, ldc, st);
  }
  // AMG V-cycle per mode on a coarse block
  sg_status amg(const T* B, T* X, cudaStream_t st) {
    const AmgLevel& L0 = pc->amg[0];
    SG_CUDA(cudaMemcpy2DAsync(aw.b[0], L0.ld * sizeof(T), B, ldc * sizeof(T), pc->co.nc * sizeof(T), pr->P,
                              cudaMemcpyDeviceToDevice, st));
    return amg_vcycle<T>(pc->amg, aw, pr->P, st, X, ldc);
  }
  // coarse preconditioner on a block already in the AMG level-0 input:
  // V-cycle, copy out to `out` (coarse ld), Kronecker factor
  // (with Zs: the result also into slot dg.iv[0] of Zs, slot stride lenc)
  sg_status coarse_pc_from_b0(T* out, cudaStream_t st, T* Zs = nullptr) {
    SG_TRY(amg_vcycle<T>(pc->amg, aw, pr->P, st, out, ldc));
    return node_transform<T>(out, ldc, pc->co.nc, pr->P, dp_sel<T>(pc->gkron64, pc->gkron32), st, Zs, lenc,
                             Zs ? dg.iv : nullptr);
  }

  // adds a WHILE node driven by `h` at the capture point of `st`
  static sg_status add_while(cudaStream_t st, cudaGraphConditionalHandle h, cudaGraph_t* body) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* ed = nullptr;
    size_t nd = 0;
    SG_CUDA(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, &ed, &nd));
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    SG_CUDA(cudaGraphAddNode(&node, g, deps, ed, nd, &p));
    *body = p.conditional.phGraph_out[0];
    SG_CUDA(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    return SG_OK;
  }

  // fine apply without the profiler (Y = F - A X when F, else A X)
  sg_status apply_raw_fine(const T* X, T* Y, const T* F, cudaStream_t st) {
    return apply_any<T>(pr, false, X, ld, F, ld, Y, ld, st);
  }
  // iteration counters summed over solves (device): fine FGMRES, coarse GMRES
  sg_status clear_counters(cudaStream_t st) {
    for (int* iv : {fdg.iv, dg.iv}) {
      SG_CUDA(cudaMemsetAsync(iv + 4, 0, sizeof(int), st));
      SG_CUDA(cudaMemsetAsync(iv + 6, 0, sizeof(int), st));
    }
    coarse_graph_launches = 0;
    return SG_OK;
  }
  // fine and coarse iterations and restart cycles summed since clear_counters
  sg_status read_counters(int* fine_its, int* coarse_its, int* fine_restarts = nullptr,
                          int* coarse_restarts = nullptr) {
    int f[8], c[8];
    SG_CUDA(cudaMemcpy(f, fdg.iv, sizeof f, cudaMemcpyDeviceToHost));
    SG_CUDA(cudaMemcpy(c, dg.iv, sizeof c, cudaMemcpyDeviceToHost));
    *fine_its = f[4];
    *coarse_its = c[4];
    if (fine_restarts) *fine_restarts = f[6];
    if (coarse_restarts) *coarse_restarts = c[6];
    return SG_OK;
  }
  // kernels run inside the standalone coarse-solve graph launches since
  // clear_counters (host-driven solves)
  sg_status coarse_graph_kernels(int64_t* out) {
    int fits = 0, cits = 0, fr = 0, cr = 0;
    SG_TRY(read_counters(&fits, &cits, &fr, &cr));
    *out = cc_coarse.total(coarse_graph_launches, cr, cits);
    return SG_OK;
  }

  // coarse apply without the profiler (used inside graph capture)
  sg_status apply_raw(const T* X, T* Y, const T* F, cudaStream_t st) {
    return apply_any<T>(pr, true, X, ldc, F, ldc, Y, ldc, st);
  }

  // Device-driven restarted GMRES on the coarse system (the 2GV3 inner
  // solve): every decision is taken on the device, loops are conditional
  // WHILE nodes, so one graph launch performs a whole coarse solve from rc
  // into ec without a host round trip.
  sg_status build_coarse_graph() {
    SG_TRY(capture_prepare());
    for (auto& c : cap)
      if (!c) SG_CUDA(cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking));
    cudaGraph_t g;
    SG_CUDA(cudaStreamBeginCapture(cap[0], cudaStreamCaptureModeRelaxed));
    const sg_status s = capture_coarse<T>(*this, cap[0], cap[1], cap[2]);
    const cudaError_t e = cudaStreamEndCapture(cap[0], &g);
    SG_TRY(s);
    SG_CUDA(e);
    SG_CUDA(cudaGraphInstantiate(&cexec, g, 0));
    SG_CUDA(cudaGraphDestroy(g));
    return SG_OK;
  }

  // everything a captured launch needs must exist before a capture starts:
  // specialised kernels, kernel attributes, network buffers
  sg_status capture_prepare() {
    if (sizeof(T) == 8) {
      SG_TRY(asm_prepare(pr, pr->fine, pr->asm_fine, nullptr));
      SG_TRY(asm_prepare(pr, pc->co.ell, pc->co.asm_c, nullptr));
      SG_TRY(resid_prepare(pr, nullptr));
    }
    if (pr->apply_mode != 1 && jit_eligible(pr)) {
      SG_TRY(jit_apply_build(pr, sizeof(T) == 8 ? 2 : 0));
      SG_TRY(jit_apply_build(pr, sizeof(T) == 8 ? 3 : 1));
    }
    SG_TRY(kernel_attrs_init());
    if (pr->cnn) SG_TRY(pr->cnn->reserve(pr->P));
    return SG_OK;
  }

  // e_c ~ A_c^{-1} r_c by one launch of the device-driven coarse GMRES graph
  sg_status coarse_solve_graph(cudaStream_t st) {
    if (!cexec) SG_TRY(build_coarse_graph());
    SG_CUDA(cudaGraphLaunch(cexec, st));
    ++coarse_graph_launches;
    return SG_OK;
  }

  // e_c ~ A_c^{-1} r_c by GMRES preconditioned with the AMG V-cycle
  // (host-driven reference path of the same algorithm)
  sg_status coarse_solve(const T* Rc, T* Ec, cudaStream_t st) {
    SG_CUDA(cudaMemsetAsync(Ec, 0, lenc * sizeof(T), st));
    // absolute tolerance relative to ||r_c||
    SG_TRY(vec_norm2<T>(Rc, lenc, coarse.s.scal + 5, dp<double>(coarse.partial), dp<unsigned>(coarse.counter), st));
    SG_CUDA(cudaMemcpyAsync(coarse.host + 5, coarse.s.scal + 5, sizeof(double), cudaMemcpyDeviceToHost, st));
    SG_CUDA(cudaStreamSynchronize(st));
    const double nr = std::sqrt(coarse.host[5]);
    if (nr == 0.0) return SG_OK;
    Op<T> A = [&](const T* x, T* y) { return apply_coarse(x, y, st); };
    Op<T> M = [&](const T* x, T* y) {
      SG_TRY(amg(x, y, st));
      return node_transform<T>(y, ldc, pc->co.nc, pr->P, dp_sel<T>(pc->gkron64, pc->gkron32), st);
    };
    GmresResult res;
    SG_TRY(gmres_run<T>(coarse, A, M, Rc, Ec, true, pc->inner_rtol * nr, pc->inner_max, res, nullptr, 1.0, st,
                        true));
    pc->inner_its_last = res.its;
    pc->inner_its_total += res.its;
    pc->inner_calls++;
    return SG_OK;
  }
  // Q r = R_0^T A_c^{-1} R_0 r
  sg_status coarse_correction(const T* R, T* Z, bool add, cudaStream_t st) {
    ProfScope phase(&pr->prof, 7, st);
    SG_TRY(spmm<T>(pc->co.R, R, ld, nullptr, 0, dp<T>(rc), ldc, pr->P, 0, st));
    if (pc->device_loops) {
      SG_TRY(coarse_solve_graph(st));
      pc->last_coarse_dtype = sizeof(T) == 8 ? 0 : 1;
    }
    else
      SG_TRY(coarse_solve(dp<T>(rc), dp<T>(ec), st));
    if (!add) SG_CUDA(cudaMemsetAsync(Z, 0, len * sizeof(T), st));
    SG_TRY(spmm<T>(pc->co.RT, dp<T>(ec), ldc, nullptr, 0, Z, ld, pr->P, 1, st));
    return SG_OK;
  }
  // smoother S r = omega G~^{-1} RAS(r), or omega_cnn G~^{-1} CNN(r) while
  // the learned smoother is active; FP32 inputs are recorded while a
  // harvest for training is on
  sg_status smooth(const T* R, T* Z, cudaStream_t st) {
    ProfScope phase(&pr->prof, 6, st);
    Harvest& h = pc->harvest;
    if (sizeof(T) == 4 && h.on && h.count < h.cap) {
      SG_CUDA(cudaMemcpyAsync(dp<float>(h.pool) + h.count * len, R, len * sizeof(T), cudaMemcpyDeviceToDevice, st));
      ++h.count;
    }
    if (pc->use_cnn) return cnn_smooth<T>(pr, *pc, R, ld, Z, true, st);
    return ras_apply<T>(*pc, pr->n, pr->P, R, ld, Z, st, true, &pr->prof);
  }
  // two-level cycle: z = S r; z += Q (r - A z); z += S (r - A z)
  sg_status twolevel(const T* R, T* Z, cudaStream_t st) {
    SG_TRY(smooth(R, Z, st));
    SG_TRY(apply_fine(Z, dp<T>(r1), R, st));
    SG_TRY(coarse_correction(dp<T>(r1), Z, true, st));
    SG_TRY(apply_fine(Z, dp<T>(r1), R, st));
    SG_TRY(smooth(dp<T>(r1), dp<T>(zt), st));
    static thread_local double* one = nullptr;
    if (!one) {
      SG_CUDA(cudaMalloc(&one, sizeof(double)));
      const double v = 1.0;
      SG_CUDA(cudaMemcpy(one, &v, sizeof(double), cudaMemcpyHostToDevice));
    }
    return vec_axpy_multi<T>(dp<T>(zt), 0, 1, one, Z, len, st);
  }
};


struct SolverState {
  Precond pc;
  std::unique_ptr<SolverCtx<double>> c64;
  std::unique_ptr<SolverCtx<float>> c32;
  int restart = 30;
  DevBuf x64, r64, r32, d32, io, io2, scal;  // IR and I/O buffers
  DevBuf ir_d, ir_i;                         // graph-captured refinement: scalars, counters
  bool dirty = false;                        // the last solve ended on an error
  double* host = nullptr;                    // pinned scalars
  uint64_t serial;                           // distinguishes successive preconditioner setups
  uint64_t ctx_gen = 0;                      // bumped whenever c64 or c32 is dropped or re-created:
                                             // recorded graphs hold their buffers by address
  SolverState() {
    static std::atomic<uint64_t> next{1};
    serial = next++;
  }
  ~SolverState() {
    if (host) cudaFreeHost(host);
  }
};

template <typename T> std::unique_ptr<SolverCtx<T>>& ctx_of(SolverState& S);
template <> inline std::unique_ptr<SolverCtx<double>>& ctx_of<double>(SolverState& S) { return S.c64; }
template <> inline std::unique_ptr<SolverCtx<float>>& ctx_of<float>(SolverState& S) { return S.c32; }

template <typename T>
inline sg_status get_ctx(sg_problem* pr, SolverCtx<T>*& out) {
  SolverState& S = *pr->solver;
  auto& c = ctx_of<T>(S);
  if (!c || !c->ready || c->fine.m != S.restart) {
    ++S.ctx_gen;
    c.reset(new SolverCtx<T>());
    SG_TRY(c->init(pr, &S.pc, S.restart));
  }
  out = c.get();
  return SG_OK;
}

// Gram-Schmidt passes of the outer (F)GMRES chosen by the solve options
inline int fine_orth_passes(const sg_solve_opts& o) { return o.orth_passes > 0 ? o.orth_passes : 1; }

}  // namespace sg
