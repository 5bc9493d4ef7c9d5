// Graph-captured solves: the whole mixed-precision solve of Sec. 3's
// two-level FGMRES (refinement loop, fine FGMRES restarts and Arnoldi
// steps, the inner coarse GMRES of the 2GV3 variant) recorded as one CUDA
// graph whose loops are conditional WHILE nodes decided on the device, and
// a batch of independent systems of different sizes recorded as parallel
// branches of one graph, so one launch solves them all.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

#include "sg_ctx.h"

namespace sg {

namespace {

// profiling brackets apply launches with events read on the host; they are
// switched off while a graph is recorded
struct ProfilerOff {
  Profiler& p;
  bool was;
  explicit ProfilerOff(Profiler& pp) : p(pp), was(pp.on) { p.on = false; }
  ~ProfilerOff() { p.on = was; }
};

}  // namespace

template <typename T>
sg_status capture_coarse(SolverCtx<T>& c, cudaStream_t s1, cudaStream_t s2, cudaStream_t s3) {
  KrylovWork<T>& W = c.coarse;
  const int m = W.m;
  const Precond& pc = *c.pc;
  const AmgLevel& L0 = pc.amg[0];
  double* h1 = W.s.hsum;
  double* h2 = W.s.hsum + (m + 1);
  T* V = dp<T>(W.V);
  T* Zc = dp<T>(W.Z);
  T* w = dp<T>(W.w);
  T* tmp = dp<T>(W.tmp);
  T* Rc = dp<T>(c.rc);
  T* Ec = dp<T>(c.ec);
  double* part = dp<double>(W.partial);
  unsigned* cnt = dp<unsigned>(W.counter);
  const int64_t ldc = c.ldc, lenc = c.lenc;
  const int* jdev = c.dg.iv;

  cudaStreamCaptureStatus cs;
  cudaGraph_t g;
  SG_CUDA(cudaStreamGetCaptureInfo(s1, &cs, nullptr, &g, nullptr, nullptr, nullptr));
  cudaGraphConditionalHandle hout;
  SG_CUDA(cudaGraphConditionalHandleCreate(&hout, g, 0, 0));
  // one Arnoldi step (the WHILE body of a cycle), recorded on s3
  auto arnoldi_step = [&](cudaGraph_t body_in, cudaGraphConditionalHandle hin) -> sg_status {
    SG_CUDA(cudaStreamBeginCaptureToGraph(s3, body_in, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    // the AMG input b_0 holds V_j (written with V_j), Z_j = M V_j
    SG_TRY(c.coarse_pc_from_b0(tmp, s3, Zc));
    SG_TRY(c.apply_raw(tmp, w, nullptr, s3));
    SG_TRY(dg_mdot<T>(V, lenc, w, lenc, h1, part, cnt, jdev, m, s3));
    if (W.passes == 1) {
      SG_TRY(dg_axpy_norm<T>(V, lenc, h1, w, lenc, W.s.scal, part, cnt, jdev, s3));
    } else {
      SG_TRY(dg_axpy_norm<T>(V, lenc, h1, w, lenc, nullptr, part, cnt, jdev, s3));
      SG_TRY(dg_mdot<T>(V, lenc, w, lenc, h2, part, cnt, jdev, m, s3));
      SG_TRY(dg_axpy_norm<T>(V, lenc, h2, w, lenc, W.s.scal, part, cnt, jdev, s3));
    }
    SG_TRY(dg_givens(c.dg, W.s, m, hin, s3));
    SG_TRY(dg_scale_next<T>(w, V, lenc, lenc, c.dg, W.s.scal + 1, s3, c.aw.b[0], L0.ld, ldc, pc.co.nc));
    SG_CUDA(cudaStreamEndCapture(s3, &body_in));
    return SG_OK;
  };
  // one restart cycle from V_0 = r0 with ||r0||^2 in scal[3], recorded on sc
  // (part of graph gc); n_step receives the kernels of one Arnoldi step
  auto cycle = [&](cudaStream_t sc, cudaGraph_t gc, int64_t* n_step) -> sg_status {
    cudaGraphConditionalHandle hin;
    SG_CUDA(cudaGraphConditionalHandleCreate(&hin, gc, 0, 0));
    SG_TRY(dg_start(c.dg, W.s, m, W.s.scal + 3, hin, sc));
    SG_TRY(vec_scale_by<T>(V, V, lenc, W.s.scal + 3, true, sc));
    SG_TRY(dg_copy_vj<T>(V, lenc, ldc, c.aw.b[0], L0.ld, pc.co.nc, c.pr->P, c.dg, sc));  // b_0 = V_0
    cudaGraph_t body_in;
    SG_TRY(SolverCtx<T>::add_while(sc, hin, &body_in));
    const int64_t a = launch_count();
    SG_TRY(arnoldi_step(body_in, hin));
    *n_step = launch_count() - a;
    // x += M (V y) = Z y with the stored Z_j = M V_j
    SG_TRY(dg_backsolve(c.dg, W.s, m, sc));
    SG_TRY(dg_axpy_multi<T>(Zc, lenc, W.s.y, Ec, lenc, jdev, sc));
    SG_TRY(dg_end(c.dg, W.s, hout, sc));
    return SG_OK;
  };

  const int64_t k0 = launch_count();
  // e_c = 0, so the first cycle starts from r0 = r_c without an apply
  SG_CUDA(cudaMemsetAsync(Ec, 0, lenc * sizeof(T), s1));
  if (W.passes == 1) SG_CUDA(cudaMemsetAsync(h2, 0, (m + 1) * sizeof(double), s1));
  SG_TRY(vec_norm2<T>(Rc, lenc, W.s.scal + 5, part, cnt, s1));
  SG_CUDA(cudaMemcpyAsync(V, Rc, lenc * sizeof(T), cudaMemcpyDeviceToDevice, s1));
  SG_CUDA(cudaMemcpyAsync(W.s.scal + 3, W.s.scal + 5, sizeof(double), cudaMemcpyDeviceToDevice, s1));
  SG_TRY(dg_init(c.dg, W.s.scal + 5, pc.inner_rtol, hout, s1));
  const int64_t k1 = launch_count();
  int64_t n1 = 0, n2 = 0;
  SG_TRY(cycle(s1, g, &n1));
  const int64_t k2 = launch_count();
  // further cycles (a full cycle without convergence): r0 = r_c - A_c e_c
  cudaGraph_t body_out;
  SG_TRY(SolverCtx<T>::add_while(s1, hout, &body_out));
  SG_CUDA(cudaStreamBeginCaptureToGraph(s2, body_out, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  SG_TRY(c.apply_raw(Ec, V, Rc, s2));
  SG_TRY(vec_norm2<T>(V, lenc, W.s.scal + 3, part, cnt, s2));
  SG_TRY(cycle(s2, body_out, &n2));
  SG_CUDA(cudaStreamEndCapture(s2, &body_out));
  const int64_t k3 = launch_count();
  // kernels per solve = fixed + cycles x restart + steps x iter, every
  // solve running the first cycle once
  const int64_t first = (k2 - k1) - n1, later = (k3 - k2) - n2;
  c.cc_coarse = RegionCounts{(k1 - k0) + first - later, later, n2};
  note_launches(-(k3 - k0));  // recorded, not launched
  return SG_OK;
}

// Streams of one recorded solve: [0] top level, [1] refinement body,
// [2] fine restart body, [3] fine Arnoldi body, [4] coarse restart body,
// [5] coarse Arnoldi body.
struct CapStreams {
  cudaStream_t s[6] = {};
  sg_status create() {
    for (auto& x : s)
      if (!x) SG_CUDA(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
    return SG_OK;
  }
  ~CapStreams() {
    for (auto& x : s)
      if (x) cudaStreamDestroy(x);
  }
};

// z = B r, the two-level cycle of Eq. RAS_2L (smoother, coarse correction,
// smoother), recorded with the coarse solve inline.
template <typename T>
static sg_status capture_twolevel(SolverCtx<T>& c, const T* R, T* Z, cudaStream_t st, cudaStream_t c2,
                                  cudaStream_t c3) {
  const int P = c.pr->P;
  T* r1 = dp<T>(c.r1);
  SG_TRY(c.smooth(R, Z, st));
  SG_TRY(c.apply_raw_fine(Z, r1, R, st));
  SG_TRY(spmm<T>(c.pc->co.R, r1, c.ld, nullptr, 0, dp<T>(c.rc), c.ldc, P, 0, st));
  SG_TRY(capture_coarse<T>(c, st, c2, c3));
  SG_TRY(spmm<T>(c.pc->co.RT, dp<T>(c.ec), c.ldc, nullptr, 0, Z, c.ld, P, 1, st));
  SG_TRY(c.apply_raw_fine(Z, r1, R, st));
  SG_TRY(c.smooth(r1, dp<T>(c.zt), st));
  return vec_axpy_multi<T>(dp<T>(c.zt), 0, 1, dp<double>(c.consts), Z, c.len, st);
}

// Flexible GMRES(m) on the fine system A x = b, device-driven: x is updated
// in place from its current value until ||b - A x|| <= rtol ||b|| (by the
// Arnoldi estimate when trust, else by the true residual of a restart) or
// the iteration cap stored in fdg.iv[2].
template <typename T>
static sg_status capture_fine(SolverCtx<T>& c, const T* b, T* x, double rtol, bool trust, const CapStreams& S,
                              cudaStream_t top, const double* rr2 = nullptr, const double* nf2 = nullptr,
                              double target = 0.0) {
  KrylovWork<T>& W = c.fine;
  const int m = W.m;
  const int64_t len = c.len;
  double* h1 = W.s.hsum;
  double* h2 = W.s.hsum + (m + 1);
  T* V = dp<T>(W.V);
  T* Zs = dp<T>(W.Z);
  T* w = dp<T>(W.w);
  T* vbuf = dp<T>(W.tmp);
  T* zbuf = dp<T>(W.tmp2);
  double* part = dp<double>(W.partial);
  unsigned* cnt = dp<unsigned>(W.counter);
  const int* jdev = c.fdg.iv;
  const cudaStream_t f2 = S.s[2], f3 = S.s[3];

  const int64_t k0 = launch_count();
  if (W.passes == 1) SG_CUDA(cudaMemsetAsync(h2, 0, (m + 1) * sizeof(double), top));
  SG_TRY(vec_norm2<T>(b, len, W.s.scal + 5, part, cnt, top));
  cudaStreamCaptureStatus cs;
  cudaGraph_t g;
  SG_CUDA(cudaStreamGetCaptureInfo(top, &cs, nullptr, &g, nullptr, nullptr, nullptr));
  cudaGraphConditionalHandle hout, hin;
  SG_CUDA(cudaGraphConditionalHandleCreate(&hout, g, 0, 0));
  SG_TRY(dg_init(c.fdg, W.s.scal + 5, rtol, hout, top, rr2, nf2, target));
  const int64_t k1 = launch_count();
  int64_t k2 = 0, k3 = 0;
  cudaGraph_t body_out;
  SG_TRY(SolverCtx<T>::add_while(top, hout, &body_out));
  {
    SG_CUDA(cudaStreamBeginCaptureToGraph(f2, body_out, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    // V_0 = (b - A x) / beta
    SG_TRY(c.apply_raw_fine(x, V, b, f2));
    SG_TRY(vec_norm2<T>(V, len, W.s.scal + 3, part, cnt, f2));
    SG_CUDA(cudaGraphConditionalHandleCreate(&hin, body_out, 0, 0));
    SG_TRY(dg_start(c.fdg, W.s, m, W.s.scal + 3, hin, f2));
    SG_TRY(vec_scale_by<T>(V, V, len, W.s.scal + 3, true, f2));
    cudaGraph_t body_in;
    SG_TRY(SolverCtx<T>::add_while(f2, hin, &body_in));
    k2 = launch_count();
    {
      SG_CUDA(cudaStreamBeginCaptureToGraph(f3, body_in, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
      // Z_j = B V_j, w = A Z_j, Gram-Schmidt against V_0..V_j, rotation, V_{j+1}
      SG_TRY(dg_copy_vj<T>(V, len, c.ld, vbuf, c.ld, c.pr->n, c.pr->P, c.fdg, f3));
      SG_TRY(capture_twolevel<T>(c, vbuf, zbuf, f3, S.s[4], S.s[5]));
      SG_TRY(dg_store_j<T>(zbuf, Zs, len, len, c.fdg, f3));
      SG_TRY(c.apply_raw_fine(zbuf, w, nullptr, f3));
      SG_TRY(dg_mdot<T>(V, len, w, len, h1, part, cnt, jdev, m, f3));
      if (W.passes == 1) {
        SG_TRY(dg_axpy_norm<T>(V, len, h1, w, len, W.s.scal, part, cnt, jdev, f3));
      } else {
        SG_TRY(dg_axpy_norm<T>(V, len, h1, w, len, nullptr, part, cnt, jdev, f3));
        SG_TRY(dg_mdot<T>(V, len, w, len, h2, part, cnt, jdev, m, f3));
        SG_TRY(dg_axpy_norm<T>(V, len, h2, w, len, W.s.scal, part, cnt, jdev, f3));
      }
      SG_TRY(dg_givens(c.fdg, W.s, m, hin, f3));
      SG_TRY(dg_scale_next<T>(w, V, len, len, c.fdg, W.s.scal + 1, f3));
      SG_CUDA(cudaStreamEndCapture(f3, &body_in));
    }
    k3 = launch_count();
    // x += Z y
    SG_TRY(dg_backsolve(c.fdg, W.s, m, f2));
    SG_TRY(dg_axpy_multi<T>(Zs, len, W.s.y, x, len, jdev, f2));
    SG_TRY(dg_end(c.fdg, W.s, hout, f2, trust));
    SG_CUDA(cudaStreamEndCapture(f2, &body_out));
  }
  const int64_t k4 = launch_count();
  c.cc_fine = RegionCounts{k1 - k0, (k2 - k1) + (k4 - k3), k3 - k2};
  note_launches(-(k4 - k0));  // recorded, not launched
  return SG_OK;
}

// Everything one system needs for a recorded solve.
struct GraphSystem {
  sg_problem* pr = nullptr;
  uint64_t serial = 0;
  uint64_t ctx_gen = 0;         // generation of the workspaces the graph was recorded with
  const void* ctx64 = nullptr;
  const void* ctx32 = nullptr;
  RegionCounts ir;              // refinement loop: fixed, -, per step
  CapStreams streams;
};

static sg_status capture_system_nodes(GraphSystem& gs, const sg_solve_opts& o, cudaStream_t top);

// Records the solve of one system on `top` (already capturing):
// mode 1: x64 += corrections of FP32 FGMRES solves of the normalised FP64
//         residual, until relres <= rtol (refinement loop as a WHILE node);
// mode 0: FP64 FGMRES on F64 from x64.
static sg_status capture_system(GraphSystem& gs, const sg_solve_opts& o, cudaStream_t top) {
  const int64_t k0 = launch_count();
  const sg_status s = capture_system_nodes(gs, o, top);
  note_launches(-(launch_count() - k0));  // recorded, not launched
  return s;
}

static sg_status capture_system_nodes(GraphSystem& gs, const sg_solve_opts& o, cudaStream_t top) {
  sg_problem* pr = gs.pr;
  SolverState& S = *pr->solver;
  const int64_t len = int64_t(pr->P) * pr->ld;
  SolverCtx<double>* c64 = nullptr;
  SG_TRY(get_ctx<double>(pr, c64));
  double* x64 = dp<double>(S.x64);
  double* F64 = dp<double>(S.io);
  double* ird = dp<double>(S.ir_d);  // [0] rr, [1] ||F||^2
  int* iri = dp<int>(S.ir_i);        // [0] refinement steps, [1] non-finite flag
  ProfilerOff off(pr->prof);
  if (o.mode == 0) {
    SG_TRY(vec_norm2<double>(F64, len, ird + 1, dp<double>(c64->fine.partial), dp<unsigned>(c64->fine.counter), top));
    gs.ir = RegionCounts{1, 0, 0};
    return capture_fine<double>(*c64, F64, x64, o.rtol, false, gs.streams, top);
  }
  SolverCtx<float>* c32 = nullptr;
  SG_TRY(get_ctx<float>(pr, c32));
  float* r32 = dp<float>(S.r32);
  float* d32 = dp<float>(S.d32);
  double* r64 = dp<double>(S.r64);
  double* part = dp<double>(c64->fine.partial);
  unsigned* cnt = dp<unsigned>(c64->fine.counter);
  const double inner = o.inner_rtol > 0 ? o.inner_rtol : 3e-4;  // the host-driven refinement's default
  const int max_ir = o.max_ir > 0 ? o.max_ir : 20;
  const cudaStream_t i2 = gs.streams.s[1];
  const int64_t k0 = launch_count();
  SG_TRY(vec_norm2<double>(F64, len, ird + 1, part, cnt, top));
  SG_TRY(refine_residual(pr, F64, pr->ld, x64, pr->ld, r64, pr->ld, top));
  SG_TRY(vec_norm2<double>(r64, len, ird, part, cnt, top));
  cudaGraphConditionalHandle hir;
  cudaStreamCaptureStatus cs;
  cudaGraph_t g;
  SG_CUDA(cudaStreamGetCaptureInfo(top, &cs, nullptr, &g, nullptr, nullptr, nullptr));
  SG_CUDA(cudaGraphConditionalHandleCreate(&hir, g, 0, 0));
  SG_TRY(ir_decide(ird, ird + 1, iri, o.rtol, max_ir, c32->fdg.iv + 4, o.max_it, hir, top));
  const int64_t k1 = launch_count();
  cudaGraph_t body;
  SG_TRY(SolverCtx<float>::add_while(top, hir, &body));
  SG_CUDA(cudaStreamBeginCaptureToGraph(i2, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  SG_TRY((vec_convert<double, float>(r64, r32, len, nullptr, ird, i2)));
  SG_CUDA(cudaMemsetAsync(d32, 0, len * 4, i2));
  // the FP32 correction stops at the reduction left to the target when
  // that is looser than `inner` (the host-driven refinement's rule)
  SG_TRY(capture_fine<float>(*c32, r32, d32, inner, true, gs.streams, i2, ird, ird + 1, o.rtol));
  SG_TRY(vec_add_scaled_f32(x64, d32, len, ird, i2));
  SG_TRY(refine_residual(pr, F64, pr->ld, x64, pr->ld, r64, pr->ld, i2));
  SG_TRY(vec_norm2<double>(r64, len, ird, part, cnt, i2));
  SG_TRY(ir_decide(ird, ird + 1, iri, o.rtol, max_ir, c32->fdg.iv + 4, o.max_it, hir, i2));
  SG_CUDA(cudaStreamEndCapture(i2, &body));
  gs.ir = RegionCounts{k1 - k0, 0, launch_count() - k1};
  return SG_OK;
}

// buffers and contexts of one system, created before any capture
static sg_status prepare_system(GraphSystem& gs, const sg_solve_opts& o) {
  sg_problem* pr = gs.pr;
  SolverState& S = *pr->solver;
  S.restart = o.restart > 0 ? std::min(o.restart, 31) : 30;
  const int64_t len = int64_t(pr->P) * pr->ld;
  for (DevBuf* b : {&S.x64, &S.r64, &S.io}) {
    if (!b->ptr) SG_TRY(b->alloc(len * 8));
  }
  for (DevBuf* b : {&S.r32, &S.d32}) {
    if (!b->ptr) SG_TRY(b->alloc(len * 4));
  }
  if (!S.ir_d.ptr) SG_TRY(S.ir_d.alloc(8 * 8));
  if (!S.ir_i.ptr) SG_TRY(S.ir_i.alloc(8 * 4));
  SolverCtx<double>* c64 = nullptr;
  SG_TRY(get_ctx<double>(pr, c64));
  SG_TRY(c64->capture_prepare());
  SolverCtx<float>* c32 = nullptr;
  SG_TRY(get_ctx<float>(pr, c32));
  SG_TRY(c32->capture_prepare());
  c64->fine.passes = fine_orth_passes(o);
  c32->fine.passes = fine_orth_passes(o);
  // iteration caps of the device-driven loops
  const int cap_fine = o.max_it;
  SG_CUDA(cudaMemcpy(c64->fdg.iv + 2, &cap_fine, sizeof(int), cudaMemcpyHostToDevice));
  SG_CUDA(cudaMemcpy(c32->fdg.iv + 2, &cap_fine, sizeof(int), cudaMemcpyHostToDevice));
  // the recorded smoother is the one selected now
  S.pc.use_cnn = S.pc.smoother == 1 && pr->cnn && pr->cnn->trained;
  S.pc.harvest.on = false;
  gs.serial = S.serial;
  gs.ctx_gen = S.ctx_gen;
  gs.ctx64 = c64;
  gs.ctx32 = c32;
  return gs.streams.create();
}

}  // namespace sg

using namespace sg;

struct sg_batch {
  std::vector<GraphSystem> sys;
  sg_solve_opts opts{};
  cudaGraphExec_t exec = nullptr;
  cudaStream_t origin = nullptr;
  std::vector<cudaEvent_t> events;
  ~sg_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    for (auto e : events) cudaEventDestroy(e);
    if (origin) cudaStreamDestroy(origin);
    for (auto& g : sys)
      if (g.pr && g.pr->solver && g.pr->solver->serial == g.serial) g.pr->solver->pc.use_cnn = false;
  }
};

static sg_status batch_build(sg_batch* B) {
  SG_CUDA(cudaStreamCreateWithFlags(&B->origin, cudaStreamNonBlocking));
  const size_t n = B->sys.size();
  B->events.assign(n + 1, nullptr);
  for (auto& e : B->events) SG_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  cudaGraph_t g = nullptr;
  SG_CUDA(cudaStreamBeginCapture(B->origin, cudaStreamCaptureModeRelaxed));
  sg_status s = SG_OK;
  cudaError_t e = cudaEventRecord(B->events[n], B->origin);
  for (size_t i = 0; i < n && s == SG_OK && e == cudaSuccess; ++i) {
    cudaStream_t top = B->sys[i].streams.s[0];
    e = cudaStreamWaitEvent(top, B->events[n], 0);
    if (e != cudaSuccess) break;
    s = capture_system(B->sys[i], B->opts, top);
    if (s != SG_OK) break;
    e = cudaEventRecord(B->events[i], top);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(B->origin, B->events[i], 0);
  }
  const cudaError_t e2 = cudaStreamEndCapture(B->origin, &g);
  if (s != SG_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  SG_CUDA(e);
  SG_CUDA(e2);
  const cudaError_t e3 = cudaGraphInstantiate(&B->exec, g, 0);
  cudaGraphDestroy(g);
  SG_CUDA(e3);
  return SG_OK;
}

extern "C" {

sg_status sg_batch_create(sg_problem* const* probs, int count, const sg_solve_opts* o, sg_batch** out) {
  SG_ARG(probs && o && out && count >= 1 && count <= 256, "sg_batch_create: need 1..256 problems and options");
  SG_ARG(o->rtol > 0 && o->max_it > 0, "sg_batch_create: rtol and max_it must be > 0");
  SG_ARG(o->mode == 0 || o->mode == 1, "sg_batch_create: mode must be 0 or 1");
  SG_ARG(o->orth_passes >= 0 && o->orth_passes <= 2, "sg_batch_create: orth_passes must be 0, 1 or 2");
  for (int i = 0; i < count; ++i) {
    SG_ARG(probs[i] && probs[i]->solver && probs[i]->solver->pc.ready,
           "sg_batch_create: every problem needs sg_precond_setup");
    for (int j = 0; j < i; ++j) SG_ARG(probs[i] != probs[j], "sg_batch_create: a problem appears twice");
  }
  *out = nullptr;
  sg_batch* B = new sg_batch();
  B->opts = *o;
  B->opts.hist_host = nullptr;
  B->opts.hist_cap = 0;
  B->sys.resize(count);
  sg_status s = SG_OK;
  for (int i = 0; i < count && s == SG_OK; ++i) {
    B->sys[i].pr = probs[i];
    s = prepare_system(B->sys[i], B->opts);
  }
  if (s == SG_OK) s = batch_build(B);
  if (s != SG_OK) {
    delete B;
    return s;
  }
  *out = B;
  return SG_OK;
}

sg_status sg_batch_destroy(sg_batch* B) {
  delete B;
  return SG_OK;
}

sg_status sg_batch_solve(sg_batch* B, const double* const* F, const int64_t* ldf, double* const* X,
                         const int64_t* ldx, sg_solve_info* infos, void* stream) {
  SG_ARG(B && B->exec && X && ldx, "sg_batch_solve: NULL argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t n = B->sys.size();
  auto t0 = std::chrono::steady_clock::now();
  for (size_t i = 0; i < n; ++i) {
    sg_problem* pr = B->sys[i].pr;
    SG_ARG(pr->solver && pr->solver->serial == B->sys[i].serial && pr->solver->ctx_gen == B->sys[i].ctx_gen &&
               pr->solver->c64.get() == B->sys[i].ctx64 && pr->solver->c32.get() == B->sys[i].ctx32,
           "sg_batch_solve: a problem's preconditioner or solver workspace changed after sg_batch_create");
    SG_ARG(X[i] && ldx[i] >= pr->n && (!F || !F[i] || (ldf && ldf[i] >= pr->n)),
           "sg_batch_solve: bad block or leading dimension");
  }
  // inputs into the recorded buffers, counters cleared
  for (size_t i = 0; i < n; ++i) {
    sg_problem* pr = B->sys[i].pr;
    SolverState& S = *pr->solver;
    const int P = pr->P;
    const int64_t ld = pr->ld, len = int64_t(P) * ld;
    if (S.dirty) {
      SG_TRY(S.c64->scrub(st));
      SG_TRY(S.c32->scrub(st));
      S.dirty = false;
    }
    double* F64 = dp<double>(S.io);
    double* x64 = dp<double>(S.x64);
    SG_CUDA(cudaMemsetAsync(F64, 0, len * 8, st));
    SG_CUDA(cudaMemsetAsync(x64, 0, len * 8, st));
    if (F && F[i])
      SG_CUDA(cudaMemcpy2DAsync(F64, ld * 8, F[i], ldf[i] * 8, pr->n * 8, P, cudaMemcpyDeviceToDevice, st));
    else
      SG_CUDA(cudaMemcpyAsync(F64, pr->b.data(), pr->n * 8, cudaMemcpyHostToDevice, st));
    SG_CUDA(cudaMemcpy2DAsync(x64, ld * 8, X[i], ldx[i] * 8, pr->n * 8, P, cudaMemcpyDeviceToDevice, st));
    SG_CUDA(cudaMemsetAsync(S.ir_i.ptr, 0, S.ir_i.bytes, st));
    SG_TRY(S.c64->clear_counters(st));
    SG_TRY(S.c32->clear_counters(st));
  }
  SG_CUDA(cudaGraphLaunch(B->exec, st));
  // results out, the true FP64 residual of each returned iterate
  sg_status worst = SG_OK;
  for (size_t i = 0; i < n; ++i) {
    sg_problem* pr = B->sys[i].pr;
    SolverState& S = *pr->solver;
    const int P = pr->P;
    const int64_t ld = pr->ld, len = int64_t(P) * ld;
    double* x64 = dp<double>(S.x64);
    double* F64 = dp<double>(S.io);
    double* ird = dp<double>(S.ir_d);
    SolverCtx<double>* c64 = S.c64.get();
    if (B->opts.mode == 1)
      SG_TRY(refine_residual(pr, F64, ld, x64, ld, dp<double>(S.r64), ld, st));
    else
      SG_TRY(apply_op<double>(pr, false, x64, ld, F64, ld, dp<double>(S.r64), ld, st));
    SG_TRY(vec_norm2<double>(dp<double>(S.r64), len, ird + 2, dp<double>(c64->fine.partial),
                             dp<unsigned>(c64->fine.counter), st));
    SG_TRY(vec_norm2<double>(F64, len, ird + 3, dp<double>(c64->fine.partial), dp<unsigned>(c64->fine.counter), st));
    SG_CUDA(cudaMemcpy2DAsync(X[i], ldx[i] * 8, x64, ld * 8, pr->n * 8, P, cudaMemcpyDeviceToDevice, st));
  }
  SG_CUDA(cudaStreamSynchronize(st));
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (size_t i = 0; i < n; ++i) {
    sg_problem* pr = B->sys[i].pr;
    SolverState& S = *pr->solver;
    double d[4];
    int iv[8];
    SG_CUDA(cudaMemcpy(d, S.ir_d.ptr, sizeof d, cudaMemcpyDeviceToHost));
    SG_CUDA(cudaMemcpy(iv, S.ir_i.ptr, sizeof iv, cudaMemcpyDeviceToHost));
    int fits = 0, cits = 0, fr = 0, cr = 0;
    const bool m1 = B->opts.mode == 1;
    const RegionCounts& cf = m1 ? S.c32->cc_fine : S.c64->cc_fine;
    const RegionCounts& cc = m1 ? S.c32->cc_coarse : S.c64->cc_coarse;
    if (m1)
      SG_TRY(S.c32->read_counters(&fits, &cits, &fr, &cr));
    else
      SG_TRY(S.c64->read_counters(&fits, &cits, &fr, &cr));
    // kernels the graph ran for this system: refinement steps, FGMRES
    // solves (one per step), two-level cycles with their coarse solves (one
    // per FGMRES iteration)
    const int64_t steps = m1 ? iv[0] : 0, fine_calls = m1 ? steps : 1;
    note_launches(B->sys[i].ir.total(1, 0, steps) + cf.total(fine_calls, fr, fits) + cc.total(fits, cr, cits));
    sg_solve_info inf{};
    inf.outer_it = fits;
    inf.inner_it = cits;
    inf.ir_steps = B->opts.mode == 1 ? iv[0] : 0;
    inf.relres = d[3] > 0 ? std::sqrt(d[2] / d[3]) : 0.0;
    inf.t_solve = secs;
    if (infos) infos[i] = inf;
    if (!std::isfinite(inf.relres)) {
      S.dirty = true;
      worst = SG_ERR_BREAKDOWN;
    } else if (inf.relres > B->opts.rtol && worst == SG_OK) {
      worst = SG_NOT_CONVERGED;
    }
  }
  if (worst == SG_ERR_BREAKDOWN) set_error("sg_batch_solve: non-finite residual in a system");
  if (worst == SG_NOT_CONVERGED) set_error("sg_batch_solve: a system reached max_it before rtol");
  return worst;
}

sg_status sg_solve_batch(sg_problem* const* probs, int count, const double* const* F, const int64_t* ldf,
                         double* const* X, const int64_t* ldx, const sg_solve_opts* o, sg_solve_info* infos,
                         void* stream) {
  sg_batch* B = nullptr;
  SG_TRY(sg_batch_create(probs, count, o, &B));
  const sg_status s = sg_batch_solve(B, F, ldf, X, ldx, infos, stream);
  sg_batch_destroy(B);
  return s;
}

}  // extern "C"

namespace sg {
template sg_status capture_coarse<float>(SolverCtx<float>&, cudaStream_t, cudaStream_t, cudaStream_t);
template sg_status capture_coarse<double>(SolverCtx<double>&, cudaStream_t, cudaStream_t, cudaStream_t);
}  // namespace sg
