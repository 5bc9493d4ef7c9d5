// C ABI of the learned smoother: network weights, inference, one training
// step, the batched mean solves that give the training targets, and the
// training driver that harvests residuals from the method's own solves.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>

#include "sg_cnn.h"
#include "sg_train.h"

using namespace sg;

namespace {

// network on the (N-1) x (N-1) interior grid; channel 1 of its input is
// log(a_rr / 4) with a_rr the diagonal of A_0
sg_status ensure_cnn(sg_problem* pr) {
  if (pr->cnn) return SG_OK;
  const int m = pr->N - 1;
  if (int64_t(m) * m != pr->n) {
    set_error("learned smoother: the node set is not an (N-1) x (N-1) grid");
    return SG_ERR_UNSUPPORTED;
  }
  std::vector<double> logd(pr->n, 0.0);
  for (int64_t r = 0; r < pr->n; ++r)
    for (int32_t t = pr->rowptr[r]; t < pr->rowptr[r + 1]; ++t)
      if (pr->colidx[t] == r) logd[r] = std::log(pr->a0[t] / 4.0);
  Cnn* c = new Cnn();
  sg_status s = c->init(logd, m, m, pr->rowptr, pr->colidx, pr->a0);
  if (s != SG_OK) {
    delete c;
    return s;
  }
  c->wait_limit = pr->wait_limit;
  pr->cnn = c;
  return SG_OK;
}

uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Fisher-Yates permutation of 0..n-1 from a splitmix64 stream
std::vector<int64_t> permutation(int64_t n, uint64_t seed) {
  std::vector<int64_t> p(n);
  std::iota(p.begin(), p.end(), 0);
  uint64_t s = seed;
  for (int64_t i = n - 1; i > 0; --i) std::swap(p[i], p[int64_t(splitmix(s) % uint64_t(i + 1))]);
  return p;
}

double seconds_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

extern "C" {

int64_t sg_cnn_param_count(void) { return cnn_param_count(); }

sg_status sg_cnn_init(sg_problem* pr, uint64_t seed, void* stream) {
  SG_ARG(pr, "sg_cnn_init: NULL handle");
  SG_TRY(ensure_cnn(pr));
  std::vector<float> w = cnn_he_init(seed);
  SG_TRY(pr->cnn->set_weights(w.data(), static_cast<cudaStream_t>(stream)));
  SG_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  return SG_OK;
}

sg_status sg_cnn_set_weights(sg_problem* pr, const float* w, int64_t count, void* stream) {
  SG_ARG(pr && w, "sg_cnn_set_weights: NULL argument");
  SG_ARG(count == cnn_param_count(), "sg_cnn_set_weights: count must be sg_cnn_param_count()");
  SG_TRY(ensure_cnn(pr));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SG_TRY(pr->cnn->set_weights(w, st));
  SG_CUDA(cudaStreamSynchronize(st));
  return SG_OK;
}

sg_status sg_cnn_get_weights(sg_problem* pr, float* w, int64_t count, int what, void* stream) {
  SG_ARG(pr && w, "sg_cnn_get_weights: NULL argument");
  SG_ARG(count == cnn_param_count(), "sg_cnn_get_weights: count must be sg_cnn_param_count()");
  SG_ARG(what == 0 || what == 1, "sg_cnn_get_weights: what must be 0 (weights) or 1 (gradient)");
  SG_ARG(pr->cnn && pr->cnn->trained, "sg_cnn_get_weights: no weights set");
  return pr->cnn->get_weights(w, what == 1, static_cast<cudaStream_t>(stream));
}

sg_status sg_cnn_apply(sg_problem* pr, const float* R, int64_t ldr, float* Z, int64_t ldz, int nimg, void* stream) {
  SG_ARG(pr && (nimg == 0 || (R && Z)), "sg_cnn_apply: NULL argument");
  SG_ARG(pr->cnn && pr->cnn->trained, "sg_cnn_apply: no weights set");
  SG_ARG(nimg >= 0 && nimg <= 65535, "sg_cnn_apply: nimg must be in [0, 65535]");
  SG_ARG(ldr >= pr->n && ldz >= pr->n, "sg_cnn_apply: leading dimension < n");
  if (nimg == 0) return SG_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Cnn& c = *pr->cnn;
  SG_TRY(c.reserve(nimg));
  SG_TRY(c.pack_input<float>(R, ldr, nimg, st));
  SG_TRY(c.forward(nimg, st));
  SG_TRY(c.unpack_output<float>(Z, ldz, nimg, st));
  if (c.use_tc) {  // a tensor-core wait that ran out is reported here
    int e = 0;
    SG_CUDA(cudaMemcpyAsync(&e, c.tcerr.ptr, sizeof e, cudaMemcpyDeviceToHost, st));
    SG_CUDA(cudaStreamSynchronize(st));
    if (e) {
      SG_CUDA(cudaMemsetAsync(c.tcerr.ptr, 0, sizeof e, st));
      set_error("sg_cnn_apply: a tensor-core completion wait timed out");
      return SG_ERR_TIMEOUT;
    }
  }
  return SG_OK;
}

sg_status sg_set_wait_limit(sg_problem* pr, int limit) {
  SG_ARG(pr, "sg_set_wait_limit: NULL handle");
  pr->wait_limit = limit < 0 ? kTcWaitDefault : limit;
  if (pr->cnn) pr->cnn->wait_limit = pr->wait_limit;
  if (pr->solver) precond_of(pr).wait_limit = pr->wait_limit;
  return SG_OK;
}

sg_status sg_cnn_set_kernel(sg_problem* pr, int kind) {
  SG_ARG(pr, "sg_cnn_set_kernel: NULL handle");
  SG_ARG(kind == 0 || kind == 1, "sg_cnn_set_kernel: kind must be 0 (mma.sync) or 1 (tcgen05)");
  SG_TRY(ensure_cnn(pr));
  pr->cnn->use_tc = kind == 1;
  return SG_OK;
}

sg_status sg_cnn_train_step(sg_problem* pr, const float* R, int64_t ldr, const float* Zs, int64_t ldz, int nimg,
                            float lr, int update, double* loss, void* stream) {
  SG_ARG(pr && R && Zs, "sg_cnn_train_step: NULL argument");
  SG_ARG(pr->cnn && pr->cnn->trained, "sg_cnn_train_step: no weights set");
  SG_ARG(nimg >= 1 && nimg <= 65535, "sg_cnn_train_step: nimg must be in [1, 65535]");
  SG_ARG(ldr >= pr->n && ldz >= pr->n, "sg_cnn_train_step: leading dimension < n");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Cnn& c = *pr->cnn;
  SG_TRY(c.reserve(nimg));
  SG_TRY(c.pack_input<float>(R, ldr, nimg, st));
  SG_TRY(c.scale_targets(Zs, ldz, nimg, st));
  SG_TRY(c.forward(nimg, st));
  SG_TRY(c.loss_and_grad(nimg, loss, st));
  SG_TRY(c.backward(nimg, st));
  if (update) SG_TRY(c.adam(lr, st));
  return SG_OK;
}

sg_status sg_cnn_set_loss(sg_problem* pr, int kind) {
  SG_ARG(pr, "sg_cnn_set_loss: NULL handle");
  SG_ARG(kind == 0 || kind == 1, "sg_cnn_set_loss: kind must be 0 (energy norm) or 1 (relative L2)");
  SG_TRY(ensure_cnn(pr));
  pr->cnn->loss_kind = kind;
  return SG_OK;
}

sg_status sg_mean_solve(sg_problem* pr, const float* B, int64_t ldb, float* Z, int64_t ldz, int nb, double rtol,
                        int max_it, double* relres_max, int* its, void* stream) {
  SG_ARG(pr && B && Z, "sg_mean_solve: NULL argument");
  SG_ARG(nb >= 1 && nb <= 65535, "sg_mean_solve: nb must be in [1, 65535]");
  SG_ARG(ldb >= pr->n && ldz >= pr->n, "sg_mean_solve: leading dimension < n");
  SG_ARG(rtol > 0 && max_it > 0, "sg_mean_solve: rtol and max_it must be > 0");
  SG_TRY(ensure_cnn(pr));
  if (!pr->cnn->mean) pr->cnn->mean = new MeanSolver();
  SG_TRY(pr->cnn->mean->init(pr, nb));
  return pr->cnn->mean->solve(B, ldb, Z, ldz, nb, rtol, max_it, relres_max, its, static_cast<cudaStream_t>(stream));
}

sg_status sg_precond_set_smoother(sg_problem* pr, int smoother, double omega, void* stream) {
  SG_ARG(pr && pr->solver, "sg_precond_set_smoother: call sg_precond_setup first");
  SG_ARG(smoother == 0 || smoother == 1, "sg_precond_set_smoother: smoother must be 0 (RAS) or 1 (learned)");
  Precond& pc = precond_of(pr);
  if (smoother == 0) {
    pc.smoother = 0;
    return SG_OK;
  }
  SG_ARG(pr->cnn && pr->cnn->trained, "sg_precond_set_smoother: the learned smoother has no weights");
  return learned_smoother_enable(pr, omega, static_cast<cudaStream_t>(stream));
}

// Saved learned smoother: a fixed header, then the flat FP32 weights in the
// order of sg_cnn_set_weights.
namespace {
struct SavedSmoother {
  char magic[8];      // "SGLSMTH" + NUL
  int32_t version;    // 1
  int32_t nparam;     // sg_cnn_param_count()
  double omega_cnn;   // damping of the learned smoother, 0 = not known
  int32_t selected;   // 1: the learned smoother was the selected one
  int32_t reserved;
};
constexpr char kSavedMagic[8] = {'S', 'G', 'L', 'S', 'M', 'T', 'H', '\0'};
}  // namespace

sg_status sg_precond_save(const sg_problem* pr, void* buf, int64_t* bytes) {
  SG_ARG(pr && bytes, "sg_precond_save: NULL argument");
  SG_ARG(pr->cnn && pr->cnn->trained, "sg_precond_save: the learned smoother has no weights");
  const int64_t np = cnn_param_count();
  const int64_t need = int64_t(sizeof(SavedSmoother)) + np * int64_t(sizeof(float));
  if (!buf) {
    *bytes = need;
    return SG_OK;
  }
  SG_ARG(*bytes >= need, "sg_precond_save: buffer smaller than the size asked with buf = NULL");
  SavedSmoother h{};
  std::memcpy(h.magic, kSavedMagic, sizeof h.magic);
  h.version = 1;
  h.nparam = int32_t(np);
  const Precond* pc = pr->solver ? &precond_of(const_cast<sg_problem*>(pr)) : nullptr;
  h.omega_cnn = pc ? pc->omega_cnn : 0.0;
  h.selected = pc && pc->smoother == 1 ? 1 : 0;
  if (!h.selected) h.omega_cnn = 0.0;
  std::vector<float> w(np);
  SG_TRY(pr->cnn->get_weights(w.data(), false, nullptr));
  std::memcpy(buf, &h, sizeof h);
  std::memcpy(static_cast<char*>(buf) + sizeof h, w.data(), np * sizeof(float));
  *bytes = need;
  return SG_OK;
}

sg_status sg_precond_load(sg_problem* pr, const void* buf, int64_t bytes) {
  SG_ARG(pr && buf, "sg_precond_load: NULL argument");
  SG_ARG(bytes >= int64_t(sizeof(SavedSmoother)), "sg_precond_load: buffer shorter than the header");
  SavedSmoother h;
  std::memcpy(&h, buf, sizeof h);
  SG_ARG(std::memcmp(h.magic, kSavedMagic, sizeof h.magic) == 0 && h.version == 1,
         "sg_precond_load: not a saved learned smoother (magic or version)");
  const int64_t np = cnn_param_count();
  SG_ARG(h.nparam == np && bytes >= int64_t(sizeof h) + np * int64_t(sizeof(float)),
         "sg_precond_load: parameter count or size does not match this build's network");
  SG_ARG(!(h.omega_cnn < 0.0) && std::isfinite(h.omega_cnn), "sg_precond_load: bad damping");
  std::vector<float> w(np);
  std::memcpy(w.data(), static_cast<const char*>(buf) + sizeof h, np * sizeof(float));
  SG_TRY(sg_cnn_set_weights(pr, w.data(), np, nullptr));
  // with a preconditioner set up, the saved selection and damping return
  if (h.selected && pr->solver && precond_of(pr).ready) return sg_precond_set_smoother(pr, 1, h.omega_cnn, nullptr);
  return SG_OK;
}

sg_status sg_train_precond(sg_problem* pr, const sg_train_opts* o, sg_train_info* info, void* stream) {
  SG_ARG(pr && o, "sg_train_precond: NULL argument");
  SG_ARG(pr->solver, "sg_train_precond: call sg_precond_setup first");
  SG_ARG(o->n_pairs >= 1 && o->epochs >= 0 && o->batch >= 1 && o->batch <= o->n_pairs,
         "sg_train_precond: need n_pairs >= 1, epochs >= 0, 1 <= batch <= n_pairs");
  SG_ARG(o->lr > 0, "sg_train_precond: lr must be > 0");
  SG_ARG(o->loss == 0 || o->loss == 1, "sg_train_precond: loss must be 0 (energy norm) or 1 (relative L2)");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Precond& pc = precond_of(pr);
  const int P = pr->P;
  const int64_t ld = pr->ld, n = pr->n, len = int64_t(P) * ld;
  sg_train_info inf{};
  SG_TRY(ensure_cnn(pr));
  Cnn& cnn = *pr->cnn;
  if (!cnn.trained || !o->keep_weights) {
    std::vector<float> w = cnn_he_init(o->seed);
    SG_TRY(cnn.set_weights(w.data(), st));
  }
  const int prev_smoother = pc.smoother;
  pc.smoother = 0;
  cnn.loss_kind = o->loss;

  // 1. harvest smoother inputs of plain mixed-precision solves: first with
  //    the problem's load vector, then with seeded Gaussian right-hand sides
  auto t0 = std::chrono::steady_clock::now();
  const int64_t want_images = (3 * int64_t(o->n_pairs) + 1) / 2;
  Harvest& hv = pc.harvest;
  hv.cap = (want_images + P - 1) / P;
  SG_TRY(hv.pool.alloc(size_t(hv.cap) * len * 4));
  hv.count = 0;
  {
    DevBuf X, F;
    SG_TRY(X.alloc(len * 8));
    SG_TRY(F.alloc(len * 8));
    std::vector<double> hF(len, 0.0);
    uint64_t rs = o->seed ^ 0x5eed5eed5eedULL;
    const double scale = *std::max_element(pr->b.begin(), pr->b.end());
    sg_solve_opts so{};
    so.rtol = 1e-8;
    so.max_it = 400;
    so.mode = 1;
    for (int solve = 0; hv.count < hv.cap && solve < 64; ++solve) {
      hv.on = true;
      SG_CUDA(cudaMemsetAsync(X.ptr, 0, len * 8, st));
      const double* Fp = nullptr;
      if (solve > 0) {
        for (int a = 0; a < P; ++a)
          for (int64_t r = 0; r < n; ++r) {
            const double u1 = (double(splitmix(rs) >> 11) + 0.5) / 9007199254740992.0;
            const double u2 = (double(splitmix(rs) >> 11) + 0.5) / 9007199254740992.0;
            hF[size_t(a) * ld + r] = scale * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
          }
        SG_CUDA(cudaMemcpyAsync(F.ptr, hF.data(), len * 8, cudaMemcpyHostToDevice, st));
        Fp = dp<double>(F);
      }
      sg_solve_info si{};
      sg_status s = sg_solve(pr, Fp, ld, dp<double>(X), ld, &so, &si, st);
      hv.on = false;
      if (s != SG_OK && s != SG_NOT_CONVERGED) return s;
      inf.harvest_solves++;
    }
  }
  hv.on = false;
  const int64_t pool_images = hv.count * P;
  const int np = int(std::min<int64_t>(o->n_pairs, pool_images));
  SG_ARG(np >= o->batch, "sg_train_precond: harvest produced fewer images than one batch");
  inf.n_pairs = np;
  // uniform sample over (smoother call, mode) without replacement
  std::vector<int64_t> pick = permutation(pool_images, o->seed + 1);
  pick.resize(np);
  DevBuf Rt, Zt;
  SG_TRY(Rt.alloc(size_t(np) * ld * 4));
  SG_TRY(Zt.alloc(size_t(np) * ld * 4));
  for (int i = 0; i < np; ++i)
    SG_CUDA(cudaMemcpyAsync(dp<float>(Rt) + size_t(i) * ld, dp<float>(hv.pool) + pick[i] * ld, n * 4,
                            cudaMemcpyDeviceToDevice, st));
  hv.pool.free_();
  hv.cap = hv.count = 0;
  SG_CUDA(cudaStreamSynchronize(st));
  inf.t_harvest = seconds_since(t0);

  // 2. targets z* = A_0^{-1} r by batched AMG-preconditioned CG
  t0 = std::chrono::steady_clock::now();
  const int chunk = int(std::min<int64_t>(np, std::max<int64_t>(1, (int64_t(1) << 32) / (ld * 8 * 8))));
  if (!cnn.mean) cnn.mean = new MeanSolver();
  SG_TRY(cnn.mean->init(pr, chunk));
  const double trtol = o->target_rtol > 0 ? o->target_rtol : 1e-6;
  for (int i0 = 0; i0 < np; i0 += chunk) {
    const int cols = std::min(chunk, np - i0);
    double rel = 0.0;
    int its = 0;
    SG_TRY(cnn.mean->solve(dp<float>(Rt) + size_t(i0) * ld, ld, dp<float>(Zt) + size_t(i0) * ld, ld, cols, trtol, 500,
                           &rel, &its, st));
    inf.target_relres = std::max(inf.target_relres, rel);
    inf.target_its = std::max(inf.target_its, its);
  }
  SG_CUDA(cudaStreamSynchronize(st));
  inf.t_targets = seconds_since(t0);

  // 3. Adam on batches of consecutive (already shuffled) pairs, the batch
  //    order reshuffled every epoch
  t0 = std::chrono::steady_clock::now();
  const int nbatch = np / o->batch;
  SG_TRY(cnn.reserve(o->batch));
  for (int ep = 0; ep < o->epochs; ++ep) {
    std::vector<int64_t> order = permutation(nbatch, o->seed + 2 + uint64_t(ep));
    for (int bi = 0; bi < nbatch; ++bi) {
      const size_t off = size_t(order[bi]) * o->batch * ld;
      const bool first = ep == 0 && bi == 0, last = ep == o->epochs - 1 && bi == nbatch - 1;
      double L = 0.0;
      SG_TRY(sg_cnn_train_step(pr, dp<float>(Rt) + off, ld, dp<float>(Zt) + off, ld, o->batch, o->lr, 1,
                               (first || last) ? &L : nullptr, st));
      if (first) inf.loss_first = L / o->batch;
      if (last) inf.loss_last = L / o->batch;
      inf.steps++;
    }
  }
  SG_CUDA(cudaStreamSynchronize(st));
  inf.t_train = seconds_since(t0);
  if (!std::isfinite(inf.loss_last)) {
    pc.smoother = prev_smoother;
    set_error("sg_train_precond: non-finite training loss");
    return SG_ERR_BREAKDOWN;
  }
  SG_TRY(learned_smoother_enable(pr, 0.0, st));
  inf.omega_cnn = pc.omega_cnn;
  if (info) *info = inf;
  return SG_OK;
}

}  // extern "C"
