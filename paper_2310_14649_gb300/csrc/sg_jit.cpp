// Register-specialised Galerkin apply (Sec. 2.1, Eq. Galerkin_L_exp):
//     y_r[a] = sum_s sum_{(k,a,b)} v_k^{r,s} g_kab x_{col(r,s)}[b].
//
// The triple list depends only on (L, p, q), so at setup the library writes
// a CUDA kernel in which every nonzero g_kab is an immediate operand and
// every accumulator y[a] and gathered value x[b] lives in a named register.
// Per stencil slot a thread gathers the P values of its rows' neighbours,
// then streams the K matrix values of that slot (coalesced across the warp:
// lanes hold consecutive rows) and, for each input term k, updates the
// outputs coupled to it:  y_a += v_k * (sum_b g_kab x_b).
//
// Tile shape (chosen by the autotuner, cached per problem shape):
//   R  rows per thread: 1, or 2 adjacent rows packed in float2 registers
//      and updated with the paired FP32 FMA of sm_100+ (one instruction for
//      two rows; matrix values loaded as 8-byte pairs);
//   H  output groups: the P outputs are split into H contiguous ranges of
//      about T/H triples each, one range per group of 4 warps, so the
//      registers per thread stay bounded for large P;
//   pf input terms whose values are loaded ahead of use;
//   mb CTAs per SM requested from the register allocator.
// Kernels are compiled for sm_103a with NVRTC and cached on disk by a hash
// of their source.  The same kernel serves the fine (5 slots) and the
// coarse (7 slots) family.
#include <nvrtc.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <sys/stat.h>
#include <unistd.h>

#include "sg_solver.h"

namespace sg {

namespace {

uint64_t fnv1a(const std::string& s) {
  uint64_t h = 1469598103934665603ull;
  for (unsigned char c : s) {
    h ^= c;
    h *= 1099511628211ull;
  }
  return h;
}

std::string cache_dir() {
  const char* env = std::getenv("SG_JIT_CACHE");
  if (env && *env) return env;
  const char* home = std::getenv("HOME");
  return std::string(home && *home ? home : "/tmp") + "/.cache/sg_gb300";
}

void mkdirs(const std::string& path) {
  std::string cur;
  std::stringstream ss(path);
  std::string part;
  if (!path.empty() && path[0] == '/') cur = "/";
  while (std::getline(ss, part, '/')) {
    if (part.empty()) continue;
    cur += part + "/";
    mkdir(cur.c_str(), 0755);
  }
}

std::string hexf(float g) {
  uint32_t u;
  std::memcpy(&u, &g, 4);
  char b[16];
  std::snprintf(b, sizeof b, "0x%08x", u);
  return b;
}

// contiguous output ranges [lo_h, hi_h) with about T/H triples each
std::vector<int> output_split(const sg_problem* pr, int H) {
  std::vector<int64_t> per_a(pr->P, 0);
  for (int64_t t = 0; t < pr->T; ++t) per_a[pr->kab[3 * t + 1]]++;
  std::vector<int> cut(H + 1, pr->P);
  cut[0] = 0;
  int64_t acc = 0;
  int h = 1;
  for (int a = 0; a < pr->P && h < H; ++a) {
    acc += per_a[a];
    if (acc * H >= int64_t(h) * pr->T) cut[h++] = a + 1;
  }
  for (int i = 1; i <= H; ++i) cut[i] = std::max(cut[i], cut[i - 1]);
  return cut;
}

}  // namespace

std::string jit_apply_source(const sg_problem* pr, const JitConfig& c) {
  const int P = pr->P, K = pr->K, R = c.rows, H = c.groups, pf = c.prefetch;
  const int mb = c.min_blocks;
  const std::vector<int> cut = output_split(pr, H);
  // triples grouped by k, then by a
  std::vector<std::map<int, std::vector<std::pair<int, float>>>> by_k(K);
  for (int64_t t = 0; t < pr->T; ++t) {
    int k = pr->kab[3 * t], a = pr->kab[3 * t + 1], b = pr->kab[3 * t + 2];
    by_k[k][a].push_back({b, float(pr->g[t])});
  }
  const char* ty = R == 2 ? "float2" : "float";
  std::ostringstream os;
  os << "// generated: Galerkin apply, P=" << P << " K=" << K << " T=" << pr->T << " R=" << R << " H=" << H
     << " pf=" << pf << " mb=" << mb << "\n";
  os << "#define G(h) __int_as_float(h)\n#define GG(h) make_float2(__int_as_float(h), __int_as_float(h))\n";
  os << "extern \"C\" __global__ void __launch_bounds__(" << 128 * H << ", " << mb << ") sg_k1(\n"
        "    const float* __restrict__ V, const int* __restrict__ col, long long ldr, int n, int S,\n"
        "    const float* __restrict__ X, long long ldx, const float* __restrict__ F, long long ldf,\n"
        "    float* __restrict__ Y, long long ldy) {\n"
        "  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;\n"
        "  const int grp = warp >> 2;\n"
        "  const int r = blockIdx.x * "
     << 128 * R << " + (warp & 3) * " << 32 * R << " + lane * " << R << ";\n"
     << "  if (r >= n) return;\n"
        "  const long long kst = (long long)S * ldr;\n";
  for (int h = 0; h < H; ++h) {
    const int lo = cut[h], hi = cut[h + 1];
    std::vector<int> ks;
    for (int k = 0; k < K; ++k) {
      bool any = false;
      for (const auto& ga : by_k[k]) any |= ga.first >= lo && ga.first < hi;
      if (any) ks.push_back(k);
    }
    std::vector<char> need_b(P, 0);
    for (int k : ks)
      for (const auto& ga : by_k[k])
        if (ga.first >= lo && ga.first < hi)
          for (const auto& e : ga.second) need_b[e.first] = 1;
    os << "  " << (h ? "else " : "") << "if (grp == " << h << ") {\n";
    for (int a = lo; a < hi; ++a)
      os << "    " << ty << " y" << a << (R == 2 ? " = make_float2(0.f, 0.f);\n" : " = 0.f;\n");
    os << "#pragma unroll 1\n"
          "    for (int s = 0; s < S; ++s) {\n"
          "      const float* xp0 = X + col[(long long)s * ldr + r];\n";
    if (R == 2) os << "      const float* xp1 = X + col[(long long)s * ldr + r + 1];\n";
    for (int b = 0; b < P; ++b) {
      if (!need_b[b]) continue;
      if (R == 2)
        os << "      const float2 x" << b << " = make_float2(__ldg(xp0 + (long long)" << b << " * ldx), __ldg(xp1 + (long long)"
           << b << " * ldx));\n";
      else
        os << "      const float x" << b << " = __ldg(xp0 + (long long)" << b << " * ldx);\n";
    }
    os << "      const float* vp = V + (long long)s * ldr + r;\n";
    auto load = [&](int k) {
      if (R == 2)
        os << "      const float2 v" << k << " = __ldg(reinterpret_cast<const float2*>(vp + (long long)" << k
           << " * kst));\n";
      else
        os << "      const float v" << k << " = __ldg(vp + (long long)" << k << " * kst);\n";
    };
    const int nk = int(ks.size());
    for (int i = 0; i < std::min(nk, pf); ++i) load(ks[i]);
    for (int i = 0; i < nk; ++i) {
      if (i + pf < nk) load(ks[i + pf]);
      const int k = ks[i];
      for (const auto& ga : by_k[k]) {
        const int a = ga.first;
        if (a < lo || a >= hi) continue;
        const auto& lst = ga.second;
        if (R == 1) {
          if (lst.size() == 1 && lst[0].second == 1.0f) {
            os << "      y" << a << " = fmaf(v" << k << ", x" << lst[0].first << ", y" << a << ");\n";
            continue;
          }
          os << "      { float t = x" << lst[0].first << " * G(" << hexf(lst[0].second) << ");";
          for (size_t e = 1; e < lst.size(); ++e)
            os << " t = fmaf(x" << lst[e].first << ", G(" << hexf(lst[e].second) << "), t);";
          os << " y" << a << " = fmaf(v" << k << ", t, y" << a << "); }\n";
        } else {
          if (lst.size() == 1 && lst[0].second == 1.0f) {
            os << "      y" << a << " = __ffma2_rn(v" << k << ", x" << lst[0].first << ", y" << a << ");\n";
            continue;
          }
          os << "      { float2 t = __fmul2_rn(x" << lst[0].first << ", GG(" << hexf(lst[0].second) << "));";
          for (size_t e = 1; e < lst.size(); ++e)
            os << " t = __ffma2_rn(x" << lst[e].first << ", GG(" << hexf(lst[e].second) << "), t);";
          os << " y" << a << " = __ffma2_rn(v" << k << ", t, y" << a << "); }\n";
        }
      }
    }
    os << "    }\n";
    for (int a = lo; a < hi; ++a) {
      if (R == 2) {
        os << "    Y[(long long)" << a << " * ldy + r] = F ? F[(long long)" << a << " * ldf + r] - y" << a
           << ".x : y" << a << ".x;\n";
        os << "    if (r + 1 < n) Y[(long long)" << a << " * ldy + r + 1] = F ? F[(long long)" << a
           << " * ldf + r + 1] - y" << a << ".y : y" << a << ".y;\n";
      } else {
        os << "    Y[(long long)" << a << " * ldy + r] = F ? F[(long long)" << a << " * ldf + r] - y" << a << " : y"
           << a << ";\n";
      }
    }
    os << "  }\n";
  }
  os << "}\n";
  return os.str();
}

// Compile (or load from the cache) one configuration.
static sg_status jit_compile(const std::string& src, cudaLibrary_t* lib, cudaKernel_t* kern, bool* cached,
                             double* seconds) {
  auto t0 = std::chrono::steady_clock::now();
  char key[32];
  std::snprintf(key, sizeof key, "%016llx", (unsigned long long)fnv1a(src + "|sm_103a|v3"));
  const std::string dir = cache_dir();
  const std::string path = dir + "/k1_" + key + ".cubin";
  std::vector<char> cubin;
  {
    std::ifstream in(path, std::ios::binary);
    if (in) cubin.assign(std::istreambuf_iterator<char>(in), std::istreambuf_iterator<char>());
  }
  if (cached) *cached = !cubin.empty();
  if (cubin.empty()) {
    nvrtcProgram prog;
    if (nvrtcCreateProgram(&prog, src.c_str(), "sg_k1.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) {
      set_error("NVRTC: cannot create the specialised apply program");
      return SG_ERR_CUDA;
    }
    const char* opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "--fmad=true", "-lineinfo"};
    nvrtcResult rc = nvrtcCompileProgram(prog, 4, opts);
    if (rc != NVRTC_SUCCESS) {
      size_t ls = 0;
      nvrtcGetProgramLogSize(prog, &ls);
      std::string log(ls, '\0');
      nvrtcGetProgramLog(prog, &log[0]);
      nvrtcDestroyProgram(&prog);
      set_error("NVRTC compile of the specialised apply failed: " + log.substr(0, 2000));
      return SG_ERR_CUDA;
    }
    size_t sz = 0;
    nvrtcGetCUBINSize(prog, &sz);
    cubin.resize(sz);
    nvrtcGetCUBIN(prog, cubin.data());
    nvrtcDestroyProgram(&prog);
    mkdirs(dir);
    const std::string tmp = path + ".tmp" + std::to_string(::getpid());
    std::ofstream out(tmp, std::ios::binary);
    if (out) {
      out.write(cubin.data(), std::streamsize(cubin.size()));
      out.close();
      std::rename(tmp.c_str(), path.c_str());
    }
  }
  SG_CUDA(cudaLibraryLoadData(lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0));
  SG_CUDA(cudaLibraryGetKernel(kern, *lib, "sg_k1"));
  if (seconds) *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return SG_OK;
}

JitConfig jit_default_config(const sg_problem* pr) {
  JitConfig c;
  if (pr->P <= 48) {
    c.rows = 2;
    c.groups = 1;
    c.prefetch = 16;
  } else {
    c.rows = 1;
    c.groups = pr->P <= 96 ? 2 : 3;
    c.prefetch = 8;
  }
  c.min_blocks = 1;
  return c;
}

sg_status jit_apply_build(sg_problem* pr) {
  if (pr->jit && pr->jit->kern) return SG_OK;
  if (!pr->jit) pr->jit = new JitApply();
  JitApply& J = *pr->jit;
  if (!pr->jit_cfg_set) {
    pr->jit_cfg = jit_default_config(pr);
    pr->jit_cfg_set = true;
  }
  return jit_compile(jit_apply_source(pr, pr->jit_cfg), &J.lib, &J.kern, &J.from_cache, &J.compile_s);
}

sg_status jit_configure(sg_problem* pr, const JitConfig& c) {
  if (c.rows < 1 || c.rows > 2 || c.groups < 1 || c.groups > 4 || c.prefetch < 0 || c.prefetch > 64 ||
      c.min_blocks < 1 || c.min_blocks > 8) {
    set_error("sg_apply_config: rows in {1,2}, groups in [1,4], prefetch in [0,64], min_blocks in [1,8]");
    return SG_ERR_ARG;
  }
  jit_free(pr);
  pr->jit_cfg = c;
  pr->jit_cfg_set = true;
  if (!jit_eligible(pr)) return SG_OK;
  return jit_apply_build(pr);
}

void jit_free(sg_problem* pr) {
  if (!pr->jit) return;
  if (pr->jit->lib) cudaLibraryUnload(pr->jit->lib);
  delete pr->jit;
  pr->jit = nullptr;
}

bool jit_eligible(const sg_problem* pr) { return pr->P <= kJitMaxP && pr->T <= kJitMaxT; }

static sg_status launch_kernel(cudaKernel_t kern, const JitConfig& c, const Ell& A, const float* X, int64_t ldx,
                               const float* F, int64_t ldf, float* Y, int64_t ldy, cudaStream_t st) {
  if (A.n == 0) return SG_OK;
  const float* V = dp<float>(A.v32);
  const int* col = dp<int>(A.col);
  long long ldr = A.ldr, lx = ldx, lf = ldf, ly = ldy;
  int n = int(A.n), S = A.S;
  void* args[] = {(void*)&V, (void*)&col, &ldr, &n, &S, (void*)&X, &lx, (void*)&F, &lf, (void*)&Y, &ly};
  const int64_t rows_per_cta = 128LL * c.rows;
  dim3 grid(unsigned((A.n + rows_per_cta - 1) / rows_per_cta)), block(unsigned(128 * c.groups));
  SG_CUDA(cudaLaunchKernel((const void*)kern, grid, block, args, 0, st));
  note_launch();
  return SG_OK;
}

sg_status jit_apply_launch(sg_problem* pr, const Ell& A, const float* X, int64_t ldx, const float* F, int64_t ldf,
                           float* Y, int64_t ldy, cudaStream_t st) {
  SG_TRY(jit_apply_build(pr));
  return launch_kernel(pr->jit->kern, pr->jit_cfg, A, X, ldx, F, ldf, Y, ldy, st);
}

// --------------------------------------------------------------------------
// Autotuner: compile the candidate tile shapes, time each on this problem's
// fine operator (median of a few launches after a warm-up, CUDA events),
// keep the fastest and remember the choice in the cache directory, keyed by
// the triple structure, n and the device name.
// --------------------------------------------------------------------------
static std::vector<JitConfig> candidates(const sg_problem* pr) {
  std::vector<JitConfig> out;
  for (int R : {1, 2})
    for (int H : {1, 2, 3})
      for (int pf : {8, 16, 32}) {
        const int per = (pr->P + H - 1) / H;
        const int est = R * (per + pr->P + pf);  // live registers, roughly
        if (est > 200) continue;
        if (H > 1 && pr->P <= 24) continue;
        JitConfig c;
        c.rows = R;
        c.groups = H;
        c.prefetch = pf;
        c.min_blocks = 1;
        out.push_back(c);
      }
  if (out.empty()) out.push_back(jit_default_config(pr));
  return out;
}

static std::string tune_key(const sg_problem* pr) {
  cudaDeviceProp prop{};
  cudaGetDeviceProperties(&prop, pr->device);
  std::ostringstream os;
  os << prop.name << "|" << pr->P << "|" << pr->K << "|" << pr->T << "|" << pr->n;
  for (int64_t t = 0; t < pr->T; ++t) os << "," << pr->kab[3 * t] << ":" << pr->kab[3 * t + 1] << ":" << pr->kab[3 * t + 2];
  char key[32];
  std::snprintf(key, sizeof key, "%016llx", (unsigned long long)fnv1a(os.str()));
  return key;
}

sg_status jit_autotune(sg_problem* pr, int force, double* best_ms) {
  if (!jit_eligible(pr)) {
    set_error("sg_apply_autotune: the specialised kernel is not available for this size");
    return SG_ERR_UNSUPPORTED;
  }
  const std::string path = cache_dir() + "/tune_" + tune_key(pr) + ".txt";
  if (!force) {
    std::ifstream in(path);
    JitConfig c;
    double ms = 0;
    if (in >> c.rows >> c.groups >> c.prefetch >> c.min_blocks >> ms) {
      if (best_ms) *best_ms = ms;
      return jit_configure(pr, c);
    }
  }
  const Ell& A = pr->fine;
  const int64_t len = int64_t(pr->P) * pr->ld;
  DevBuf X, Y;
  SG_TRY(X.alloc(len * 4));
  SG_TRY(Y.alloc(len * 4));
  cudaStream_t st;
  SG_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  cudaEvent_t e0, e1;
  SG_CUDA(cudaEventCreate(&e0));
  SG_CUDA(cudaEventCreate(&e1));
  JitConfig best = jit_default_config(pr);
  double best_t = 1e30;
  sg_status status = SG_OK;
  for (const JitConfig& c : candidates(pr)) {
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kern = nullptr;
    if (jit_compile(jit_apply_source(pr, c), &lib, &kern, nullptr, nullptr) != SG_OK) continue;
    std::vector<float> ts;
    for (int rep = 0; rep < 7 && status == SG_OK; ++rep) {
      status = launch_kernel(kern, c, A, dp<float>(X), pr->ld, nullptr, 0, dp<float>(Y), pr->ld, st);
      if (status != SG_OK) break;
      if (rep < 2) continue;
      cudaEventRecord(e0, st);
      launch_kernel(kern, c, A, dp<float>(X), pr->ld, nullptr, 0, dp<float>(Y), pr->ld, st);
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      ts.push_back(ms);
    }
    cudaLibraryUnload(lib);
    if (status != SG_OK) break;
    std::sort(ts.begin(), ts.end());
    const double med = ts.empty() ? 1e30 : ts[ts.size() / 2];
    if (med < best_t) {
      best_t = med;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  SG_TRY(status);
  if (best_ms) *best_ms = best_t;
  mkdirs(cache_dir());
  std::ofstream out(path);
  if (out) out << best.rows << " " << best.groups << " " << best.prefetch << " " << best.min_blocks << " " << best_t << "\n";
  return jit_configure(pr, best);
}

}  // namespace sg
