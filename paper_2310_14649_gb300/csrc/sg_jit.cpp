// Register-specialised Galerkin apply (Sec. 2.1, Eq. Galerkin_L_exp):
//     y_r[a] = sum_s sum_{(k,a,b)} v_k^{r,s} g_kab x_{col(r,s)}[b].
//
// The triple list depends only on (L, p, q), so at setup the library writes
// a CUDA kernel in which every nonzero g_kab is an immediate operand and
// every accumulator y[a] and gathered value x[b] lives in a named register.
// One thread owns one row; per stencil slot it gathers the P values of the
// neighbour, then streams the K matrix values of that slot (coalesced across
// the warp: lanes are consecutive rows) and, for each input term k, updates
// the outputs coupled to it:  y_a += v_k * (sum_b g_kab x_b).  The kernel is
// compiled for sm_103a with NVRTC and cached on disk by a hash of its source.
// The same kernel serves the fine (5 slots) and the coarse (7 slots) family.
#include <nvrtc.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <sys/stat.h>

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

}  // namespace

std::string jit_apply_source(const sg_problem* pr) {
  const int P = pr->P, K = pr->K;
  // input terms whose matrix values are loaded ahead of use, and the
  // minimum resident CTAs per SM (bounds the registers per thread)
  const int kPrefetch = pr->jit_cfg.prefetch;
  const int kMinBlocks = pr->jit_cfg.min_blocks > 0 ? pr->jit_cfg.min_blocks
                         : (P <= 40 ? 3 : (P <= 64 ? 2 : 1));
  // triples grouped by k, then by a
  std::vector<std::map<int, std::vector<std::pair<int, float>>>> by_k(K);
  for (int64_t t = 0; t < pr->T; ++t) {
    int k = pr->kab[3 * t], a = pr->kab[3 * t + 1], b = pr->kab[3 * t + 2];
    by_k[k][a].push_back({b, float(pr->g[t])});
  }
  std::ostringstream os;
  os << "// generated: stochastic Galerkin apply for P=" << P << " K=" << K << " T=" << pr->T << "\n";
  os << "#define G(h) __int_as_float(h)\n";
  os << "extern \"C\" __global__ void __launch_bounds__(128, " << kMinBlocks << ") sg_k1(\n"
        "    const float* __restrict__ V, const int* __restrict__ col, long long ldr, int n, int S,\n"
        "    const float* __restrict__ X, long long ldx, const float* __restrict__ F, long long ldf,\n"
        "    float* __restrict__ Y, long long ldy) {\n"
        "  const int r = blockIdx.x * 128 + threadIdx.x;\n"
        "  if (r >= n) return;\n";
  for (int a = 0; a < P; ++a) os << "  float y" << a << " = 0.f;\n";
  os << "  const long long kst = (long long)S * ldr;\n"
        "#pragma unroll 1\n"
        "  for (int s = 0; s < S; ++s) {\n"
        "    const float* xp = X + col[(long long)s * ldr + r];\n";
  for (int b = 0; b < P; ++b) os << "    const float x" << b << " = __ldg(xp + (long long)" << b << " * ldx);\n";
  os << "    const float* vp = V + (long long)s * ldr + r;\n";
  auto load = [&](int k) { os << "    const float v" << k << " = __ldg(vp + (long long)" << k << " * kst);\n"; };
  for (int k = 0; k < std::min(K, kPrefetch); ++k) load(k);
  char hex[16];
  for (int k = 0; k < K; ++k) {
    if (k + kPrefetch < K) load(k + kPrefetch);
    for (const auto& ga : by_k[k]) {
      const int a = ga.first;
      const auto& lst = ga.second;
      if (lst.size() == 1) {
        const auto& e = lst[0];
        if (e.second == 1.0f) {
          os << "    y" << a << " = fmaf(v" << k << ", x" << e.first << ", y" << a << ");\n";
        } else {
          uint32_t u;
          std::memcpy(&u, &e.second, 4);
          std::snprintf(hex, sizeof hex, "0x%08x", u);
          os << "    y" << a << " = fmaf(v" << k << ", x" << e.first << " * G(" << hex << "), y" << a << ");\n";
        }
        continue;
      }
      os << "    { float t = ";
      for (size_t i = 0; i < lst.size(); ++i) {
        uint32_t u;
        std::memcpy(&u, &lst[i].second, 4);
        std::snprintf(hex, sizeof hex, "0x%08x", u);
        if (i == 0)
          os << "x" << lst[i].first << " * G(" << hex << ");";
        else
          os << " t = fmaf(x" << lst[i].first << ", G(" << hex << "), t);";
      }
      os << " y" << a << " = fmaf(v" << k << ", t, y" << a << "); }\n";
    }
  }
  os << "  }\n";
  for (int a = 0; a < P; ++a)
    os << "  Y[(long long)" << a << " * ldy + r] = F ? F[(long long)" << a << " * ldf + r] - y" << a << " : y" << a
       << ";\n";
  os << "}\n";
  return os.str();
}

sg_status jit_apply_build(sg_problem* pr) {
  if (pr->jit && pr->jit->kern) return SG_OK;
  if (!pr->jit) pr->jit = new JitApply();
  JitApply& J = *pr->jit;
  const std::string src = jit_apply_source(pr);
  char key[32];
  std::snprintf(key, sizeof key, "%016llx", (unsigned long long)fnv1a(src + "|sm_103a|v2"));
  const std::string dir = cache_dir();
  const std::string path = dir + "/k1_" + key + ".cubin";
  std::vector<char> cubin;
  {
    std::ifstream in(path, std::ios::binary);
    if (in) cubin.assign(std::istreambuf_iterator<char>(in), std::istreambuf_iterator<char>());
  }
  J.from_cache = !cubin.empty();
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
    std::ofstream out(path + ".tmp", std::ios::binary);
    if (out) {
      out.write(cubin.data(), std::streamsize(cubin.size()));
      out.close();
      std::rename((path + ".tmp").c_str(), path.c_str());
    }
  }
  SG_CUDA(cudaLibraryLoadData(&J.lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0));
  SG_CUDA(cudaLibraryGetKernel(&J.kern, J.lib, "sg_k1"));
  return SG_OK;
}

sg_status jit_configure(sg_problem* pr, int min_blocks, int prefetch) {
  if (min_blocks < 0 || min_blocks > 8 || prefetch < 0 || prefetch > 64) {
    set_error("sg_apply_config: min_blocks in [0, 8], prefetch in [0, 64]");
    return SG_ERR_ARG;
  }
  jit_free(pr);
  pr->jit_cfg.min_blocks = min_blocks;
  pr->jit_cfg.prefetch = prefetch;
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

sg_status jit_apply_launch(sg_problem* pr, const Ell& A, const float* X, int64_t ldx, const float* F, int64_t ldf,
                           float* Y, int64_t ldy, cudaStream_t st) {
  SG_TRY(jit_apply_build(pr));
  if (A.n == 0) return SG_OK;
  const float* V = dp<float>(A.v32);
  const int* col = dp<int>(A.col);
  long long ldr = A.ldr, lx = ldx, lf = ldf, ly = ldy;
  int n = int(A.n), S = A.S;
  void* args[] = {(void*)&V, (void*)&col, &ldr, &n, &S, (void*)&X, &lx, (void*)&F, &lf, (void*)&Y, &ly};
  dim3 grid(unsigned((A.n + 127) / 128)), block(128);
  SG_CUDA(cudaLaunchKernel((const void*)pr->jit->kern, grid, block, args, 0, st));
  note_launch();
  return SG_OK;
}

}  // namespace sg
