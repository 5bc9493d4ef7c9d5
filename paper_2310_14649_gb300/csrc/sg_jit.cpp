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
//   HI input groups: the gathered x[b] are split into HI ranges as well;
//      each (output, input) group accumulates partial sums that meet in
//      shared memory, in a fixed order, before the single write of Y;
//   SG slot groups: the stencil slots are dealt round-robin to SG groups
//      (more threads for small row counts such as the coarse operator);
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

std::string hexd(double g) {
  uint64_t u;
  std::memcpy(&u, &g, 8);
  char b[24];
  std::snprintf(b, sizeof b, "0x%016llxull", (unsigned long long)u);
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

std::string jit_apply_source(const sg_problem* pr, const JitConfig& c, bool fp64) {
  // output groups either as 4-warp groups of one CTA (partial sums meet in
  // shared memory, registers capped by the CTA width) or as separate
  // 128-thread CTAs (each writes its own outputs; rows shared by
  // consecutive CTAs, so their matrix values meet in L2)
  const bool csplit = c.cgroups > 1;
  const int P = pr->P, K = pr->K, R = fp64 ? 1 : c.rows, HO = csplit ? c.cgroups : c.groups,
            HI = csplit ? 1 : c.igroups, SG = csplit ? 1 : c.sgroups, pf = c.prefetch;
  // FP64 family: the same code over double values, inputs and outputs, the
  // coefficients as exact double immediates
  const char* T = fp64 ? "double" : "float";
  const std::string Ts = T;
  const bool flux = c.flux != 0 && !fp64;
  const int mb = c.min_blocks, NG = HO * HI * SG, NPART = HI * SG, W = csplit ? 4 : c.warps;
  const std::vector<int> cut = output_split(pr, HO);
  std::vector<int> icut(HI + 1);
  for (int i = 0; i <= HI; ++i) icut[i] = int(int64_t(P) * i / HI);
  // triples grouped by k, then by a
  std::vector<std::map<int, std::vector<std::pair<int, double>>>> by_k(K);
  for (int64_t t = 0; t < pr->T; ++t) {
    int k = pr->kab[3 * t], a = pr->kab[3 * t + 1], b = pr->kab[3 * t + 2];
    by_k[k][a].push_back({b, fp64 ? pr->g[t] : double(float(pr->g[t]))});
  }
  // paired rows take their coefficients from the constant bank (the paired
  // FMA has no immediate operand)
  std::map<uint32_t, int> gslot;
  std::vector<float> gvals;
  auto gref = [&](double gd) -> std::string {
    if (fp64) return "GD(" + hexd(gd) + ")";
    const float g = float(gd);
    if (R == 1) return "G(" + hexf(g) + ")";
    uint32_t u;
    std::memcpy(&u, &g, 4);
    auto it = gslot.find(u);
    int id;
    if (it == gslot.end()) {
      id = int(gvals.size());
      gslot[u] = id;
      gvals.push_back(g);
    } else {
      id = it->second;
    }
    return "gq2[" + std::to_string(id) + "]";
  };
  const char* ty = R == 2 ? "float2" : T;
  std::ostringstream body;
  std::string staged_table;
  // slot groups alone run the same code from different first slots: one
  // body with the slot offset taken from the group index (separate unrolled
  // bodies per group multiply the instruction footprint)
  const bool slot_only = !csplit && HO == 1 && HI == 1 && SG > 1;
  for (int g = 0; g < (slot_only ? 1 : NG); ++g) {
    const int ho = g / (HI * SG), hi = (g / SG) % HI, sgi = g % SG;
    const int lo = cut[ho], up = cut[ho + 1], blo = icut[hi], bup = icut[hi + 1];
    auto in_grp = [&](int a, int b) { return a >= lo && a < up && b >= blo && b < bup; };
    std::vector<int> ks;
    std::vector<char> need_b(P, 0), has_a(P, 0);
    for (int k = 0; k < K; ++k) {
      bool any = false;
      for (const auto& ga : by_k[k])
        for (const auto& e : ga.second)
          if (in_grp(ga.first, e.first)) {
            any = true;
            need_b[e.first] = 1;
            has_a[ga.first] = 1;
          }
      if (any) ks.push_back(k);
    }
    if (slot_only)
      body << "  {\n";
    else
      body << "  " << (g ? "else " : "") << "if (grp == " << g << ") {\n";
    for (int a = lo; a < up; ++a)
      if (has_a[a]) body << "    " << ty << " y" << a << (R == 2 ? " = make_float2(0.f, 0.f);\n" : (fp64 ? " = 0.0;\n" : " = 0.f;\n"));
    body << "#pragma unroll 1\n"
            "    for (int s = " << (slot_only ? std::string("grp") : std::to_string(sgi)) << "; s < S; s += " << SG
         << ") {\n";
    if (flux)
      body << "      const int cn = col[(long long)s * ldr + rr];\n"
              "      const float mk = cn >= 0 ? 1.f : 0.f;\n"
              "      const float* xp0 = X + (cn >= 0 ? cn : rr);\n"
              "      const float* xr0 = X + rr;\n";
    else
      body << "      const " << Ts << "* xp0 = X + col[(long long)s * ldr + rr];\n";
    if (R == 2) body << "      const float* xp1 = X + col[(long long)s * ldr + rr + 1];\n";
    for (int b = 0; b < P; ++b) {
      if (!need_b[b]) continue;
      if (R == 2)
        body << "      const float2 x" << b << " = make_float2(__ldg(xp0 + (long long)" << b
             << " * ldx), __ldg(xp1 + (long long)" << b << " * ldx));\n";
      else if (flux)  // the difference across the edge: x_r - x_neighbour (0 at a Dirichlet node)
        body << "      const float x" << b << " = fmaf(-mk, __ldg(xp0 + (long long)" << b
             << " * ldx), __ldg(xr0 + (long long)" << b << " * ldx));\n";
      else
        body << "      const " << Ts << " x" << b << " = __ldg(xp0 + (long long)" << b << " * ldx);\n";
    }
    const bool staged = c.stages >= 2;
    if (!staged && flux) body << "      const float* vp = V + vidx[(long long)s * ldr + rr];\n";
    else if (!staged) body << "      const " << Ts << "* vp = V + (long long)s * ldr + rr;\n";
    auto load = [&](int k) {
      if (R == 2)
        body << "      const float2 v" << k << " = __ldg(reinterpret_cast<const float2*>(vp + (long long)" << k
             << " * kst));\n";
      else
        body << "      const " << Ts << " v" << k << " = __ldg(vp + (long long)" << k << " * kst);\n";
    };
    const int nk = int(ks.size());
    // staged: blocks of KB input terms arrive in shared memory (cp.async,
    // stages - 1 blocks ahead, across slot boundaries); each thread reads
    // back only the values it copied, so no barrier is needed
    const int KB = std::max(1, pf);
    if (!staged)
      for (int i = 0; i < std::min(nk, pf); ++i) load(ks[i]);
    for (int i = 0; i < nk; ++i) {
      if (staged && i % KB == 0) {
        if (i) body << "      }\n";
        body << "      {\n        asm volatile(\"cp.async.wait_group " << (c.stages - 2) << ";\" ::: \"memory\");\n"
             << "        issue_blk(gb + " << (c.stages - 1) << ", S, V, ldr, kst, rr, vsm);\n"
             << "        const " << Ts << "* vb = vsm + (gb % " << c.stages << ") * " << KB * 128 << ";\n"
             << "        ++gb;\n";
        for (int q = i; q < std::min(nk, i + KB); ++q)
          body << "        const " << Ts << " v" << ks[q] << " = vb[" << (q - i) * 128 << "];\n";
      }
      if (!staged && i + pf < nk) load(ks[i + pf]);
      const int k = ks[i];
      for (const auto& ga : by_k[k]) {
        const int a = ga.first;
        std::vector<std::pair<int, double>> lst;
        for (const auto& e : ga.second)
          if (in_grp(a, e.first)) lst.push_back(e);
        if (lst.empty()) continue;
        const char* fma = R == 2 ? "__ffma2_rn" : (fp64 ? "fma" : "fmaf");
        if (lst.size() == 1 && lst[0].second == 1.0) {
          body << "      y" << a << " = " << fma << "(v" << k << ", x" << lst[0].first << ", y" << a << ");\n";
          continue;
        }
        if (R == 2)
          body << "      { float2 t = __fmul2_rn(x" << lst[0].first << ", " << gref(lst[0].second) << ");";
        else
          body << "      { " << Ts << " t = x" << lst[0].first << " * " << gref(lst[0].second) << ";";
        for (size_t e = 1; e < lst.size(); ++e)
          body << " t = " << fma << "(x" << lst[e].first << ", " << gref(lst[e].second) << ", t);";
        body << " y" << a << " = " << fma << "(v" << k << ", t, y" << a << "); }\n";
      }
    }
    if (staged && nk > 0) body << "      }\n";
    body << "    }\n";
    if (staged) {
      // the table of input terms per block, for the copy helper
      std::ostringstream tab;
      const int NB = (nk + KB - 1) / KB;
      tab << "#define STG_NB " << NB << "\n__constant__ int c_ktab[" << std::max(1, NB * KB) << "] = {";
      for (int e = 0; e < NB * KB; ++e) tab << (e ? ", " : "") << (e < nk ? ks[e] : -1);
      if (NB * KB == 0) tab << "-1";
      tab << "};\n";
      staged_table = tab.str();
    }
    if (csplit) {  // this CTA's outputs, written straight from registers
      for (int a = lo; a < up; ++a) {
        const std::string val = has_a[a] ? "y" + std::to_string(a) : std::string(fp64 ? "0.0" : "0.f");
        body << "    if (r < n) Y[(long long)" << a << " * ldy + r] = F ? F[(long long)" << a << " * ldf + r] - " << val
             << " : " << val << ";\n";
      }
      body << "  }\n";
      continue;
    }
    // partial sums of the input and slot groups meet in shared memory, in
    // group order; outputs this group never touches contribute zero
    for (int a = lo; a < up; ++a) {
      if (!has_a[a]) {
        for (int q = 0; q < R; ++q) body << "    part[" << a << " * " << 32 * W * R << " + lrow + " << q << "] = 0;\n";
        continue;
      }
      for (int q = 0; q < R; ++q) {
        const std::string val = R == 2 ? ("y" + std::to_string(a) + (q ? ".y" : ".x")) : ("y" + std::to_string(a));
        body << "    part[" << a << " * " << 32 * W * R << " + lrow + " << q << "] = " << val << ";\n";
      }
    }
    body << "  }\n";
  }
  std::ostringstream os;
  os << "// generated: Galerkin apply, P=" << P << " K=" << K << " T=" << pr->T << " R=" << R << " groups=" << HO
     << "x" << HI << "x" << SG << " pf=" << pf << " mb=" << mb << (fp64 ? " fp64" : "") << (flux ? " flux" : "")
     << "\n";
  os << (fp64 ? "#define GD(h) __longlong_as_double(h)\n" : "#define G(h) __int_as_float(h)\n");
  if (c.stages >= 2) {
    const int KB = std::max(1, pf);
    os << staged_table;
    os << "__device__ __forceinline__ void cpa(" << Ts << "* d, const " << Ts << "* s) {\n"
          "  const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(d));\n"
          "  asm volatile(\"cp.async.ca.shared.global [%0], [%1], " << (fp64 ? 8 : 4) << ";\" :: \"r\"(a), \"l\"(s) : \"memory\");\n"
          "}\n"
          "// copy block gb (slot gb / NB, terms c_ktab[(gb % NB) * KB ...]) of this thread's row\n"
          "__device__ __forceinline__ void issue_blk(int gb, int S, const " << Ts << "* V, long long ldr, long long kst,\n"
          "                                           int rr, " << Ts << "* vsm) {\n"
          "  if (gb < S * STG_NB) {\n"
          "    const int s = gb / STG_NB, b = gb - s * STG_NB;\n"
          "    const " << Ts << "* vp = V + (long long)s * ldr + rr;\n"
          "    " << Ts << "* d = vsm + (gb % " << c.stages << ") * " << KB * 128 << ";\n"
          "#pragma unroll\n"
          "    for (int i = 0; i < " << KB << "; ++i) {\n"
          "      const int k = c_ktab[b * " << KB << " + i];\n"
          "      if (k >= 0) cpa(d + i * 128, vp + (long long)k * kst);\n"
          "    }\n"
          "  }\n"
          "  asm volatile(\"cp.async.commit_group;\" ::: \"memory\");\n"
          "}\n";
  }
  if (R == 2 && !gvals.empty()) {
    // both halves of each pair carry the same coefficient bits
    os << "__constant__ unsigned long long gq_bits[" << gvals.size() << "] = {";
    for (size_t i = 0; i < gvals.size(); ++i) {
      const std::string h = hexf(gvals[i]).substr(2);
      os << (i ? ", " : "") << "0x" << h << h << "ull";
    }
    os << "};\n#define gq2 (reinterpret_cast<const float2*>(gq_bits))\n";
  }
  const int rows_cta = 32 * W * R;
  if (csplit) {
    os << "extern \"C\" __global__ void __launch_bounds__(128, " << mb << ") " << (fp64 ? "sg_k1_f64" : "sg_k1")
       << "(\n"
          "    const " << Ts << "* __restrict__ V, const int* __restrict__ col, long long ldr, int n, int S,\n"
          "    const " << Ts << "* __restrict__ X, long long ldx, const " << Ts << "* __restrict__ F, long long ldf,\n"
          "    " << Ts << "* __restrict__ Y, long long ldy, const int* __restrict__ vidx, long long vkst) {\n"
          "  const int grp = blockIdx.x % " << HO << ";\n"
          "  const int r = (blockIdx.x / " << HO << ") * 128 + threadIdx.x;\n"
          "  const int rr = r < n ? r : n - 1;\n"
          "  const long long kst = vkst > 0 ? vkst : (long long)S * ldr;\n";
    os << body.str();
    os << "}\n";
    return os.str();
  }
  os << "extern \"C\" __global__ void __launch_bounds__(" << 32 * W * NG << ", " << mb << ") "
     << (fp64 ? "sg_k1_f64" : "sg_k1") << "(\n"
        "    const " << Ts << "* __restrict__ V, const int* __restrict__ col, long long ldr, int n, int S,\n"
        "    const " << Ts << "* __restrict__ X, long long ldx, const " << Ts << "* __restrict__ F, long long ldf,\n"
        "    " << Ts << "* __restrict__ Y, long long ldy, const int* __restrict__ vidx, long long vkst) {\n"
        "  extern __shared__ " << Ts << " smem[];\n"
        "  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;\n"
        "  const int grp = warp / " << W << ";\n"
        "  const int lrow = (warp % " << W << ") * "
     << 32 * R << " + lane * " << R << ";\n"
     << "  const int r = blockIdx.x * " << rows_cta << " + lrow;\n"
     << "  const int rr = r < n ? r : (n - 1) & ~" << (R - 1) << ";\n"
     << "  const long long kst = vkst > 0 ? vkst : (long long)S * ldr;\n";
  if (NG == 1) {
    os << "  " << Ts << "* part = smem;\n  (void)part;\n";
    if (c.stages >= 2)
      os << "  " << Ts << "* vsm = smem + lrow;\n"
         << "  for (int g0 = 0; g0 < " << (c.stages - 1) << "; ++g0) issue_blk(g0, S, V, ldr, kst, rr, vsm);\n"
         << "  int gb = 0;\n";
    // single group: write straight from registers
    std::string b = body.str();
    // drop the shared-memory hand-off of the single group
    std::ostringstream direct;
    std::istringstream in(b);
    std::string line;
    while (std::getline(in, line)) {
      if (line.find("part[") != std::string::npos) continue;
      direct << line << "\n";
      if (line == "    }") {  // end of the slot loop: write the outputs
        for (int a = 0; a < P; ++a)
          for (int q = 0; q < R; ++q) {
            const std::string val = R == 2 ? ("y" + std::to_string(a) + (q ? ".y" : ".x")) : ("y" + std::to_string(a));
            direct << "    if (r + " << q << " < n) Y[(long long)" << a << " * ldy + r + " << q << "] = F ? F[(long long)"
                   << a << " * ldf + r + " << q << "] - " << val << " : " << val << ";\n";
          }
      }
    }
    os << direct.str();
  } else {
    os << "  " << Ts << "* part = smem + (size_t)(grp % " << NPART << ") * " << P * rows_cta << ";\n";
    os << body.str();
    os << "  __syncthreads();\n";
    os << "  for (int e = threadIdx.x; e < " << P * rows_cta << "; e += " << 32 * W * NG << ") {\n"
          "    const int a = e / "
       << rows_cta << ", lr = e - a * " << rows_cta << ";\n"
       << "    const int row = blockIdx.x * " << rows_cta << " + lr;\n"
       << "    if (row >= n) continue;\n"
          "    " << Ts << " acc = smem[e];\n";
    for (int q = 1; q < NPART; ++q) os << "    acc += smem[" << q * P * rows_cta << " + e];\n";
    os << "    Y[(long long)a * ldy + row] = F ? F[(long long)a * ldf + row] - acc : acc;\n  }\n";
  }
  os << "}\n";
  return os.str();
}

size_t jit_smem_bytes(const sg_problem* pr, const JitConfig& c, bool fp64) {
  if (c.cgroups > 1) return 0;
  if (c.stages >= 2) return size_t(c.stages) * std::max(1, c.prefetch) * 128 * (fp64 ? sizeof(double) : sizeof(float));
  if (c.groups * c.igroups * c.sgroups == 1) return 0;
  return size_t(c.igroups) * c.sgroups * pr->P * 32 * c.warps * c.rows * (fp64 ? sizeof(double) : sizeof(float));
}

// Compile (or load from the cache) one configuration.
static sg_status jit_compile(const std::string& src, cudaLibrary_t* lib, cudaKernel_t* kern, bool* cached,
                             double* seconds, int dev, bool fp64) {
  auto t0 = std::chrono::steady_clock::now();
  char key[32];
  std::snprintf(key, sizeof key, "%016llx", (unsigned long long)fnv1a(src + "|sm_103a|v" + std::to_string(kJitGeneratorVersion)));
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
  SG_CUDA(cudaLibraryGetKernel(kern, *lib, fp64 ? "sg_k1_f64" : "sg_k1"));
  SG_CUDA(cudaKernelSetAttributeForDevice(*kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024, dev));
  if (seconds) *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return SG_OK;
}

JitConfig jit_default_config(const sg_problem* pr, int which) {
  const bool fp64 = which >= 2, coarse = which % 2 == 1;
  JitConfig c;
  c.rows = 1;
  c.min_blocks = 1;
  if (pr->P > 48) {
    // large P: output groups as separate CTAs keep every register of a
    // 128-thread CTA for one output range
    c.prefetch = 8;
    c.cgroups = std::min(16, (pr->P + (fp64 ? 15 : 23)) / (fp64 ? 16 : 24));
    return c;
  }
  c.prefetch = fp64 ? 16 : 32;
  // the coarse operator has a quarter of the rows: deal the slots to two
  // groups so that the grid still fills the GPU (four groups of 4 warps cap
  // the CTA at 128 registers a thread and spill: 0.115 against 0.053 ms at
  // 127^2 coarse rows, P = 35)
  c.sgroups = coarse ? 2 : 1;
  return c;
}

sg_status jit_apply_build(sg_problem* pr, int which) {
  if (pr->jit[which] && pr->jit[which]->kern) return SG_OK;
  if (!pr->jit[which]) pr->jit[which] = new JitApply();
  JitApply& J = *pr->jit[which];
  if (!pr->jit_cfg_set[which]) {
    pr->jit_cfg[which] = jit_default_config(pr, which);
    pr->jit_cfg_set[which] = true;
  }
  return jit_compile(jit_apply_source(pr, pr->jit_cfg[which], which >= 2), &J.lib, &J.kern, &J.from_cache,
                     &J.compile_s, pr->device, which >= 2);
}

sg_status jit_configure(sg_problem* pr, int which, const JitConfig& c) {
  if (c.rows < 1 || c.rows > 2 || c.groups < 1 || c.groups > 4 || c.igroups < 1 || c.igroups > 4 ||
      c.sgroups < 1 || c.sgroups > 8 || c.groups * c.igroups * c.sgroups > 8 || c.prefetch < 0 ||
      c.prefetch > 64 || c.min_blocks < 1 || c.min_blocks > 8 || (which >= 2 && c.rows != 1) ||
      c.stages < 0 || c.stages == 1 || c.stages > 8 ||
      (c.stages >= 2 && (c.rows != 1 || c.groups * c.igroups * c.sgroups != 1 || c.prefetch < 1)) ||
      c.cgroups < 1 || c.cgroups > 16 ||
      (c.cgroups > 1 && (c.rows != 1 || c.groups * c.igroups * c.sgroups != 1 || c.stages != 0)) ||
      (c.warps != 1 && c.warps != 2 && c.warps != 4) || (c.warps != 4 && (c.stages != 0 || c.cgroups > 1)) ||
      (c.flux != 0 && c.flux != 1) ||
      (c.flux == 1 && (which != 0 || c.rows != 1 || c.stages != 0 || c.cgroups != 1))) {
    set_error("sg_apply_config: rows in {1,2}; groups, igroups in [1,4]; sgroups in [1,8]; "
              "groups*igroups*sgroups <= 8; prefetch in [0,64]; min_blocks in [1,8]; FP64 families: rows 1; "
              "stages 0 or 2..8, staged only with one row and one group and prefetch >= 1; "
              "cgroups 1..16, split only with one row, one group and no staging; warps per group 1, 2 or 4, "
              "fewer than 4 only without staging or separate CTAs; flux (fine FP32 family only) with one row, "
              "no staging and no separate CTAs");
    return SG_ERR_ARG;
  }
  if (jit_smem_bytes(pr, c, which >= 2) > 200 * 1024) {
    set_error("sg_apply_config: the input-group hand-off does not fit in shared memory");
    return SG_ERR_ARG;
  }
  if (c.flux) SG_TRY(flux_build(pr));
  // recorded coarse-solve graphs reference the kernel about to be unloaded
  if (pr->jit[which] || (which == 0 && pr->flux_on != c.flux)) drop_recorded(pr);
  jit_free(pr, which);
  pr->jit_cfg[which] = c;
  pr->jit_cfg_set[which] = true;
  if (which == 0) pr->flux_on = c.flux;
  if (!jit_eligible(pr)) return SG_OK;
  return jit_apply_build(pr, which);
}

void jit_free(sg_problem* pr, int which) {
  if (!pr->jit[which]) return;
  if (pr->jit[which]->lib) cudaLibraryUnload(pr->jit[which]->lib);
  delete pr->jit[which];
  pr->jit[which] = nullptr;
}

bool jit_eligible(const sg_problem* pr) { return pr->P <= kJitMaxP && pr->T <= kJitMaxT; }

template <typename T>
static sg_status launch_kernel(cudaKernel_t kern, const JitConfig& c, size_t smem, const Ell& A, const T* X,
                               int64_t ldx, const T* F, int64_t ldf, T* Y, int64_t ldy, cudaStream_t st) {
  if (A.n == 0) return SG_OK;
  const T* V = sizeof(T) == 8 ? reinterpret_cast<const T*>(A.v64.ptr) : reinterpret_cast<const T*>(A.v32.ptr);
  const int* col = dp<int>(A.col);
  const int* vidx = dp<int>(A.vidx);
  long long ldr = A.ldr, lx = ldx, lf = ldf, ly = ldy, vkst = A.vkst;
  int n = int(A.n), S = A.S;
  void* args[] = {(void*)&V, (void*)&col, &ldr, &n, &S, (void*)&X, &lx, (void*)&F, &lf, (void*)&Y, &ly,
                  (void*)&vidx, &vkst};
  const bool cs = c.cgroups > 1;
  const int64_t rows_per_cta = 32LL * (cs ? 4 : c.warps) * c.rows;
  dim3 grid(unsigned((A.n + rows_per_cta - 1) / rows_per_cta * (cs ? c.cgroups : 1))),
      block(unsigned(cs ? 128 : 32 * c.warps * c.groups * c.igroups * c.sgroups));
  SG_CUDA(cudaLaunchKernel((const void*)kern, grid, block, args, smem, st));
  note_launch();
  return SG_OK;
}

sg_status jit_apply_launch(sg_problem* pr, int which, const Ell& A, const float* X, int64_t ldx, const float* F,
                           int64_t ldf, float* Y, int64_t ldy, cudaStream_t st) {
  SG_TRY(jit_apply_build(pr, which));
  const JitConfig& c = pr->jit_cfg[which];
  return launch_kernel<float>(pr->jit[which]->kern, c, jit_smem_bytes(pr, c, false), A, X, ldx, F, ldf, Y, ldy, st);
}

sg_status jit_apply_launch(sg_problem* pr, int which, const Ell& A, const double* X, int64_t ldx, const double* F,
                           int64_t ldf, double* Y, int64_t ldy, cudaStream_t st) {
  SG_TRY(jit_apply_build(pr, which));
  const JitConfig& c = pr->jit_cfg[which];
  return launch_kernel<double>(pr->jit[which]->kern, c, jit_smem_bytes(pr, c, true), A, X, ldx, F, ldf, Y, ldy, st);
}

// --------------------------------------------------------------------------
// Autotuner: compile the candidate tile shapes, time each on this problem's
// fine operator (median of a few launches after a warm-up, CUDA events),
// keep the fastest and remember the choice in the cache directory, keyed by
// the triple structure, n and the device name.
// --------------------------------------------------------------------------
// A short list of tile shapes per family, from sweeps on GB300: small P
// keeps the whole row in one thread (more prefetch helps); large P splits
// outputs and inputs over warp groups; the coarse family (a quarter of the
// rows) adds stencil-slot groups to fill the GPU.  Values staged through
// shared memory by 4-byte cp.async measured half the bandwidth of the
// register prefetch at 256^2 / P = 35 (0.144 ms against 0.071 ms), so the
// staged shapes are available through sg_apply_config but not tuned.  Groups
// of one warp (every slot its own group) measured slower everywhere except
// the fine FP64 family, where two output by two slot groups of one warp
// each beat the 4-warp shapes by 10 % at 256^2 / P = 35.  Slot groups alone
// share one generated body (0.0526 -> 0.0487 ms for the coarse family's two
// slot groups at 127^2 coarse rows, P = 35).
static std::vector<JitConfig> candidates(const sg_problem* pr, int which) {
  struct S7 {
    int r, g, i, s, pf, st, mb = 1, cg = 1, w = 4;
  };
  std::vector<S7> list;
  const bool fp64 = which >= 2;
  if (fp64) {
    // twice the register bytes per value: more output/input splitting, or
    // values staged through shared memory
    if (pr->P <= 48) {
      if (which == 2)
        list = {{1, 1, 1, 1, 16, 0}, {1, 1, 1, 1, 8, 0}, {1, 2, 1, 1, 16, 0}, {1, 1, 2, 1, 16, 0},
                {1, 2, 2, 1, 8, 0}, {1, 2, 1, 2, 8, 0, 1, 1, 1}};
      else
        list = {{1, 1, 1, 2, 16, 0}, {1, 1, 1, 4, 8, 0}, {1, 2, 1, 2, 8, 0}, {1, 1, 2, 2, 8, 0}};
    } else {
      list = {{1, 1, 1, 1, 8, 0, 1, 4}, {1, 1, 1, 1, 8, 0, 1, 6}, {1, 1, 1, 1, 8, 0, 1, 8},
              {1, 1, 1, 1, 4, 0, 1, 6}};
    }
  } else if (pr->P <= 48) {
    if (which == 0)
      list = {{1, 1, 1, 1, 32, 0}, {1, 1, 1, 1, 16, 0}, {1, 1, 2, 1, 16, 0}, {1, 2, 1, 1, 16, 0}};
    else
      list = {{1, 1, 1, 1, 32, 0}, {1, 1, 1, 2, 32, 0}, {1, 1, 1, 4, 16, 0}, {1, 1, 1, 2, 16, 0},
              {1, 2, 1, 2, 16, 0}};
  } else {
    list = {{1, 1, 1, 1, 8, 0, 1, 3}, {1, 1, 1, 1, 8, 0, 1, 4}, {1, 1, 1, 1, 16, 0, 1, 4},
            {1, 1, 1, 1, 8, 0, 1, 6}, {1, 1, 1, 1, 4, 0, 1, 8}};
  }
  std::vector<JitConfig> out;
  for (const S7& e : list) {
    JitConfig c;
    c.rows = e.r;
    c.groups = e.g;
    c.igroups = e.i;
    c.sgroups = e.s;
    c.prefetch = e.pf;
    c.stages = e.st;
    c.min_blocks = e.mb;
    c.cgroups = e.cg;
    c.warps = e.w;
    if (jit_smem_bytes(pr, c, fp64) > 200 * 1024) continue;
    out.push_back(c);
  }
  // the fine FP32 family also in the edge-flux form (one row per thread,
  // no staging, no separate CTAs)
  if (which == 0 && !fp64 && pr->flux_allowed) {
    const size_t nslot = out.size();
    for (size_t i = 0; i < nslot; ++i) {
      JitConfig c = out[i];
      if (c.rows != 1 || c.stages != 0 || c.cgroups != 1) continue;
      c.flux = 1;
      out.push_back(c);
    }
  }
  if (out.empty()) out.push_back(jit_default_config(pr, which));
  return out;
}

static std::string tune_key(const sg_problem* pr, const Ell& A, bool fp64) {
  cudaDeviceProp prop{};
  cudaGetDeviceProperties(&prop, pr->device);
  std::ostringstream os;
  os << prop.name << "|v" << kJitGeneratorVersion << "|" << pr->P << "|" << pr->K << "|" << pr->T << "|" << A.n << "|"
     << A.S << (fp64 ? "|f64" : "");
  for (int64_t t = 0; t < pr->T; ++t) os << "," << pr->kab[3 * t] << ":" << pr->kab[3 * t + 1] << ":" << pr->kab[3 * t + 2];
  char key[32];
  std::snprintf(key, sizeof key, "%016llx", (unsigned long long)fnv1a(os.str()));
  return key;
}

sg_status jit_autotune(sg_problem* pr, int which, int force, double* best_ms) {
  if (!jit_eligible(pr)) {
    set_error("sg_apply_autotune: the specialised kernel is not available for this size");
    return SG_ERR_UNSUPPORTED;
  }
  const bool coarse = which % 2 == 1, fp64 = which >= 2;
  if (coarse && !pr->solver) {
    set_error("sg_apply_autotune: the coarse operator exists after sg_precond_setup");
    return SG_ERR_ARG;
  }
  const Ell& A = coarse ? coarse_ell(pr) : pr->fine;
  const std::string path = cache_dir() + "/tune_" + tune_key(pr, A, fp64) + (pr->flux_allowed ? "_fx" : "") + ".txt";
  if (!force) {
    std::ifstream in(path);
    JitConfig c;
    double ms = 0;
    if (in >> c.rows >> c.groups >> c.igroups >> c.sgroups >> c.prefetch >> c.min_blocks >> c.stages >> c.cgroups >>
        c.warps >> c.flux >> ms) {
      if (best_ms) *best_ms = ms;
      return jit_configure(pr, which, c);
    }
  }
  const int64_t len = int64_t(pr->P) * std::max<int64_t>(pr->ld, A.ldr);
  const size_t esz = fp64 ? 8 : 4;
  DevBuf X, Y;
  SG_TRY(X.alloc(len * esz));
  SG_TRY(Y.alloc(len * esz));
  cudaStream_t st;
  SG_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  cudaEvent_t e0, e1;
  SG_CUDA(cudaEventCreate(&e0));
  SG_CUDA(cudaEventCreate(&e1));
  JitConfig best = jit_default_config(pr, which);
  double best_t = 1e30;
  sg_status status = SG_OK;
  for (const JitConfig& c : candidates(pr, which)) {
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kern = nullptr;
    if (c.flux && flux_build(pr) != SG_OK) continue;
    if (jit_compile(jit_apply_source(pr, c, fp64), &lib, &kern, nullptr, nullptr, pr->device, fp64) != SG_OK) continue;
    const size_t sm = jit_smem_bytes(pr, c, fp64);
    const Ell& Ac = c.flux ? pr->flux : A;
    auto run = [&]() {
      return fp64 ? launch_kernel<double>(kern, c, sm, Ac, dp<double>(X), A.ldr, nullptr, 0, dp<double>(Y), A.ldr, st)
                  : launch_kernel<float>(kern, c, sm, Ac, dp<float>(X), A.ldr, nullptr, 0, dp<float>(Y), A.ldr, st);
    };
    std::vector<float> ts;
    for (int rep = 0; rep < 7 && status == SG_OK; ++rep) {
      status = run();
      if (status != SG_OK) break;
      if (rep < 2) continue;
      cudaEventRecord(e0, st);
      run();
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
  if (out)
    out << best.rows << " " << best.groups << " " << best.igroups << " " << best.sgroups << " " << best.prefetch
        << " " << best.min_blocks << " " << best.stages << " " << best.cgroups << " " << best.warps << " " << best.flux
        << " " << best_t << "\n";
  return jit_configure(pr, which, best);
}

}  // namespace sg
