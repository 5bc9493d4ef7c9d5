// Internal declarations of libsg (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "sg.h"

namespace sg {

void set_error(const std::string& msg);
// process-wide count of kernel launches made by the library
void note_launch();
// adds n (possibly negative) to the launch count: kernels executed inside
// graphs, minus kernel nodes counted while a graph was being recorded
void note_launches(int64_t n);
int64_t launch_count();
int64_t launch_count();

#define SG_CUDA(call)                                                                    \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      ::sg::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));               \
      return SG_ERR_CUDA;                                                                \
    }                                                                                    \
  } while (0)

#define SG_TRY(call)                    \
  do {                                  \
    sg_status s_ = (call);              \
    if (s_ != SG_OK) return s_;         \
  } while (0)

#define SG_ARG(cond, msg)               \
  do {                                  \
    if (!(cond)) {                      \
      ::sg::set_error(msg);             \
      return SG_ERR_ARG;                \
    }                                   \
  } while (0)

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Device buffer owned by a handle.
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : ptr(o.ptr), bytes(o.bytes) {
    o.ptr = nullptr;
    o.bytes = 0;
  }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) {
      free_();
      ptr = o.ptr;
      bytes = o.bytes;
      o.ptr = nullptr;
      o.bytes = 0;
    }
    return *this;
  }
  ~DevBuf() { free_(); }
  sg_status alloc(size_t nbytes);
  void free_();
  template <typename T> T* as() const { return static_cast<T*>(ptr); }
};

template <typename T> inline T* dp(const DevBuf& b) { return static_cast<T*>(b.ptr); }

// ELL ("sliced by slot") storage of a family of K matrices sharing one
// pattern with at most S entries per row: col[s * ldr + r] and
// val[(k * S + s) * ldr + r].  Padding entries carry col = r, value 0.
struct Ell {
  int S = 0;
  int64_t n = 0, ldr = 0;
  DevBuf col;      // int32 S x ldr
  DevBuf v64;      // double K x S x ldr
  DevBuf v32;      // float  K x S x ldr
  // edge-flux form (fine FP32 operator only): col[s * ldr + r] is the
  // neighbour across edge s of row r or -1 (a Dirichlet node), vidx[s * ldr
  // + r] the offset of that edge's conductance within a term's block, the
  // conductances of term k at v32[k * vkst + vidx]
  DevBuf vidx;     // int32 S x ldr
  int64_t vkst = 0;
};

// The Galerkin operator summed per stencil edge into its P x P block (FP64),
//   C_ab^{r,s} = sum_k g_kab v_k^{r,s}   (symmetric: a <= b stored, packed
//   row by row), layout [S][npair][ldr]; built on demand for FP64 applies.
struct AsmBlocks {
  int npair = 0;
  bool tried = false;  // the policy was applied (built or declined)
  DevBuf c;
};

// The fine operator in the edge-flux form with each edge's P x P block
// summed once, B_ab^e = sum_k g_kab w_k(e) (symmetric: a <= b stored,
// packed row by row), each entry split into two FP32 numbers hi + lo;
// layout [npair][lde].  A row of the operator is sum over its four edges of
// B^e (x_r - x_neighbour), the neighbour's term dropped on the Dirichlet
// boundary.  Built on demand for the refinement residuals.
struct FluxDf {
  int npair = 0;
  int64_t lde = 0;
  bool tried = false;  // the policy was applied (built or declined)
  DevBuf b;            // float2 [npair][lde]
  DevBuf xs;           // float2 [P][ldr]: the split iterate
};

struct SolverState;
void solver_free(sg_problem* pr);
struct NewtonWork;
void newton_free(sg_problem* pr);
struct Cnn;
void cnn_free(sg_problem* pr);

// Triple products re-ordered by output mode a, then k, then b, split into
// chunks of input terms [c*kc, (c+1)*kc) for the shared-memory apply.
struct TripleTables {
  int kc = 0, nchunk = 0;
  DevBuf tk, tb;   // int32 T
  DevBuf g64, g32; // T
  DevBuf off;      // int32 P x (nchunk + 1)
};

// Optional per-launch timing (bench mode): CUDA events bracket each launch
// or phase on its stream; read() sums the elapsed times per kind.  Kernel
// kinds: 0 fine apply FP32, 1 fine apply FP64, 2 coarse apply FP32, 3
// coarse apply FP64, 4 RAS local solve FP32, 5 RAS local solve FP64.
// Phase kinds of the host-driven solve (a phase holds the kernels it
// launches, so kinds 4 and 5 lie inside kind 6): 6 smoother, 7 coarse
// correction (restriction, coarse GMRES graph, interpolation), 8 Arnoldi
// step (Gram-Schmidt, Givens rotation, normalisation), 9 refinement step
// bookkeeping (FP64 residual norm, conversion to FP32, the update of x).
constexpr int kProfKinds = 10;
struct Profiler {
  bool on = false;
  struct Rec {
    cudaEvent_t a = nullptr, b = nullptr;
    int kind = 0;
  };
  std::vector<Rec> pool;
  size_t used = 0;
  sg_status begin(int kind, cudaStream_t st, size_t& slot);
  sg_status end(size_t slot, cudaStream_t st);
  sg_status read(int kind, int64_t* launches, double* ms);
  void reset() { used = 0; }
  ~Profiler();
};

// Brackets a phase with profiler events when the profiler is on (errors of
// the event calls are ignored: timing never fails a solve).
struct ProfScope {
  Profiler* p;
  cudaStream_t st;
  size_t slot = 0;
  bool on;
  ProfScope(Profiler* p_, int kind, cudaStream_t st_) : p(p_), st(st_), on(p_ && p_->on) {
    if (on && p->begin(kind, st, slot) != SG_OK) on = false;
  }
  void stop() {
    if (on) p->end(slot, st);
    on = false;
  }
  ~ProfScope() { stop(); }
};

// Register-specialised apply compiled at setup time (sg_jit.cpp).  Four
// families: which = 0 fine FP32, 1 coarse FP32, 2 fine FP64, 3 coarse FP64.
constexpr int kJitFamilies = 4;
constexpr int kJitMaxP = 128;
constexpr int kJitGeneratorVersion = 10;  // bump when the generated code changes
constexpr int64_t kJitMaxT = 40000;
struct JitConfig {
  int rows = 1;        // rows per thread (2: paired FP32 FMA)
  int groups = 1;      // output groups (warp groups of 4 warps)
  int igroups = 1;     // input groups (partial sums meet in shared memory)
  int sgroups = 1;     // stencil-slot groups (partial sums meet in shared memory)
  int prefetch = 8;    // input terms loaded ahead
  int min_blocks = 1;  // CTAs per SM requested from the register allocator
  int stages = 0;      // 0: matrix values prefetched into registers; >= 2: staged through shared
                       // memory by cp.async in blocks of `prefetch` terms, stages - 1 blocks ahead
  int cgroups = 1;     // output groups as separate 128-thread CTAs (no register cap from wide CTAs)
  int warps = 4;       // warps per group (rows per group = 32 x warps x rows): narrow groups keep
                       // several slot or input groups within one register-rich CTA
  int flux = 0;        // 1: edge-flux form (fine FP32 family): y_r = sum over the four edges of
                       // sum_k w_k G_k (x_r - x_neighbour), conductances stored once per edge
};
struct JitApply {
  cudaLibrary_t lib = nullptr;
  cudaKernel_t kern = nullptr;
  bool from_cache = false;
  double compile_s = 0.0;
};

}  // namespace sg

struct sg_problem {
  int device = 0;
  int N = 0, L = 0, p = 0, q = 0, P = 0, K = 0;
  int64_t n = 0, nnzA = 0, T = 0, E = 0;
  double sigma2 = 0, bx = 0, by = 0, g0 = 0;
  std::vector<int32_t> mi_out, mi_in;  // P x L, K x L
  std::vector<int32_t> kab;            // T x 3, ordered k, a, b
  std::vector<int64_t> num;            // T
  std::vector<double> g;               // T
  std::vector<double> gfield;          // L x E
  std::vector<int32_t> rowptr, colidx; // shared CSR pattern
  std::vector<double> b;               // load vector (n)
  std::vector<double> a0;              // A_0 values on the CSR pattern (host)

  sg::Ell fine;                        // A_k on the device
  sg::TripleTables tri;
  int64_t ld = 0;                      // internal leading dimension of blocks
  sg::SolverState* solver = nullptr;   // preconditioner + solver workspaces
  sg::Cnn* cnn = nullptr;              // learned smoother network
  sg::NewtonWork* nl = nullptr;        // nonlinear problem: coefficients, operators, triple lists
  sg::DevBuf gfield_dev;               // KL modes at the element centroids (sampled solves)
  sg::Profiler prof;
  sg::JitApply* jit[sg::kJitFamilies] = {};     // specialised apply per family (fine/coarse x f32/f64)
  sg::JitConfig jit_cfg[sg::kJitFamilies];
  bool jit_cfg_set[sg::kJitFamilies] = {};
  sg::DevBuf mdot_partial, mdot_counter;  // scratch of sg_mdot
  int apply_mode = 0;                  // 0 auto, 1 shared-memory kernel, 2 specialised
  sg::AsmBlocks asm_fine;              // assembled FP64 blocks of the fine operator
  sg::Ell flux;                        // edge-flux form of the fine operator (FP32 conductances)
  int flux_on = 0;                     // fine FP32 applies use the edge-flux form
  bool flux_allowed = true;            // the autotuner may choose the edge-flux form
  int wait_limit = 1 << 22;            // mbarrier polls of a tcgen05 completion wait
  int asm_mode = 0;                    // FP64 applies: 0 auto, 1 never assembled, 2 always
  sg::FluxDf fdf;                      // double-FP32 edge blocks of the fine operator
  int res_mode = 0;                    // refinement residuals: 0 auto, 1 FP64 applies, 2 double-FP32 edge blocks
};

namespace sg {
// setup helpers (sg_setup.cpp)
std::vector<int32_t> multi_indices(int L, int p);
// <He_a He_b He_c> (integer, textbook linearisation formula)
int64_t he_triple_1d(int a, int b, int c);
sg_status build_host(sg_problem* pr, const sg_kl_desc* kl);
// device assembly (sg_assemble.cu)
sg_status assemble_fine(sg_problem* pr);
// lognormal input coefficients c_bar_k(e) of terms [k0, k0 + kn) at every
// element, written as out[(k - k0) E + e] (FP64 device array); synchronous
sg_status element_coefficients(sg_problem* pr, int k0, int kn, double* out, cudaStream_t st);
// edge-flux form of the fine operator: neighbours, offsets and the FP32
// conductances of every input term on every edge (allocated on first use)
sg_status flux_build(sg_problem* pr);
// the edge conductances of every input term in FP64, w[k * vkst + e] (the
// edge numbering of the edge-flux form); synchronous
sg_status flux_values64(sg_problem* pr, double* w, int64_t vkst);
sg_status build_triple_tables(sg_problem* pr, TripleTables& t, int S);
// apply (sg_apply.cu)
template <typename T>
sg_status apply_ell(const Ell& A, const TripleTables& tri, int P, int K, const T* X, int64_t ldx,
                    const T* F, int64_t ldf, T* Y, int64_t ldy, cudaStream_t st);
std::string jit_apply_source(const sg_problem* pr, const JitConfig& c, bool fp64 = false);
JitConfig jit_default_config(const sg_problem* pr, int which);
size_t jit_smem_bytes(const sg_problem* pr, const JitConfig& c, bool fp64 = false);
sg_status jit_autotune(sg_problem* pr, int which, int force, double* best_ms);
sg_status jit_apply_build(sg_problem* pr, int which);
void jit_free(sg_problem* pr, int which);
sg_status jit_configure(sg_problem* pr, int which, const JitConfig& c);
bool jit_eligible(const sg_problem* pr);
sg_status jit_apply_launch(sg_problem* pr, int which, const Ell& A, const double* X, int64_t ldx, const double* F,
                           int64_t ldf, double* Y, int64_t ldy, cudaStream_t st);
sg_status jit_apply_launch(sg_problem* pr, int which, const Ell& A, const float* X, int64_t ldx, const float* F,
                           int64_t ldf, float* Y, int64_t ldy, cudaStream_t st);
// assembled FP64 blocks (sg_apply.cu): build per the problem's policy (no-op
// once tried; never while `st` is capturing), and the apply over them
sg_status asm_prepare(sg_problem* pr, const Ell& A, AsmBlocks& B, cudaStream_t st);
// (k, g_kab) list of every packed pair a <= b (pair index a P - a (a - 1) / 2
// + b - a): pair q owns entries [pptr[q], pptr[q + 1]) of pk, pg
void pair_lists(const sg_problem* pr, std::vector<int>& pptr, std::vector<int>& pk, std::vector<double>& pg);
// refinement residuals (sg_resid_df.cu): the double-FP32 edge blocks built
// per the problem's policy (no-op once tried; never while `st` is
// capturing), and R = F - A X (FP64 in and out) over them, or with the FP64
// apply when they are not built
sg_status resid_prepare(sg_problem* pr, cudaStream_t st);
sg_status resid_df(sg_problem* pr, const double* F, int64_t ldf, const double* X, int64_t ldx, double* R,
                   int64_t ldr, cudaStream_t st);
sg_status refine_residual(sg_problem* pr, const double* F, int64_t ldf, const double* X, int64_t ldx, double* R,
                          int64_t ldr, cudaStream_t st);
sg_status apply_asm64(const sg_problem* pr, const Ell& A, const AsmBlocks& B, const double* X, int64_t ldx,
                      const double* F, int64_t ldf, double* Y, int64_t ldy, cudaStream_t st);
// the operator apply without timing: assembled blocks (FP64, when built),
// else the specialised kernel, else the shared-memory kernel
template <typename T>
sg_status apply_any(sg_problem* pr, bool coarse, const T* X, int64_t ldx, const T* F, int64_t ldf, T* Y,
                    int64_t ldy, cudaStream_t st);
// apply_ell on the fine (coarse = false) or coarse family of a problem,
// timed when the problem's profiler is on
template <typename T>
sg_status apply_op(sg_problem* pr, bool coarse, const T* X, int64_t ldx, const T* F, int64_t ldf, T* Y,
                   int64_t ldy, cudaStream_t st);
}  // namespace sg
