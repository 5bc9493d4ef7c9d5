// Internal declarations of the preconditioner and Krylov solvers.
#pragma once

#include "sg_internal.h"

namespace sg {

// Generic CSR matrix on the device (FP64 and FP32 values).
struct DevCsr {
  int64_t n = 0, m = 0, nnz = 0;  // rows, cols, entries
  DevBuf rowptr, col, v64, v32;
  sg_status upload(int64_t rows, int64_t cols, const std::vector<int32_t>& rp,
                   const std::vector<int32_t>& ci, const std::vector<double>& v);
  void free_() {
    rowptr.free_();
    col.free_();
    v64.free_();
    v32.free_();
  }
};

// One level of the smoothed-aggregation hierarchy.
struct AmgLevel {
  int64_t n = 0, ld = 0;
  DevCsr A, Pm, R;        // operator, prolongation (n x n_next), restriction
  DevBuf dinv64, dinv32;  // 1 / l1 row norms
  // host copies for tests
  std::vector<int32_t> agg;
};

// Smoothed-aggregation hierarchy: levels plus the explicit FP64 inverse of
// the coarsest matrix.
struct AmgHier {
  std::vector<AmgLevel> lev;
  DevBuf coarsest_inv64;
  bool fused = true;  // V-cycle: lane groups per sparse row, Jacobi steps folded into the products
  size_t size() const { return lev.size(); }
  AmgLevel& operator[](size_t l) { return lev[l]; }
  const AmgLevel& operator[](size_t l) const { return lev[l]; }
};

// Restricted additive Schwarz data: per box, block-tridiagonal (line)
// Cholesky factors of the local mean block, stored as explicit inverses of
// the diagonal blocks and the sub-diagonal blocks, padded to wmax x wmax.
struct RasData {
  int nbox = 0, wmax = 0, lmax = 0;
  double flops_per_mode = 0.0;             // useful flops of one local solve per PCE mode
  std::vector<int32_t> nlines;             // per box
  std::vector<std::vector<int32_t>> idx;   // per box: ascending global indices
  std::vector<std::vector<int32_t>> owned; // per box: 1 if owned
  DevBuf d_nlines;                         // int32 nbox
  DevBuf d_gidx;                           // int32 nbox x lmax x wmax (-1 pad, owned | 1<<30)
  DevBuf linv64, loff64, linv32, loff32;   // nbox x lmax x wmax x wmax
  // explicit local inverses (ras_kernel 2): the owned rows of A_{0,i}^{-1}
  // in FP32 as chunks of 128 rows x 32 overlapped nodes in the tensor-core
  // operand layout (tiles of 128 owned rows in box order, chunks in node
  // order), the buffer of the packed residual, the index tables (offsets in
  // ints into d_inv_meta, InvMeta order) and a timeout flag
  int inv_kp = 0, inv_n = 0, inv_p = 0, inv_ntiles = 0, inv_grid = 0, inv_nsplit = 0, inv_stages = 0;
  int64_t inv_chunks = 0, inv_bchunks = 0;
  int64_t inv_off[10] = {};
  DevBuf d_inv, d_inv_meta, d_inv_bpack, d_inv_err;
  void inv_free() {
    d_inv.free_();
    d_inv_meta.free_();
    d_inv_bpack.free_();
    inv_chunks = 0;
  }
};

// Coarse 2h space: interpolation R_0^T and the coarse Galerkin operator.
struct CoarseData {
  int Nc = 0;
  int64_t nc = 0, ldc = 0;
  std::vector<int32_t> rowptr, colidx;     // coarse CSR pattern (host)
  Ell ell;                                 // coarse A_k in ELL form (device)
  TripleTables tri;
  DevCsr RT, R;                            // interpolation (n x nc) and restriction
  AsmBlocks asm_c;                         // assembled FP64 blocks of the coarse operator
};

// Smoother inputs recorded during solves: the training residuals of the
// learned smoother.  pool holds cap blocks of P x ld FP32 values.
struct Harvest {
  bool on = false;
  int64_t cap = 0, count = 0;
  DevBuf pool;
};

struct Precond {
  bool ready = false;
  int sx = 0, sy = 0, overlap = 0;
  double omega = 1.0;
  double inner_rtol = 1e-5;
  int inner_max = 100, inner_restart = 30;
  int inner_passes = 1;  // Gram-Schmidt passes of the coarse GMRES
  int ras_modes = 0;                       // modes per CTA of the RAS kernel (0 automatic)
  int ras_stages = 0;                      // depth of its ring of line matrices (0 automatic)
  int ras_kernel = 0;                      // 0: FMA kernel; 1: tensor cores for FP32 data (line
                                           // recurrence); 2: explicit local inverses on tcgen05
  int wait_limit = 1 << 22;                // mbarrier polls of a tcgen05 completion wait
  RasData ras;
  CoarseData co;
  AmgHier amg;                             // on the coarse mean operator
  std::vector<double> gt;                  // Kronecker factor G~ (P x P), host
  DevBuf gtinv64, gtinv32;                 // omega * G~^{-1} (P x P)
  DevBuf gkron64, gkron32;                 // G~^{-1} (coarse AMG preconditioner)
  std::vector<double> ginv;                // G~^{-1}, host
  // learned smoother: S r = omega_cnn (G~^{-1} (x) I) CNN(r)
  int smoother = 0;                        // 0 RAS, 1 learned
  bool use_cnn = false;                    // learned smoother active in the current solve
  double omega_cnn = 1.0;
  DevBuf gtcnn64, gtcnn32;                 // omega_cnn * G~^{-1}
  Harvest harvest;
  int inner_its_last = 0, inner_its_total = 0, inner_calls = 0;
  bool device_loops = true;                // coarse GMRES as one CUDA graph launch
  int last_coarse_dtype = -1;              // 0 FP64, 1 FP32: context of the last graph solve
};

// For every coarse ELL position (s * ldc + I): the fine ELL positions
// (s * ldr + f) and weights whose sum is the entry of R_0 A R_0^T.
struct CoarsePlan {
  std::vector<int32_t> rp;
  std::vector<int64_t> src;
  std::vector<double> w;
};

sg_status precond_setup_host(sg_problem* pr, Precond& pc);
// smoothed-aggregation hierarchy of the fine mean matrix A_0 (training
// targets of the learned smoother)
sg_status amg_setup_fine(const sg_problem* pr, AmgHier& h);
const Ell& coarse_ell(const sg_problem* pr);
const TripleTables& coarse_tri(const sg_problem* pr);
AsmBlocks& coarse_asm(sg_problem* pr);
// drops the solver contexts and their recorded graphs after a change of
// apply kernel (recorded batches of the problem then refuse to run)
void drop_recorded(sg_problem* pr);
sg_status precond_setup_coarse_plan(sg_problem* pr, Precond& pc, const CoarsePlan& plan);
sg_status precond_setup_device(sg_problem* pr, Precond& pc, double omega_opt, cudaStream_t st);
void precond_free(Precond& pc);

}  // namespace sg
