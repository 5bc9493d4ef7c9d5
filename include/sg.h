/*
 * libsg -- stochastic Galerkin (SG) solver for the linear stochastic Poisson
 * problem  -div(c(x, xi) grad u) = 1  on the unit square, u = 0 on the
 * boundary, with a lognormal coefficient c = exp(g), g a Gaussian field with
 * the separable exponential covariance of Sec. 2.1 (Eqs. KLE, CovarKer2DNLP),
 * expanded in a Hermite polynomial chaos (Eqs. inputpc, inputlogn, outpc) and
 * projected onto the chaos (Eq. Galerkin_L_exp).  The coupled system
 *
 *        sum_k  A_k X G_k^T = F,      G_k[a][b] = <psi_k psi_a psi_b>,
 *
 * is solved by flexible GMRES preconditioned by the two-level restricted
 * additive Schwarz cycle of Sec. 3 (Eqs. RASsto, coarse, RAS_2L).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Chaos basis: orthonormal probabilists' Hermite polynomials
 *   psi_alpha = prod_i He_{alpha_i}(xi_i) / sqrt(alpha_i!).  The paper's
 *   coefficient u_bar_a equals X[:, a] / sqrt(alpha_a!).
 * - Multi-index order: total degree ascending, then lexicographically
 *   descending in (alpha_1, ..., alpha_L).
 * - Mesh: N x N cells of size h = 1/N, each split by the "/" diagonal into
 *   two right triangles, P1 elements, coefficient constant per triangle
 *   (evaluated at its centroid).  Interior node (i, j), 1 <= i, j <= N-1, has
 *   number r = (j-1)(N-1) + (i-1); n = (N-1)^2.
 * - Blocks of PCE coefficients (X, Y, F) are MODE-MAJOR device arrays:
 *   entry (node r, mode a) lives at X[a * ld + r], ld >= n.
 * - Device pointers belong to the caller; the library never frees them.
 *   The handle owns every buffer it allocates (in sg_setup and
 *   sg_precond_setup) and frees them in sg_destroy.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Work is enqueued on it; calls return without waiting unless
 *   stated otherwise.
 * - Errors are returned as sg_status codes; no exception crosses the ABI.
 *   sg_last_error() returns a thread-local message for the last failure.
 *   A handle is not thread-safe: one host thread at a time.
 * - Errors every entry point shares, unless its comment says otherwise:
 *   SG_ERR_ARG for a NULL handle or a NULL pointer it needs, a leading
 *   dimension below n, an index out of range, or a call made before the
 *   setup it depends on (sg_precond_setup, weights of the learned smoother);
 *   SG_ERR_NOMEM when a device or host allocation fails; SG_ERR_CUDA when a
 *   CUDA call fails (the message names it).  Getters have no other errors.
 * - Entry points marked "plumbing" (tile shapes, profiling, launch counts,
 *   kernel selection) have no counterpart in the paper; those of the learned
 *   smoother and of batching come from the method statement, not the paper.
 */
#ifndef SG_H_
#define SG_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sg_problem sg_problem;

typedef enum {
  SG_OK = 0,
  SG_NOT_CONVERGED = 1,     /* solver hit max_it; best iterate written  */
  SG_ERR_ARG = -1,          /* bad argument (NULL, size, ld, order ...) */
  SG_ERR_CUDA = -2,         /* a CUDA runtime call failed               */
  SG_ERR_NOMEM = -3,        /* device or host allocation failed         */
  SG_ERR_BREAKDOWN = -4,    /* non-finite value inside the solver       */
  SG_ERR_TIMEOUT = -5,      /* a bounded device wait ran out            */
  SG_ERR_UNSUPPORTED = -6   /* feature not available in this build      */
} sg_status;

typedef enum { SG_F64 = 0, SG_F32 = 1 } sg_dtype;

/* Structured unit-square mesh: N cells per side (N >= 2, even when a
 * preconditioner with a coarse grid is set up). */
typedef struct {
  int N;
} sg_mesh_desc;

/* Gaussian field g = g0 + sum_{i<L} g_i xi_i (Sec. 2.1, Eq. KLE).
 * Analytic KL modes of sigma2 * exp(-|dx|/bx - |dy|/by) are used unless
 * user_modes is given: then it holds L x (2 N^2) values g_i(e) per triangle e
 * (element id 2 (j N + i) for the lower and 2 (j N + i) + 1 for the upper
 * triangle of cell (i, j)), sqrt(lambda_i) included; it is copied. */
typedef struct {
  double sigma2, bx, by, g0;
  int L;
  const double* user_modes;
} sg_kl_desc;

/* Build the SG system (Sec. 2.1): KL modes at triangle centroids, output
 * multi-indices of degree <= p_out (P terms), input multi-indices of degree
 * <= q_in (K terms), the nonzero triple products, the lognormal input
 * coefficients, and the K stiffness matrices A_k on one shared CSR pattern
 * (the pattern of A_0 with exact zeros dropped; every A_k is stored on it).
 * The matrices are assembled on the current CUDA device in FP64 and FP32.
 * Errors: SG_ERR_ARG for N < 2, L < 0, p_out < 0, q_in < 0 or NULL pointers;
 * SG_ERR_NOMEM / SG_ERR_CUDA on allocation or launch failure. */
sg_status sg_setup(const sg_mesh_desc* mesh, const sg_kl_desc* kl, int p_out, int q_in,
                   sg_problem** out);

/* Frees every buffer the handle owns.  NULL is accepted. */
sg_status sg_destroy(sg_problem* prob);

/* Sizes: n interior nodes, P output terms, K input terms, nnzA entries of
 * the shared pattern, T nonzero triple products.  Any pointer may be NULL. */
sg_status sg_get_sizes(const sg_problem* prob, int64_t* n, int* P, int* K, int64_t* nnzA,
                       int64_t* T);

/* Multi-index table, row-major: which = 0 gives the P x L output set,
 * which = 1 the K x L input set.  `out` is host memory of that size. */
sg_status sg_get_multi_indices(const sg_problem* prob, int32_t* out, int which);

/* Triple products <psi_k psi_a psi_b> != 0 ordered by k, a, b
 * (Eq. Galerkin_L_exp): kab is host T x 3, num is host T (unnormalised
 * integer prod_i <He_{k_i} He_{a_i} He_{b_i}>), g is host T (orthonormal
 * value num / sqrt(k! a! b!)).  num or g may be NULL. */
sg_status sg_get_triples(const sg_problem* prob, int32_t* kab, int64_t* num, double* g);

/* Fourfold products <psi_i psi_j psi_k psi_l> != 0 of the nonlinear problem
 * (Sec. 2.2, the t_ijkl of Eq. stonlp_system): i over the input set
 * (degree q), j, k, l over the output set (degree p), ordered by i, j, k, l
 * in the multi-index order of sg_get_multi_indices.  Host-only: needs no
 * handle and no GPU.  Call with ijkl = num = t = NULL to get *count; then
 * with *count = the capacity: ijkl (host count x 4), num (unnormalised
 * integer prod over dimensions of <He He He He>) and t (orthonormal value
 * num / sqrt(i! j! k! l!)), each optional; *count receives the number.
 * Errors: SG_ERR_ARG (NULL count; L outside 1..12, p outside 0..8, q
 * outside 0..16; capacity too small), SG_ERR_UNSUPPORTED (an integer beyond
 * 64 bits). */
sg_status sg_fourfold_products(int L, int p, int q, int64_t* count, int32_t* ijkl, int64_t* num, double* t);

/* Shared CSR pattern on the host: rowptr n+1, colidx nnzA, columns ascending. */
sg_status sg_get_csr(const sg_problem* prob, int32_t* rowptr, int32_t* colidx);

/* Values of A_k on the shared pattern (FP64, host array K x nnzA, CSR order),
 * copied back from the device; for tests and small problems. */
sg_status sg_get_values(const sg_problem* prob, double* vals);

/* Load vector F = b e_0^T (b_r = integral of the hat function, f = 1,
 * Eq. Galerkin_L_exp with <psi_k> = delta_k0), written as a mode-major
 * FP64 device block with leading dimension ld (all modes a >= 1 zeroed). */
sg_status sg_get_rhs(const sg_problem* prob, double* F_dev, int64_t ld, void* stream);

/* Galerkin operator apply (Eq. Galerkin_L_exp in Kronecker form):
 *     Y = sum_k A_k X G_k^T,   y_r[a] = sum_{c} sum_{(k,a,b)} v_k^{rc} g_kab x_c[b].
 * dtype selects FP64 (double X, Y, FP64 values) or FP32 (float X, Y, FP32
 * values, FP32 accumulation).  X and Y are mode-major device blocks with
 * leading dimensions ldx, ldy >= n; X and Y must not overlap.
 * Errors: SG_ERR_ARG (NULL, ld < n, overlap), SG_ERR_CUDA (launch). */
sg_status sg_apply(sg_problem* prob, sg_dtype dtype, const void* X_dev, int64_t ldx, void* Y_dev,
                   int64_t ldy, void* stream);

/* Kernel used by the applies of this handle (fine and coarse, FP32 and
 * FP64):
 *   0 auto (default): the register-specialised kernel when P <= 128 and
 *     T <= 40000, else the shared-memory kernel;
 *   1 the shared-memory kernel (any size);
 *   2 the register-specialised kernel (SG_ERR_UNSUPPORTED if too large).
 * The specialised kernel is generated from the triple list, compiled for
 * sm_103a with NVRTC on first use and cached on disk (SG_JIT_CACHE, default
 * ~/.cache/sg_gb300); this call compiles it now when it will be used.
 * Errors: SG_ERR_CUDA with the compiler log when compilation fails. */
sg_status sg_set_apply_kernel(sg_problem* prob, int mode);

/* FP64 applies (Sec. 2.1, Eq. Galerkin_L_exp) over assembled blocks: the K
 * values of each stencil edge summed once into its symmetric P x P block,
 * C_ab = sum_k g_kab v_k (P (P + 1) / 2 doubles per edge, S per row), so an
 * FP64 apply costs P^2 FMAs per edge instead of two FP64 operations per
 * triple (GB300's FP64 units bound the FP64 applies).  mode 0 (default):
 * built on the first FP64 apply of the fine and of the coarse operator
 * when the blocks take at most a quarter of the free device memory; 1:
 * never (the generated or shared-memory kernel); 2: always, built now
 * (SG_ERR_NOMEM when they do not fit).  A change drops the recorded
 * coarse-solve graphs (rebuilt on the next solve); recorded batches of this
 * problem then refuse to run.  FP32 applies are unaffected. */
sg_status sg_set_apply_fp64(sg_problem* prob, int mode);

/* Whether the fine and the coarse FP64 applies use assembled blocks (0/1)
 * and the device bytes the blocks hold.  Any pointer may be NULL. */
sg_status sg_apply_fp64_info(const sg_problem* prob, int* fine, int* coarse, int64_t* bytes);

/* How the FP64 residuals of the mixed-precision refinement (sg_solve mode
 * 1, recorded solves and batches of mode 1, sg_residual_refine) are formed
 * (Sec. 2.1, Eq. Galerkin_L_exp, in the edge form: a row of A_k is the sum
 * over the four edges of its node of w_k(e) (x_r - x_neighbour), so
 *     R_r = F_r - sum_e B^e (x_r - x_c(e)),   B^e_ab = sum_k g_kab w_k(e)).
 * mode 0 (default): in double-FP32 arithmetic over the edge blocks B^e,
 * summed once in FP64 and stored as pairs of FP32 numbers (P (P + 1) / 2
 * pairs per edge, built on first use when they take at most a quarter of
 * the free device memory, else the FP64 apply); 1: the FP64 apply
 * (sg_residual); 2: always the edge blocks, built now (SG_ERR_NOMEM when
 * they do not fit, SG_ERR_ARG for P > 128).  Double-FP32: 48-bit
 * significands, exact products of the high words (FMA), error-free sums,
 * rounding errors gathered in the low word; the residual entries agree with
 * FP64 to about 1e-13 of sum |A||X|, and the differences x_r - x_c are
 * formed before any product, so the cancellation of the stencil costs no
 * accuracy.  It runs on the FP32 units: GB300's FP64 rate is about 1/64 of
 * its FP32 rate.  A change drops the recorded graphs, as sg_set_apply_fp64. */
sg_status sg_set_refine_residual(sg_problem* prob, int mode);

/* Whether the double-FP32 edge blocks are in use (0/1) and their device
 * bytes (blocks and the split iterate).  Either pointer may be NULL. */
sg_status sg_refine_residual_info(const sg_problem* prob, int* built, int64_t* bytes);

/* R = F - sum_k A_k X G_k^T as the refinement computes it (see
 * sg_set_refine_residual): FP64 arrays, layout as sg_residual (F may equal
 * R; X must not overlap R).  Asynchronous on `stream` once the edge blocks
 * exist (the first call builds them, synchronously).  Errors: SG_ERR_ARG
 * for NULL pointers, leading dimensions < n or overlaps; SG_ERR_CUDA. */
sg_status sg_residual_refine(sg_problem* prob, const double* F_dev, int64_t ldf, const double* X_dev, int64_t ldx,
                             double* R_dev, int64_t ldr, void* stream);

/* Tile shape of the register-specialised kernel of one family: which = 0
 * fine FP32, 1 coarse FP32, 2 fine FP64, 3 coarse FP64 (the FP64 kernels
 * carry the triple products as exact double immediates): rows per thread
 * (1, or for FP32 2 adjacent rows updated with the paired FP32 FMA); output
 * groups, input groups (1..4 each) and stencil-slot groups (1..8), product
 * <= 8: the outputs, the gathered inputs and the slots are split across
 * groups of 4 warps whose partial sums meet in shared memory; prefetch (0..64:
 * input terms whose values are loaded ahead into registers, or with stages
 * the terms per staged block); min_blocks (CTAs per SM asked of the register
 * allocator, 1..8); stages (0: register prefetch; 2..8: the matrix values
 * stream through shared memory by cp.async, stages - 1 blocks ahead of use,
 * across slot boundaries; one row and one group only); cgroups (1..16: the
 * outputs split over that many separate 128-thread CTAs per row tile, each
 * with the full register file of its threads; one row and one group only);
 * warps (1, 2 or 4 warps per group, i.e. 32, 64 or 128 rows per tile: narrow
 * groups let many slot or input groups share one CTA without capping its
 * registers; fewer than 4 only without staging or separate CTAs).
 * Recompiles.
 * Errors: SG_ERR_ARG out of range, SG_ERR_CUDA compile failure. */
sg_status sg_apply_config(sg_problem* prob, int which, int rows, int groups, int igroups, int sgroups,
                          int prefetch, int min_blocks, int stages, int cgroups, int warps);

/* Edge-flux form of the fine FP32 operator (Sec. 2.1, Eq. Galerkin_L_exp
 * in Kronecker form, the stiffness written edge by edge): on this mesh the
 * rows of every A_k are
 *     (A_k x)_r = sum over the four edges (r, r') of w_k(r, r') (x_r - x_r'),
 * x_r' = 0 at a Dirichlet node, with one conductance w_k per edge (half the
 * sum of c_k over the two triangles sharing it).  Storing the K
 * conductances of the 2 N (N - 1) edges instead of the K values of five
 * stencil slots per node reads 2.5 times fewer matrix bytes per apply, and
 * four edge passes replace five slot passes.  mode 0: the five-slot form
 * (the autotuner may not choose the edge form); 1: the edge form now (its
 * K x 2 N (N - 1) FP32 conductances are built on first use); 2 (default):
 * the autotuner (sg_apply_autotune, fine FP32 family) times both forms and
 * keeps the faster; -1: no change.  on (may be NULL) receives 1 when fine
 * FP32 applies use the edge form.  sg_apply_config selects the slot form.
 * Coarse and FP64 applies are unaffected.  A change drops recorded
 * coarse-solve graphs; recorded batches of this problem then refuse to run.
 * Errors: SG_ERR_ARG (mode out of range; mode 1 without the specialised
 * kernel), SG_ERR_NOMEM, SG_ERR_CUDA. */
sg_status sg_apply_flux(sg_problem* prob, int mode, int* on);

/* Autotuner: compiles the candidate tile shapes, times each on this
 * problem's operator of family `which` (as for sg_apply_config; the
 * coarse families after sg_precond_setup) with CUDA events, keeps the fastest and stores
 * the choice in the kernel cache directory (keyed by the triple structure,
 * rows, slots and the device name) so later setups reuse it unless
 * force != 0.  best_ms (may be NULL) receives the time of the chosen shape.
 * Synchronous; allocates two temporary blocks. */
sg_status sg_apply_autotune(sg_problem* prob, int which, int force, double* best_ms);

/* Current tile shape of one family (rows, groups, igroups, sgroups,
 * prefetch, min_blocks, stages, cgroups, warps, code-generator version into
 * cfg10) and the seconds spent compiling or loading its kernel. */
sg_status sg_apply_info(const sg_problem* prob, int which, int* cfg10, double* compile_s);

/* Residual R = F - sum_k A_k X G_k^T (Sec. 2.1, Eq. Galerkin_L_exp), same
 * layout and dtype rules as sg_apply (F may equal R for an in-place
 * update; X must not overlap R).  Errors as for sg_apply. */
sg_status sg_residual(sg_problem* prob, sg_dtype dtype, const void* F_dev, int64_t ldf,
                      const void* X_dev, int64_t ldx, void* R_dev, int64_t ldr, void* stream);

/* ------------------------------------------------------------------------
 * Two-level preconditioner (Sec. 3, Eqs. RASsto, coarse, RAS_2L; variant
 * 2GV3: the coarse problem is solved by an inner GMRES preconditioned by
 * AMG).  The cycle applied to a residual r is
 *     z  = S r,   z += Q (r - A z),   z += S (r - A z),
 * with Q = R_0^T A_c^{-1} R_0 (R_0^T: P1 interpolation from the nested 2h
 * mesh, A_c = sum_k (R_0 A_k R_0^T) (x) G_k solved by GMRES + AMG to
 * inner_rtol) and the restricted additive Schwarz smoother
 *     S r = omega (G~^{-1} (x) I) sum_i R_i^T D_i (I (x) A_{0,i})^{-1} R_i r,
 * where boxes are sx x sy blocks of the interior grid grown by `overlap`
 * layers of the A_0 graph, D_i keeps owned nodes, A_{0,i} is the local mean
 * block, G~ = sum_k (<A_k, A_0>_F / <A_0, A_0>_F) G_k is the stochastic
 * Kronecker factor, and omega = 1 / rho(S A) (power iteration) unless given.
 * ------------------------------------------------------------------------ */
typedef struct {
  int sx, sy;          /* subdomain boxes per direction (>= 1)          */
  int overlap;         /* overlap layers (0..8)                         */
  double omega;        /* smoother damping; <= 0 = estimate             */
  double inner_rtol;   /* coarse GMRES tolerance; <= 0 = 1e-5           */
  int inner_max;       /* coarse GMRES iteration cap; <= 0 = 100        */
  int smoother;        /* 0 = RAS; 1 = learned (needs weights: sg_cnn_init,
                          sg_cnn_set_weights or sg_train_precond)       */
  int host_loops;      /* 0 (default): each coarse solve is one CUDA graph
                          launch whose restart and Arnoldi loops are
                          conditional WHILE nodes decided on the device;
                          1: the same GMRES driven from the host         */
  int ras_modes;       /* modes per CTA of the RAS local solve kernel
                          (tile shape); <= 0 = automatic                 */
  int inner_orth_passes; /* Gram-Schmidt passes per Arnoldi step of the
                          coarse GMRES: 1 (<= 0) = classical, the
                          PETSc default the paper's runs used (Sec. 5);
                          2 = classical with one re-orthogonalisation   */
  int amg_kernel;      /* AMG V-cycle kernels: 0 = level 0 as three
                          GPU-wide kernels and all coarser levels in one
                          launch (one CTA per PCE mode, level vectors in
                          shared memory); 1 = one launch per level
                          operation                                      */
  int ras_stages;      /* line steps whose matrices the RAS kernel keeps in
                          flight or resident (2..8); 0 = automatic       */
  int ras_kernel;      /* RAS local solves on FP32 data: 0 = FMA kernel;
                          1 = tensor cores (m16n8k8 TF32 MMA with operands
                          split into high and remainder parts, FP32
                          accumulation; 8 modes per CTA unless ras_modes
                          is given); 2 = explicit local inverses: the owned
                          rows of each (I (x) A_{0,i})^{-1}, formed at setup
                          in FP64 from the line factors and stored in FP32
                          (boxes wider than twice the overlap, P <= 96),
                          applied as dense products on the tcgen05 tensor
                          cores (kind::tf32, operands split into high and
                          remainder parts, FP32 accumulation in tensor
                          memory) with the Kronecker factor fused;
                          3 = automatic: 2 when its inverses can be built
                          and one application measures faster than the
                          FMA kernel's on this problem, else 0.  FP64
                          data always use the FMA kernel. */
} sg_precond_opts;

/* Builds partitions, local factors, the coarse space, the AMG hierarchy,
 * the Kronecker factor and omega.  Needs an even N >= 4.  Replaces a
 * previous preconditioner.  Synchronous.
 * Errors: SG_ERR_ARG (ranges), SG_ERR_NOMEM, SG_ERR_CUDA, SG_ERR_BREAKDOWN
 * (omega estimate or Kronecker factor not finite). */
sg_status sg_precond_setup(sg_problem* prob, const sg_precond_opts* opts, void* stream);

/* omega, number of AMG levels, coarse unknowns per mode, iterations of the
 * last inner coarse solve.  Any pointer may be NULL. */
sg_status sg_precond_info(const sg_problem* prob, double* omega, int* amg_levels, int64_t* nc,
                          int* inner_its_last);

/* Size of the RAS local solves: useful flops of one application over all P
 * modes (forward and backward block sweeps: per line the w_l x w_{l-1}
 * sub-diagonal block and the triangular inverse), number of boxes, padded
 * line width, and the FP32 local-solve kernel in use (0, 1 or 2 as for
 * sg_precond_opts.ras_kernel; the automatic choice 3 resolved).  Any
 * pointer may be NULL. */
sg_status sg_precond_stats(const sg_problem* prob, double* ras_flops, int* ras_boxes, int* ras_wmax,
                           int* ras_kernel);

/* Overlapped node set of box `sub` (ascending global indices) and its owned
 * flags (D_i).  Call with idx = owned = NULL to get the count first. */
sg_status sg_get_partition(const sg_problem* prob, int sub, int32_t* idx, int64_t* count,
                           int32_t* owned);

/* Pattern of the coarse matrices R_0 A_k R_0^T (symbolic product). */
sg_status sg_get_coarse_csr(const sg_problem* prob, int64_t* nc, int64_t* nnz, int32_t* rowptr,
                            int32_t* colidx);

/* Size of AMG level `level` and, for every level but the last, the
 * aggregate id of each of its unknowns (host array of n entries). */
sg_status sg_get_amg_level(const sg_problem* prob, int level, int64_t* n, int32_t* agg);

/* Applies one piece of the preconditioner to a mode-major device block
 * (for tests and for users composing their own solver):
 *   0 two-level cycle z = B r        (fine -> fine)
 *   1 smoother S r                    (fine -> fine)
 *   2 coarse correction Q r           (fine -> fine)
 *   3 one AMG V-cycle per mode        (coarse -> coarse)
 *   4 coarse operator A_c x           (coarse -> coarse)
 *   5 restriction R_0 r               (fine -> coarse)
 *   6 interpolation R_0^T e           (coarse -> fine)
 *   7 RAS local mean solves only      (fine -> fine)
 *   8 learned smoother S_cnn r        (fine -> fine; after sg_precond_set_smoother)
 *   9 network only, CNN(r) per mode   (fine -> fine)
 * Operators 0 and 1 use the smoother currently selected.
 * Coarse blocks have nc rows (sg_precond_info).  R and Z must not overlap. */
sg_status sg_precond_apply(sg_problem* prob, sg_dtype dtype, int which, const void* R, int64_t ldr,
                           void* Z, int64_t ldz, void* stream);

typedef struct {
  double rtol;        /* stop when ||F - A X|| <= rtol ||F|| (true FP64 residual) */
  int max_it;         /* cap on outer (F)GMRES iterations in total             */
  int restart;        /* FGMRES restart length (<= 31; <= 0 = 30)              */
  int mode;           /* 0: FP64 FGMRES with FP64 preconditioner;
                         1: FP32 FGMRES + FP32 preconditioner inside FP64
                            iterative refinement (FP64 residuals)              */
  double inner_rtol;  /* mode 1: tolerance of each FP32 solve (relative to the
                          step's residual; a step whose residual is within a
                          factor of the target stops at half of rtol / rr,
                          at most 0.5); <= 0 = 3e-4                         */
  int max_ir;         /* mode 1: refinement steps cap; <= 0 = 20               */
  double* hist_host;  /* optional host buffer for the residual history         */
  int hist_cap;
  int no_fallback;    /* 1: keep the learned smoother even when it stagnates   */
  int orth_passes;    /* Gram-Schmidt passes per Arnoldi step of the outer
                         (F)GMRES: 1 (<= 0) = classical (PETSc default);
                         2 = classical with one re-orthogonalisation       */
} sg_solve_opts;

typedef struct {
  int outer_it;       /* (F)GMRES iterations (all refinement steps)  */
  int inner_it;       /* coarse GMRES iterations, summed              */
  int ir_steps;       /* refinement corrections applied (mode 1)      */
  int fallback_used;  /* learned smoother replaced by RAS mid-solve    */
  int hist_len;       /* entries written to hist_host                 */
  double relres;      /* ||F - A X|| / ||F|| in FP64 at return       */
  double t_setup, t_solve; /* seconds (t_setup unused here)          */
} sg_solve_info;

/* Solves sum_k A_k X G_k^T = F (Sec. 2.1, Eq. Galerkin_L_exp) by flexible
 * GMRES with the two-level preconditioner (Sec. 3; mode 1 adds the FP32
 * inner solves in FP64 refinement of the method statement).  F = NULL uses
 * the load vector of sg_get_rhs.  X holds the initial guess on entry and the solution on
 * return (FP64 device blocks).  Needs sg_precond_setup.  Synchronises the
 * stream once per iteration to test convergence.
 * Returns SG_OK when relres <= rtol, SG_NOT_CONVERGED (X = last iterate)
 * when max_it is reached first, SG_ERR_BREAKDOWN on non-finite values. */
sg_status sg_solve(sg_problem* prob, const double* F_dev, int64_t ldf, double* X_dev, int64_t ldx,
                   const sg_solve_opts* opts, sg_solve_info* info, void* stream);

/* ------------------------------------------------------------------------
 * Nonlinear problem (Sec. 2.2, Eqs. NLP_StrongPDE, stonlp_system,
 * vectorvalPDENL, AjkTkl, with the conductivity (1 + u^2) in place of the
 * paper's (1 + alpha u)):
 *     -div( c(x, xi) (1 + u^2) grad u ) = 1,   u = 0 on the boundary,
 * c the lognormal field of sg_setup.  Inside triangle e the solution enters
 * the conductivity through its element average ubar_e (mean of the three
 * vertex values, zero at Dirichlet vertices); its square is projected onto
 * the output chaos by the triple products,
 *     w_{e,f} = sum_{a,b} ubar_{e,a} ubar_{e,b} <psi_a psi_b psi_f>,
 * so the element Galerkin matrix is
 *     sum_i cbar_i(e) <psi_i psi_l psi_m> + sum_{i,f} cbar_i(e) w_{e,f} <psi_i psi_f psi_l psi_m>.
 * The fourfold products are formed through the input chaos, which needs
 * q_in >= 2 p_out (SG_ERR_ARG otherwise).  Nonlinear operator A(U), residual
 * F - A(U) U, Jacobian J(U) = A(U) + d(A(U)) U / dU (non-symmetric).  The
 * first call builds the nonlinear work (coefficients of every input term
 * at every triangle, the triple lists, two operator value arrays:
 * about 2 (K E + 3 K n) doubles).  SG_ERR_UNSUPPORTED when (3 P + K) x 256
 * bytes exceed the 227 KB of shared memory a CTA may use.
 * ------------------------------------------------------------------------ */

/* Newton's method from the initial guess in X (FP64 mode-major device
 * block; the solution on return): each step solves J(U) dU = F - A(U) U
 * (F = the load vector) by flexible GMRES preconditioned by the two-level
 * cycle of sg_precond_setup (set up for the linear problem; the learned
 * smoother when it is selected) to the relative tolerance opts->inner_rtol
 * (<= 0: 1e-4), with at most opts->max_it iterations a step; mode 1: the
 * Jacobian applies and the preconditioner in FP32 (the Newton residual and
 * the update in FP64), mode 0: all in FP64.  Stops when
 * ||dU|| / ||U|| <= tol_update.  info: outer_it = GMRES iterations summed,
 * inner_it = coarse GMRES iterations, ir_steps = Newton steps, relres =
 * ||F - A(U) U|| / ||F|| of the returned U, hist_host = the relative
 * updates.  Needs sg_precond_setup.
 * Returns SG_OK, SG_NOT_CONVERGED (max_newton steps taken; X = last
 * iterate), SG_ERR_BREAKDOWN (non-finite residual or update), SG_ERR_ARG,
 * SG_ERR_UNSUPPORTED (see above). */
sg_status sg_newton(sg_problem* prob, double* X_dev, int64_t ldx, double tol_update, int max_newton,
                    const sg_solve_opts* opts, sg_solve_info* info, void* stream);

/* R = F - A(X) X in FP64 (F = NULL: the load vector), mode-major device
 * blocks; R must not overlap X or F.  Errors as for sg_apply, plus those of
 * the nonlinear setup above. */
sg_status sg_nonlinear_residual(sg_problem* prob, const double* F_dev, int64_t ldf, const double* X_dev,
                                int64_t ldx, double* R_dev, int64_t ldr, void* stream);

/* Y = J(U) dU, the Jacobian of the nonlinear residual's operator part at U
 * applied to dU: dtype FP64 (double blocks, FP64 arithmetic) or FP32
 * (float blocks; the operator A(U) is formed from U in FP64, everything
 * else in FP32).  Y must not overlap U or dU.  Errors as for
 * sg_nonlinear_residual. */
sg_status sg_nonlinear_jacobian_apply(sg_problem* prob, sg_dtype dtype, const void* U_dev, int64_t ldu,
                                      const void* dU_dev, int64_t lddu, void* Y_dev, int64_t ldy, void* stream);

/* Monte Carlo verification (Sec. 4.1, Fig. mcs_verify_poisson: the SG
 * mean, standard deviation and pdf against Monte Carlo samples of the
 * deterministic problem).  For each of S samples xi_s (FP64 device array,
 * S x L row-major, drawn by the caller) solves
 *     -div( c_s grad u_s ) = 1,  u_s = 0 on the boundary,
 *     c_s(e) = exp( g0 + sum_i g_i(e) xi_{s,i} )
 * (the exact lognormal field with this problem's KL modes at the element
 * centroids) with the P1 discretisation of the SG system, by
 * Jacobi-preconditioned conjugate gradients in FP32 to ||r|| <= rtol ||b||
 * or max_it iterations, one CTA per sample with its vectors in shared
 * memory.  u_s is written to U + s * ldu (n values, dtype FP32 or FP64).
 * its_max (host, may be NULL) receives the largest iteration count.
 * Synchronous.  Limits: 1 <= L <= 16 and N <= 102 (the sample's system
 * must fit one CTA: about 16 (N-1)^2 bytes of shared memory).
 * Returns SG_NOT_CONVERGED when a sample reached max_it (all are written),
 * SG_ERR_ARG for the limits or bad arguments. */
sg_status sg_sample_solve(sg_problem* prob, const double* xi_dev, int64_t S, sg_dtype dtype, void* U_dev,
                          int64_t ldu, double rtol, int max_it, int* its_max, void* stream);

/* ------------------------------------------------------------------------
 * Learned smoother.  The method statement replaces the mean-based local
 * solve (I (x) A_0)^{-1} inside the smoother by a small convolutional
 * network applied to the P mode images of the residual; the paper has no
 * counterpart.  The network: 3x3 convolutions with zero padding, channels
 * 2 -> 32 -> 32 -> 32 -> 32 -> 1, bias, ReLU after the first four layers;
 * BF16 weights and activations, FP32 accumulation and FP32 master weights.
 * Mode image a of a block R (n = (N-1)^2 nodes in mesh order, row-major
 * (N-1) x (N-1)) enters as channel 0 = r_a / rms(r_a) and channel 1 =
 * log(a_rr / 4) (a_rr: diagonal of A_0); the output is multiplied by
 * rms(r_a).  The learned smoother is
 *     S_cnn r = omega_cnn (G~^{-1} (x) I) CNN(r),
 * omega_cnn = 1 / rho(S_cnn A) by the same power iteration as RAS.  Inside
 * sg_solve a solve that stagnates (residual estimate above 0.7 x its value
 * 10 iterations earlier, or a refinement step that does not halve the
 * residual) or produces non-finite values switches to RAS for the rest of
 * the solve and reports fallback_used = 1.
 * Weights cross the ABI as a flat FP32 host array in this order, for each
 * layer l = 0..4: W_l[3][3][C_l][C_{l+1}] (tap row, tap column, input
 * channel, output channel), then b_l[C_{l+1}]; sg_cnn_param_count() values.
 * ------------------------------------------------------------------------ */
int64_t sg_cnn_param_count(void);

/* He-normal weights (standard deviation sqrt(2 / (9 C_in))), zero biases,
 * from a splitmix64 stream and the Box-Muller transform.  Resets Adam. */
sg_status sg_cnn_init(sg_problem* prob, uint64_t seed, void* stream);

/* Loads (save: sg_cnn_get_weights) the flat weight array; count must equal
 * sg_cnn_param_count().  Loading resets the Adam moments.  Synchronous. */
sg_status sg_cnn_set_weights(sg_problem* prob, const float* w_host, int64_t count, void* stream);

/* what = 0: current weights; 1: the gradient of the last training step
 * (same layout).  Synchronous. */
sg_status sg_cnn_get_weights(sg_problem* prob, float* w_host, int64_t count, int what, void* stream);

/* Z[:, a] = rms(r_a) CNN(features(r_a)) for nimg FP32 device columns of R
 * (column a at R + a ldr); rows n..ldz-1 of Z are cleared.  nimg <= 65535.
 * Allocates activation buffers on first use or growth. */
sg_status sg_cnn_apply(sg_problem* prob, const float* R_dev, int64_t ldr, float* Z_dev, int64_t ldz, int nimg,
                       void* stream);

/* One training step on nimg (residual, target) column pairs, the target in
 * residual units (e.g. A_0^{-1} r), with the loss of sg_cnn_set_loss (y_a
 * the network output, e_a = y_a - z*_a / rms(r_a)); gradients by the
 * backward convolution kernels; with update != 0 one Adam step (beta1 0.9,
 * beta2 0.999, eps 1e-8) with learning rate lr.  loss (host, may be NULL)
 * receives the loss before the update and makes the call synchronous. */
sg_status sg_cnn_train_step(sg_problem* prob, const float* R_dev, int64_t ldr, const float* Zstar_dev,
                            int64_t ldz, int nimg, float lr, int update, double* loss, void* stream);

/* Forward-convolution kernels of the network: 1 (default) the
 * fifth-generation tensor cores (tcgen05: 128-pixel row tiles, BF16 operands
 * in shared memory, FP32 accumulators in tensor memory); 0 the BF16 mma.sync
 * kernels (also used for every backward pass).  sg_cnn_apply returns
 * SG_ERR_TIMEOUT if a tcgen05 completion wait ran out (no output then). */
sg_status sg_cnn_set_kernel(sg_problem* prob, int kind);

/* Plumbing.  Polls of the mbarrier on which a tcgen05 CTA of this handle
 * (the network's convolutions, the RAS products with explicit local
 * inverses) waits for its MMAs before it gives up (limit < 0: the default,
 * 4,194,304 polls).  A CTA whose wait runs out stores nothing, sets an
 * error flag that sg_cnn_apply, sg_precond_apply and sg_solve return as
 * SG_ERR_TIMEOUT, and then waits again (bounded) for the MMAs it issued
 * before it frees their tensor memory, so the context stays usable.
 * limit = 0 makes every such wait run out at once (for tests of that path). */
sg_status sg_set_wait_limit(sg_problem* prob, int limit);

/* Loss of sg_cnn_train_step: 0 (default) sum_a (e_a^T A_0 e_a) /
 * (z*_a^T A_0 z*_a), e_a = y_a - z*_a / rms(r_a): the error in the energy
 * norm of A_0, which weights the oscillatory error a smoother must remove;
 * 1: sum_a ||e_a||^2 / ||z*_a||^2. */
sg_status sg_cnn_set_loss(sg_problem* prob, int kind);

/* Z = A_0^{-1} B for nb FP32 device columns (the training targets): FP64
 * conjugate gradients preconditioned by one smoothed-aggregation V(1,1)
 * cycle of A_0 per iteration, all columns together, until every column
 * has ||b - A_0 z|| <= rtol ||b|| or max_it iterations.  relres_max and its
 * (host, may be NULL) receive the worst relative residual and the
 * iterations.  Builds the A_0 hierarchy on first use.  Synchronous.
 * Errors: SG_ERR_ARG, SG_ERR_NOMEM, SG_ERR_BREAKDOWN (non-finite). */
sg_status sg_mean_solve(sg_problem* prob, const float* B_dev, int64_t ldb, float* Z_dev, int64_t ldz, int nb,
                        double rtol, int max_it, double* relres_max, int* its, void* stream);

typedef struct {
  int n_pairs;        /* training pairs (e.g. 4096)                      */
  int epochs;         /* passes over the pairs                           */
  int batch;          /* images per Adam step (e.g. 32)                  */
  float lr;           /* Adam learning rate (e.g. 1e-3)                  */
  uint64_t seed;      /* He init, right-hand sides, sampling, batch order */
  double target_rtol; /* relative residual of the targets; <= 0 = 1e-6   */
  int keep_weights;   /* 1: continue from the current weights            */
  int loss;           /* 0: relative error in the energy norm of A_0,
                         1: relative L2 error of the correction          */
} sg_train_opts;

typedef struct {
  int n_pairs, steps;     /* pairs used, Adam steps taken                  */
  int harvest_solves;     /* plain solves run to collect residuals         */
  int target_its;         /* CG iterations of the slowest target batch     */
  double target_relres;   /* worst relative residual of the targets        */
  double loss_first;      /* mean loss per image, first and last batch     */
  double loss_last;
  double omega_cnn;       /* damping chosen for the learned smoother       */
  double t_harvest, t_targets, t_train;  /* seconds                        */
} sg_train_info;

/* Trains the learned smoother on the method's own data and selects it:
 * (1) plain mixed-precision solves (RAS smoother; the load vector, then
 * seeded Gaussian right-hand sides) record every FP32 smoother input until
 * 1.5 n_pairs mode images are pooled; n_pairs are drawn uniformly without
 * replacement; (2) targets z* = A_0^{-1} r by sg_mean_solve; (3) Adam over
 * `epochs` passes, batches of consecutive pairs in a fresh order each
 * epoch; (4) omega_cnn estimated, smoother set to 1.  Needs
 * sg_precond_setup.  Synchronous.  Allocates the pool, the pairs and the
 * training buffers. */
sg_status sg_train_precond(sg_problem* prob, const sg_train_opts* opts, sg_train_info* info, void* stream);

/* Selects the smoother of later solves: 0 RAS, 1 learned (needs weights;
 * omega <= 0 estimates omega_cnn). */
sg_status sg_precond_set_smoother(sg_problem* prob, int smoother, double omega, void* stream);

/* Saves the learned smoother (method statement; no paper counterpart):
 * its network weights, its damping omega_cnn and whether it is the selected
 * smoother, into the caller's host buffer buf of *bytes bytes.  With
 * buf = NULL only *bytes (the size needed) is written.  The format is a
 * fixed 32-byte header (magic "SGLSMTH", version 1, parameter count,
 * omega_cnn, selection flag) followed by the FP32 weights in the order of
 * sg_cnn_set_weights.  Synchronous.
 * Errors: SG_ERR_ARG (NULL handle or bytes, no weights set, buffer too
 * small). */
sg_status sg_precond_save(const sg_problem* prob, void* buf, int64_t* bytes);

/* Restores a smoother saved by sg_precond_save into any problem (the
 * network does not depend on the mesh size or P): the weights, and, when
 * this problem has a preconditioner set up and the smoother was selected at
 * save time, the learned smoother is selected with the saved damping (or a
 * new estimate when none was saved).  Synchronous.
 * Errors: SG_ERR_ARG (NULL argument, wrong magic or version, a parameter
 * count or size that does not match this build's network, bad damping). */
sg_status sg_precond_load(sg_problem* prob, const void* buf, int64_t bytes);

/* ------------------------------------------------------------------------
 * Graph-captured and batched solves.  sg_batch_create records, for every
 * problem, the whole solve of sg_solve (mode 1: the refinement loop with
 * its FP64 residuals, every FP32 FGMRES restart and Arnoldi step, every
 * two-level cycle with its inner coarse GMRES + AMG; mode 0: the FP64
 * FGMRES) as CUDA graph nodes whose loops are conditional WHILE nodes
 * decided on the device, the problems as parallel branches of one graph.
 * sg_batch_solve launches that graph once: all systems are solved with no
 * host round trip.  The recorded smoother is the one selected at creation;
 * there is no learned-to-RAS fallback inside the graph.  The batch uses
 * each problem's solver workspaces: do not call sg_precond_setup on a member
 * problem (sg_batch_solve then fails with SG_ERR_ARG) or run the problems
 * on other streams while a batch solve is in flight; destroy the batch
 * before its problems.  The paper solves one system at a time; batching
 * independent systems is a property of this library.
 * ------------------------------------------------------------------------ */
typedef struct sg_batch sg_batch;

/* count in [1, 256] distinct problems, each after sg_precond_setup; opts as
 * for sg_solve (hist_host ignored; restart, rtol, max_it, mode, inner_rtol
 * and max_ir are recorded).  Allocates each problem's solve workspaces,
 * compiles its specialised kernels and records the graph.  Synchronous. */
sg_status sg_batch_create(sg_problem* const* probs, int count, const sg_solve_opts* opts, sg_batch** out);

/* Solves every system of the batch: F[i] (FP64 device block, ldf[i] rows;
 * F or F[i] NULL = the load vector) and X[i] (initial guess in, solution
 * out, ldx[i] rows).  infos[i] (may be NULL): outer_it = FGMRES iterations,
 * inner_it = coarse GMRES iterations, ir_steps, relres = true FP64
 * relative residual of the returned X[i], t_solve = wall time of the whole
 * batch.  Returns SG_OK when every system reached rtol, SG_NOT_CONVERGED
 * when one stopped at max_it / max_ir, SG_ERR_BREAKDOWN on a non-finite
 * residual.  Synchronises the stream once. */
sg_status sg_batch_solve(sg_batch* batch, const double* const* F, const int64_t* ldf, double* const* X,
                         const int64_t* ldx, sg_solve_info* infos, void* stream);

/* Releases a recorded batch (NULL is accepted); the problems stay valid. */
sg_status sg_batch_destroy(sg_batch* batch);

/* sg_batch_create + sg_batch_solve + sg_batch_destroy in one call (method
 * statement: batching).  Errors as for those three. */
sg_status sg_solve_batch(sg_problem* const* probs, int count, const double* const* F, const int64_t* ldf,
                         double* const* X, const int64_t* ldx, const sg_solve_opts* opts, sg_solve_info* infos,
                         void* stream);

/* Multi-vector dot products, the classical Gram-Schmidt step of the
 * Arnoldi process inside FGMRES (Sec. 3):  out[i] = sum_e V_i[e] w[e] for
 * i < nv, where V_i = V + i * stride.  dtype selects double or float
 * vectors; products of float vectors are summed in FP32 over at most 8
 * elements per thread, every other sum is FP64.  out is a device array of
 * nv doubles.  nv in [1, 32]; stride >= len when nv > 1.  The reduction
 * scratch (2 x 152 x 32 doubles and a counter) is allocated in the handle
 * on first use; calls through one handle must not overlap on the GPU.
 * Errors: SG_ERR_ARG, SG_ERR_NOMEM, SG_ERR_CUDA. */
sg_status sg_mdot(sg_problem* prob, sg_dtype dtype, const void* V, int64_t stride, int nv, const void* w,
                  int64_t len, double* out_dev, void* stream);

/* sg_mdot without any allocation, for callers that cannot call cudaMalloc:
 * code that shares the GPU with a framework whose caching allocator already
 * holds the free device memory, latency-critical loops that cannot afford
 * the device-wide synchronisation cudaMalloc may cause, and callers that
 * have no sg_problem handle to own scratch.  (The paper has no counterpart:
 * this is a property of the library, not of the method.)
 * Same arguments and results as sg_mdot, without the handle.  The reduction
 * scratch is a fixed static device array of 304 x 32 doubles plus a counter,
 * present on every GPU that loads the library until the process exits; nv
 * above 32 is rejected with SG_ERR_ARG.  Each call clears the counter on
 * `stream` and allocates nothing (no cudaMalloc, cudaFree or allocating
 * library routine).  All calls share the one array per device and it keeps
 * the last call's contents, so calls whose kernels overlap on the GPU (other
 * streams, other threads) race: serialise them.  The first call on a device
 * looks up the array's device address with that device current; make that
 * first call before any stream capture.
 * Errors: SG_ERR_ARG, SG_ERR_CUDA. */
sg_status sg_mdot_noalloc(sg_dtype dtype, const void* V, int64_t stride, int nv, const void* w,
                          int64_t len, double* out_dev, void* stream);

/* Plumbing.  Per-launch timing of the operator-apply and RAS local-solve
 * kernels and of the phases of a host-driven solve, for benchmarks.  While
 * enabled, every such launch or phase through this handle (outside recorded
 * graphs) is bracketed by CUDA events on its stream (a few microseconds of
 * overhead each, so time the headline with the profiler off).  Enabling (or
 * disabling) clears the records.  sg_profile_read waits for the recorded
 * events and returns the number of launches and their summed device time in
 * ms for one kind: 0 fine apply FP32, 1 fine apply FP64, 2 coarse apply
 * FP32, 3 coarse apply FP64, 4 RAS local solve FP32, 5 RAS local solve FP64;
 * phases (each holds the kernels it launches; 4 and 5 lie inside 6):
 * 6 smoother, 7 coarse correction (restriction, the coarse GMRES graph,
 * interpolation), 8 Arnoldi step (Gram-Schmidt, Givens rotation,
 * normalisation), 9 refinement bookkeeping (FP64 residual norm, conversion
 * to FP32, the update of x).
 * Errors: SG_ERR_ARG for a kind outside 0..9. */
sg_status sg_profile(sg_problem* prob, int enable);
sg_status sg_profile_read(sg_problem* prob, int kind, int64_t* launches, double* ms);

/* Plumbing.  Number of kernel launches this library has made in the process
 * so far (all handles, kernels inside recorded graphs included);
 * differences bracket a region of interest.  Errors: SG_ERR_ARG for NULL. */
sg_status sg_launch_count(int64_t* count);

/* Message of the last failure on this host thread ("" when none); the
 * pointer stays valid until the thread's next failing call. */
const char* sg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SG_H_ */
