"""FP64 CPU oracle for the stochastic Galerkin (SG) method of arXiv 2310.14649.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) may import, call, link or execute anything in this
package; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` use it.  It shares no code with the CUDA path: every formula
here is written out again from the paper (and, where the paper is silent or
garbled, from the readings listed in the design notes), in plain numpy /
scipy, slowly and in float64.

Modules
-------
pce        multi-index sets, Hermite triple products, lognormal input PCE
           (Sec. 2.1, Eqs. inputpc, inputlogn, outpc, Galerkin_L_exp)
kl         Karhunen-Loeve eigenpairs of the separable exponential kernel
           (Sec. 2.1, Eqs. KLE, CovarKer2DNLP)
fem        structured P1 mesh, stiffness matrices A_k, load vector
           (Sec. 2.1, Eq. Galerkin_L_exp; appendix Eq. qunlc4 for the m=0 pin)
galerkin   Kronecker-form operator sum_k A_k X G_k^T, its assembled matrix,
           direct and GMRES solves (Sec. 2.1 and Sec. 3)
ras        subdomain partitions and the one-level RAS operator (Sec. 3,
           Eqs. RASstofixedpoint, RASsto)
coarse     2h interpolation R_0^T and the Galerkin coarse operator (Sec. 3,
           Eq. coarse)
amg        smoothed-aggregation hierarchy and V-cycle (the AMG of Sec. 3)
twolevel   multiplicative two-level preconditioner (Sec. 3, Eq. RAS_2L)
variants   the paper's own preconditioner variants: RAS with ILU(0) of the
           coupled local block, the 2GV2 coarse solve (Sec. 3, Sec. 5)
nonlinear  the nonlinear problem (Sec. 2.2, Eqs. NLP_StrongPDE,
           stonlp_system, AjkTkl): fourfold products t_ijkl, the linearised
           operator A + T(U) and the Picard iteration; the deterministic
           problem for collocation pins
newton     the nonlinear problem with conductivity k (1 + u^2) (Sec. 2.2 with
           u^2 in place of alpha u): the projected square, the element
           Galerkin matrices, the residual, the exact Jacobian and Newton's
           method
par        multi-core operator apply, mean-block preconditioner and GMRES
           (plain C loops in sgo.c over all host cores), for full-size
           reference solutions and the timed CPU baseline
cnn        FP64 convolutional smoother forward/backward (not in the paper:
           parity unpinned against the paper, gradients pinned by
           central differences)
"""
