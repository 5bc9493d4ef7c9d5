/*
 * Multi-core FP64 pieces of the oracle, in plain C with OpenMP.
 *
 * TEST INFRASTRUCTURE ONLY.  Like the rest of oracle/, this file may be
 * built, loaded and called only by tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py; the product library never links it.  It
 * shares no code with the CUDA path: every loop below is the plain
 * definition of the operation, written again from the paper.
 *
 * Blocks of PCE coefficients are flat mode-major vectors: entry (node r,
 * mode a) at x[a n + r] (the vec() of the oracle's [n, P] arrays).
 *
 *   sgo_apply      y = (sum_k G_k kron A_k) x, from the entrywise form of
 *                  the Galerkin operator (Sec. 2.1, Eq. Galerkin_L_exp):
 *                  y_r[a] = sum_{c in row r} sum_{(k,a,b)} v_k^{rc} g_kab x_c[b]
 *   sgo_band_solve x = (I kron A_0)^{-1} b for a banded Cholesky factor of
 *                  A_0 (the mean-based block preconditioner of Sec. 3 used
 *                  by the oracle's GMRES), one forward and one backward
 *                  substitution per mode
 *   sgo_dot, sgo_axpy, sgo_scal
 *                  vector kernels of the GMRES driver, each a plain loop
 *                  (the dot product sums each thread's share in order, then
 *                  the shares in thread order)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <omp.h>

int sgo_threads(void) { return omp_get_max_threads(); }

void sgo_set_threads(int t) {
  if (t > 0) omp_set_num_threads(t);
}

/* rowptr [n+1], colidx [nnz]: the shared CSR pattern; vals_e [nnz][K]: the
 * values of A_k on it, edge by edge (v_k^{rc} at vals_e[e K + k]); kab [T][3]
 * and g [T]: the nonzero triple products <psi_k psi_a psi_b>; P <= 512. */
void sgo_apply(int64_t n, int P, int K, const int64_t* rowptr, const int64_t* colidx, int64_t nnz,
               const double* vals_e, int64_t T, const int64_t* kab, const double* g, const double* x,
               double* y) {
  (void)nnz;
#pragma omp parallel
  {
    double yr[512];
    double xc[512];
#pragma omp for schedule(static)
    for (int64_t r = 0; r < n; ++r) {
      for (int a = 0; a < P; ++a) yr[a] = 0.0;
      for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) {
        const int64_t c = colidx[e];
        const double* v = vals_e + e * K;
        for (int b = 0; b < P; ++b) xc[b] = x[(int64_t)b * n + c];
        for (int64_t t = 0; t < T; ++t) {
          const int64_t k = kab[3 * t], a = kab[3 * t + 1], b = kab[3 * t + 2];
          yr[a] += v[k] * g[t] * xc[b];
        }
      }
      for (int a = 0; a < P; ++a) y[(int64_t)a * n + r] = yr[a];
    }
  }
}

/* Lower banded Cholesky factor of A_0 (A_0 = L L^T) with bandwidth bw,
 * stored by columns: lb[j (bw+1) + d] = L[j+d][j], d = 0..bw (entries past
 * row n-1 unused).  b and x are P vectors of n (mode-major); x may equal b.
 * Each thread substitutes a group of modes together, so one pass over the
 * factor serves the whole group. */
void sgo_band_solve(int64_t n, int64_t bw, const double* lb, int P, const double* b, double* x) {
  const int nt = omp_get_max_threads();
  const int gs = (P + nt - 1) / nt < 1 ? 1 : (P + nt - 1) / nt;
  const int ng = (P + gs - 1) / gs;
#pragma omp parallel for schedule(dynamic, 1)
  for (int grp = 0; grp < ng; ++grp) {
    const int a0 = grp * gs, a1 = (a0 + gs < P) ? a0 + gs : P;
    for (int a = a0; a < a1; ++a)
      if (x + (int64_t)a * n != b + (int64_t)a * n) memcpy(x + (int64_t)a * n, b + (int64_t)a * n, sizeof(double) * n);
    /* L y = b, column by column */
    for (int64_t j = 0; j < n; ++j) {
      const double* col = lb + j * (bw + 1);
      const int64_t dmax = (n - 1 - j) < bw ? (n - 1 - j) : bw;
      for (int a = a0; a < a1; ++a) {
        double* v = x + (int64_t)a * n;
        const double yj = v[j] / col[0];
        v[j] = yj;
        for (int64_t d = 1; d <= dmax; ++d) v[j + d] -= col[d] * yj;
      }
    }
    /* L^T x = y, row j of L^T is column j of L */
    for (int64_t j = n - 1; j >= 0; --j) {
      const double* col = lb + j * (bw + 1);
      const int64_t dmax = (n - 1 - j) < bw ? (n - 1 - j) : bw;
      for (int a = a0; a < a1; ++a) {
        double* v = x + (int64_t)a * n;
        double s = v[j];
        for (int64_t d = 1; d <= dmax; ++d) s -= col[d] * v[j + d];
        v[j] = s / col[0];
      }
    }
  }
}

double sgo_dot(int64_t len, const double* u, const double* v) {
  int nt = omp_get_max_threads();
  double* part = (double*)calloc((size_t)nt, sizeof(double));
  if (!part) return NAN;
#pragma omp parallel
  {
    const int t = omp_get_thread_num(), tn = omp_get_num_threads();
    const int64_t lo = len * t / tn, hi = len * (t + 1) / tn;
    double s = 0.0;
    for (int64_t i = lo; i < hi; ++i) s += u[i] * v[i];
    part[t] = s;
  }
  double s = 0.0;
  for (int t = 0; t < nt; ++t) s += part[t];
  free(part);
  return s;
}

/* y += alpha x */
void sgo_axpy(int64_t len, double alpha, const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < len; ++i) y[i] += alpha * x[i];
}

/* y = alpha x */
void sgo_scal(int64_t len, double alpha, const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < len; ++i) y[i] = alpha * x[i];
}
