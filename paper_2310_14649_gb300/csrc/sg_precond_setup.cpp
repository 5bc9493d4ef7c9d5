// Host-side setup of the two-grid preconditioner of Sec. 3:
//  * restricted additive Schwarz boxes with overlap grown on the graph of
//    A_0 (Eq. RASsto) and block-tridiagonal Cholesky factors of every local
//    mean block;
//  * the nested 2h coarse space: P1 interpolation R_0^T and the pattern and
//    assembly plan of the Galerkin coarse matrices R_0 A_k R_0^T (Eq. coarse);
//  * a smoothed-aggregation AMG hierarchy on the coarse mean matrix (the
//    paper's BoomerAMG role; parameters are a stated reading).
#include <algorithm>
#include <cmath>
#include <array>
#include <set>

#include "sg_solver.h"

namespace sg {

sg_status DevCsr::upload(int64_t rows, int64_t cols, const std::vector<int32_t>& rp,
                         const std::vector<int32_t>& ci, const std::vector<double>& v) {
  n = rows;
  m = cols;
  nnz = int64_t(ci.size());
  std::vector<float> h32(v.begin(), v.end());
  SG_TRY(rowptr.alloc(rp.size() * sizeof(int32_t)));
  SG_TRY(col.alloc(std::max<size_t>(1, ci.size()) * sizeof(int32_t)));
  SG_TRY(v64.alloc(std::max<size_t>(1, v.size()) * sizeof(double)));
  SG_TRY(v32.alloc(std::max<size_t>(1, v.size()) * sizeof(float)));
  SG_CUDA(cudaMemcpy(rowptr.ptr, rp.data(), rp.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  if (!ci.empty()) {
    SG_CUDA(cudaMemcpy(col.ptr, ci.data(), ci.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    SG_CUDA(cudaMemcpy(v64.ptr, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice));
    SG_CUDA(cudaMemcpy(v32.ptr, h32.data(), h32.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
  return SG_OK;
}

namespace {

// Host CSR helper (FP64).
struct HCsr {
  int64_t n = 0, m = 0;
  std::vector<int32_t> rp, ci;
  std::vector<double> v;
  double at(int64_t i, int64_t j) const {
    for (int32_t t = rp[i]; t < rp[i + 1]; ++t)
      if (ci[t] == j) return v[t];
    return 0.0;
  }
};

HCsr transpose(const HCsr& A) {
  HCsr T;
  T.n = A.m;
  T.m = A.n;
  T.rp.assign(T.n + 1, 0);
  for (int32_t c : A.ci) T.rp[c + 1]++;
  for (int64_t i = 0; i < T.n; ++i) T.rp[i + 1] += T.rp[i];
  T.ci.resize(A.ci.size());
  T.v.resize(A.v.size());
  std::vector<int32_t> fill(T.rp.begin(), T.rp.end() - 1);
  for (int64_t i = 0; i < A.n; ++i)
    for (int32_t t = A.rp[i]; t < A.rp[i + 1]; ++t) {
      int32_t d = fill[A.ci[t]]++;
      T.ci[d] = int32_t(i);
      T.v[d] = A.v[t];
    }
  return T;
}

// C = A * B (Gustavson), columns sorted, explicit zeros kept.
HCsr matmul(const HCsr& A, const HCsr& B) {
  HCsr C;
  C.n = A.n;
  C.m = B.m;
  C.rp.assign(C.n + 1, 0);
  std::vector<int32_t> mark(B.m, -1);
  std::vector<double> acc(B.m, 0.0);
  std::vector<int32_t> cols;
  for (int64_t i = 0; i < A.n; ++i) {
    cols.clear();
    for (int32_t t = A.rp[i]; t < A.rp[i + 1]; ++t) {
      int32_t k = A.ci[t];
      double a = A.v[t];
      for (int32_t u = B.rp[k]; u < B.rp[k + 1]; ++u) {
        int32_t j = B.ci[u];
        if (mark[j] != i) {
          mark[j] = int32_t(i);
          acc[j] = 0.0;
          cols.push_back(j);
        }
        acc[j] += a * B.v[u];
      }
    }
    std::sort(cols.begin(), cols.end());
    for (int32_t j : cols) {
      C.ci.push_back(j);
      C.v.push_back(acc[j]);
    }
    C.rp[i + 1] = int32_t(C.ci.size());
  }
  return C;
}

// ------------------------------------------------------------------------
// dense helpers (row-major w x w)
void chol_lower(std::vector<double>& A, int w) {  // in place, lower
  for (int j = 0; j < w; ++j) {
    double d = A[j * w + j];
    for (int k = 0; k < j; ++k) d -= A[j * w + k] * A[j * w + k];
    d = std::sqrt(d);
    A[j * w + j] = d;
    for (int i = j + 1; i < w; ++i) {
      double s = A[i * w + j];
      for (int k = 0; k < j; ++k) s -= A[i * w + k] * A[j * w + k];
      A[i * w + j] = s / d;
    }
    for (int k = j + 1; k < w; ++k) A[j * w + k] = 0.0;
  }
}

std::vector<double> lower_inverse(const std::vector<double>& L, int w) {
  std::vector<double> X(size_t(w) * w, 0.0);
  for (int c = 0; c < w; ++c) {  // solve L x = e_c
    for (int i = 0; i < w; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int k = c; k < i; ++k) s -= L[i * w + k] * X[k * w + c];
      X[i * w + c] = (i < c) ? 0.0 : s / L[i * w + i];
    }
  }
  return X;
}

}  // namespace

// --------------------------------------------------------------------------
// RAS partitions and local factors
// --------------------------------------------------------------------------
static sg_status setup_ras(sg_problem* pr, Precond& pc) {
  RasData& R = pc.ras;
  const int N = pr->N, m = N - 1;
  const int64_t n = pr->n;
  R.nbox = pc.sx * pc.sy;
  R.flops_per_mode = 0.0;
  std::vector<int32_t> owner(n);
  for (int64_t r = 0; r < n; ++r) {
    int i = int(r % m) + 1, j = int(r / m) + 1;
    int bx = int(int64_t(i - 1) * pc.sx / m), by = int(int64_t(j - 1) * pc.sy / m);
    owner[r] = by * pc.sx + bx;
  }
  R.idx.assign(R.nbox, {});
  R.owned.assign(R.nbox, {});
  R.nlines.assign(R.nbox, 0);
  R.wmax = 1;
  R.lmax = 1;
  std::vector<char> mem(n, 0), grow(n, 0);
  // line structure per box: (row j, first i, length)
  std::vector<std::vector<std::array<int32_t, 3>>> lines(R.nbox);
  for (int b = 0; b < R.nbox; ++b) {
    std::fill(mem.begin(), mem.end(), 0);
    for (int64_t r = 0; r < n; ++r) mem[r] = owner[r] == b;
    for (int d = 0; d < pc.overlap; ++d) {
      std::fill(grow.begin(), grow.end(), 0);
      for (int64_t r = 0; r < n; ++r)
        if (mem[r])
          for (int32_t t = pr->rowptr[r]; t < pr->rowptr[r + 1]; ++t) grow[pr->colidx[t]] = 1;
      for (int64_t r = 0; r < n; ++r) mem[r] |= grow[r];
    }
    for (int64_t r = 0; r < n; ++r)
      if (mem[r]) {
        R.idx[b].push_back(int32_t(r));
        R.owned[b].push_back(owner[r] == b ? 1 : 0);
      }
    // group into grid rows; each must be one contiguous run of columns
    for (size_t t = 0; t < R.idx[b].size();) {
      int32_t r0 = R.idx[b][t];
      int32_t j = r0 / m;
      size_t u = t;
      while (u < R.idx[b].size() && R.idx[b][u] / m == j) {
        if (R.idx[b][u] != r0 + int32_t(u - t)) {
          set_error("RAS setup: a grid row of an overlapped box is not contiguous");
          return SG_ERR_ARG;
        }
        ++u;
      }
      lines[b].push_back({j, r0 % m, int32_t(u - t)});
      R.wmax = std::max<int>(R.wmax, int(u - t));
      t = u;
    }
    R.nlines[b] = int32_t(lines[b].size());
    R.lmax = std::max<int>(R.lmax, R.nlines[b]);
    // forward and backward sweep: the sub-diagonal block (w_l x w_{l-1}) and
    // the triangular inverse (w_l (w_l + 1) / 2) per line, 2 flops per term
    for (size_t l = 0; l < lines[b].size(); ++l) {
      const double w = lines[b][l][2], wp = l ? lines[b][l - 1][2] : 0.0;
      R.flops_per_mode += 2.0 * 2.0 * (w * wp + 0.5 * w * (w + 1.0));
    }
  }
  R.wmax = int(round_up(R.wmax, 4));  // 16-byte matrix rows for cp.async
  const int W = R.wmax, Lm = R.lmax;
  const size_t per_line = size_t(W) * W;
  std::vector<double> linv(size_t(R.nbox) * Lm * per_line, 0.0), loff(linv.size(), 0.0);
  std::vector<int32_t> gidx(size_t(R.nbox) * Lm * W, -1);
  auto a0 = [&](int64_t r, int64_t c) {
    for (int32_t t = pr->rowptr[r]; t < pr->rowptr[r + 1]; ++t)
      if (pr->colidx[t] == c) return pr->a0[t];
    return 0.0;
  };
  for (int b = 0; b < R.nbox; ++b) {
    std::vector<double> Lprev;  // L_{j-1,j-1}
    for (int l = 0; l < R.nlines[b]; ++l) {
      auto [j, x0, len] = lines[b][l];
      for (int t = 0; t < len; ++t) {
        int64_t r = int64_t(j) * m + x0 + t;
        bool own = owner[r] == b;
        gidx[(size_t(b) * Lm + l) * W + t] = int32_t(r) | (own ? (1 << 30) : 0);
      }
      // D = A_jj - L_{j,j-1} L_{j,j-1}^T
      std::vector<double> D(per_line, 0.0), Loff(per_line, 0.0);
      for (int t = 0; t < W; ++t) D[t * W + t] = 1.0;  // padding slots decouple
      for (int t = 0; t < len; ++t) {
        int64_t r = int64_t(j) * m + x0 + t;
        D[t * W + t] = a0(r, r);
        if (t > 0) D[t * W + t - 1] = a0(r, r - 1);
        if (t + 1 < len) D[t * W + t + 1] = a0(r, r + 1);
      }
      if (l > 0) {
        auto [jp, xp, lenp] = lines[b][l - 1];
        // A_{j,j-1}[t][u]: node (x0+t, j) couples with (xp+u, j-1) when same column
        std::vector<double> Aoff(per_line, 0.0);
        for (int t = 0; t < len; ++t) {
          int u = x0 + t - xp;
          if (u >= 0 && u < lenp) {
            int64_t r = int64_t(j) * m + x0 + t;
            Aoff[t * W + u] = a0(r, r - m);
          }
        }
        // Loff = Aoff * Lprev^{-T}: solve Loff Lprev^T = Aoff row by row
        for (int t = 0; t < W; ++t)
          for (int u = 0; u < W; ++u) {
            double s = Aoff[t * W + u];
            for (int k = 0; k < u; ++k) s -= Loff[t * W + k] * Lprev[u * W + k];
            Loff[t * W + u] = s / Lprev[u * W + u];
          }
        for (int t = 0; t < W; ++t)
          for (int u = 0; u <= t; ++u) {
            double s = 0.0;
            for (int k = 0; k < W; ++k) s += Loff[t * W + k] * Loff[u * W + k];
            D[t * W + u] -= s;
            if (u != t) D[u * W + t] -= s;
          }
      }
      chol_lower(D, W);
      std::vector<double> Dinv = lower_inverse(D, W);
      std::copy(Dinv.begin(), Dinv.end(), linv.begin() + (size_t(b) * Lm + l) * per_line);
      std::copy(Loff.begin(), Loff.end(), loff.begin() + (size_t(b) * Lm + l) * per_line);
      Lprev = D;
    }
  }
  std::vector<float> linv32(linv.begin(), linv.end()), loff32(loff.begin(), loff.end());
  SG_TRY(R.linv64.alloc(linv.size() * 8));
  SG_TRY(R.loff64.alloc(loff.size() * 8));
  SG_TRY(R.linv32.alloc(linv.size() * 4));
  SG_TRY(R.loff32.alloc(loff.size() * 4));
  SG_TRY(R.d_gidx.alloc(gidx.size() * 4));
  SG_TRY(R.d_nlines.alloc(R.nlines.size() * 4));
  SG_CUDA(cudaMemcpy(R.linv64.ptr, linv.data(), linv.size() * 8, cudaMemcpyHostToDevice));
  SG_CUDA(cudaMemcpy(R.loff64.ptr, loff.data(), loff.size() * 8, cudaMemcpyHostToDevice));
  SG_CUDA(cudaMemcpy(R.linv32.ptr, linv32.data(), linv32.size() * 4, cudaMemcpyHostToDevice));
  SG_CUDA(cudaMemcpy(R.loff32.ptr, loff32.data(), loff32.size() * 4, cudaMemcpyHostToDevice));
  SG_CUDA(cudaMemcpy(R.d_gidx.ptr, gidx.data(), gidx.size() * 4, cudaMemcpyHostToDevice));
  SG_CUDA(cudaMemcpy(R.d_nlines.ptr, R.nlines.data(), R.nlines.size() * 4, cudaMemcpyHostToDevice));
  return SG_OK;
}

// --------------------------------------------------------------------------
// Coarse space: nested 2h mesh with the same "/" split.  Fine node (i, j)
// interpolates from coarse nodes by parity: (even, even) -> itself;
// (odd, even) -> left/right; (even, odd) -> below/above; (odd, odd) -> the
// two ends of the coarse "/" diagonal through it, weight 1/2 each.  Coarse
// nodes on the boundary carry u = 0 and are dropped.
// --------------------------------------------------------------------------
static void interp_of(int N, int i, int j, std::vector<std::pair<int32_t, double>>& out) {
  const int Nc = N / 2, mc = Nc - 1;
  out.clear();
  auto add = [&](int I, int J, double w) {
    if (I >= 1 && I <= mc && J >= 1 && J <= mc) out.push_back({int32_t((J - 1) * mc + (I - 1)), w});
  };
  if (i % 2 == 0 && j % 2 == 0) {
    add(i / 2, j / 2, 1.0);
  } else if (i % 2 == 1 && j % 2 == 0) {
    add((i - 1) / 2, j / 2, 0.5);
    add((i + 1) / 2, j / 2, 0.5);
  } else if (i % 2 == 0 && j % 2 == 1) {
    add(i / 2, (j - 1) / 2, 0.5);
    add(i / 2, (j + 1) / 2, 0.5);
  } else {
    add((i - 1) / 2, (j - 1) / 2, 0.5);
    add((i + 1) / 2, (j + 1) / 2, 0.5);
  }
}

static sg_status setup_coarse(sg_problem* pr, Precond& pc, CoarsePlan& plan, HCsr& Ac0) {
  CoarseData& C = pc.co;
  const int N = pr->N, m = N - 1;
  C.Nc = N / 2;
  const int mc = C.Nc - 1;
  C.nc = int64_t(mc) * mc;
  C.ldc = round_up(C.nc, 64);
  const Ell& F = pr->fine;
  // interpolation (fine rows)
  std::vector<std::vector<std::pair<int32_t, double>>> ip(pr->n);
  std::vector<std::pair<int32_t, double>> tmp;
  for (int64_t f = 0; f < pr->n; ++f) {
    interp_of(N, int(f % m) + 1, int(f / m) + 1, tmp);
    ip[f] = tmp;
  }
  HCsr RT;
  RT.n = pr->n;
  RT.m = C.nc;
  RT.rp.assign(pr->n + 1, 0);
  for (int64_t f = 0; f < pr->n; ++f) {
    auto s = ip[f];
    std::sort(s.begin(), s.end());
    for (auto& e : s) {
      RT.ci.push_back(e.first);
      RT.v.push_back(e.second);
    }
    RT.rp[f + 1] = int32_t(RT.ci.size());
  }
  HCsr R = transpose(RT);
  SG_TRY(C.RT.upload(RT.n, RT.m, RT.rp, RT.ci, RT.v));
  SG_TRY(C.R.upload(R.n, R.m, R.rp, R.ci, R.v));
  // fine slot columns on the host (same rule as the device ELL)
  auto fine_col = [&](int s, int64_t r) -> int64_t {
    int i = int(r % m) + 1, j = int(r / m) + 1;
    switch (s) {
      case 0: return j > 1 ? r - m : -1;
      case 1: return i > 1 ? r - 1 : -1;
      case 2: return r;
      case 3: return i < m ? r + 1 : -1;
      default: return j < m ? r + m : -1;
    }
  };
  // symbolic coarse pattern
  std::vector<std::set<int32_t>> pat(C.nc);
  for (int64_t f = 0; f < pr->n; ++f)
    for (int s = 0; s < 5; ++s) {
      int64_t c = fine_col(s, f);
      if (c < 0) continue;
      for (auto& I : ip[f])
        for (auto& J : ip[c]) pat[I.first].insert(J.first);
    }
  C.rowptr.assign(C.nc + 1, 0);
  C.colidx.clear();
  int S = 1;
  for (int64_t I = 0; I < C.nc; ++I) {
    if (pat[I].empty()) pat[I].insert(int32_t(I));
    for (int32_t J : pat[I]) C.colidx.push_back(J);
    C.rowptr[I + 1] = int32_t(C.colidx.size());
    S = std::max<int>(S, int(pat[I].size()));
  }
  C.ell.S = S;
  C.ell.n = C.nc;
  C.ell.ldr = C.ldc;
  std::vector<int32_t> ccol(size_t(S) * C.ldc, 0);
  for (int64_t I = 0; I < C.ldc; ++I)
    for (int s = 0; s < S; ++s) {
      if (I >= C.nc) {
        ccol[s * C.ldc + I] = 0;
        continue;
      }
      int32_t t = C.rowptr[I] + s;
      ccol[s * C.ldc + I] = t < C.rowptr[I + 1] ? C.colidx[t] : int32_t(I);
    }
  SG_TRY(C.ell.col.alloc(ccol.size() * 4));
  SG_CUDA(cudaMemcpy(C.ell.col.ptr, ccol.data(), ccol.size() * 4, cudaMemcpyHostToDevice));
  // plan
  std::vector<std::vector<std::pair<int64_t, double>>> contrib(size_t(S) * C.ldc);
  for (int64_t f = 0; f < pr->n; ++f)
    for (int s = 0; s < 5; ++s) {
      int64_t c = fine_col(s, f);
      if (c < 0) continue;
      for (auto& I : ip[f])
        for (auto& J : ip[c]) {
          int32_t lo = C.rowptr[I.first], hi = C.rowptr[I.first + 1];
          int32_t t = int32_t(std::lower_bound(C.colidx.begin() + lo, C.colidx.begin() + hi, J.first) -
                              C.colidx.begin());
          int sc = t - lo;
          contrib[size_t(sc) * C.ldc + I.first].push_back({int64_t(s) * F.ldr + f, I.second * J.second});
        }
    }
  plan.rp.assign(contrib.size() + 1, 0);
  for (size_t q = 0; q < contrib.size(); ++q) {
    for (auto& e : contrib[q]) {
      plan.src.push_back(e.first);
      plan.w.push_back(e.second);
    }
    plan.rp[q + 1] = int32_t(plan.src.size());
  }
  // coarse mean matrix on the host from A_0 (for the AMG setup)
  std::vector<double> a0ell(size_t(5) * F.ldr, 0.0);
  for (int64_t r = 0; r < pr->n; ++r)
    for (int32_t t = pr->rowptr[r]; t < pr->rowptr[r + 1]; ++t) {
      int64_t c = pr->colidx[t];
      int s = c == r ? 2 : (c == r - m ? 0 : (c == r - 1 ? 1 : (c == r + 1 ? 3 : 4)));
      a0ell[size_t(s) * F.ldr + r] = pr->a0[t];
    }
  Ac0.n = Ac0.m = C.nc;
  Ac0.rp = C.rowptr;
  Ac0.ci = C.colidx;
  Ac0.v.assign(C.colidx.size(), 0.0);
  for (int64_t I = 0; I < C.nc; ++I)
    for (int32_t t = C.rowptr[I]; t < C.rowptr[I + 1]; ++t) {
      int sc = t - C.rowptr[I];
      size_t q = size_t(sc) * C.ldc + I;
      double s = 0.0;
      for (int32_t u = plan.rp[q]; u < plan.rp[q + 1]; ++u) s += plan.w[u] * a0ell[plan.src[u]];
      Ac0.v[t] = s;
    }
  return SG_OK;
}

// --------------------------------------------------------------------------
// Smoothed aggregation on the coarse mean matrix.
// --------------------------------------------------------------------------
static const double kTheta = 0.08;
static const int kMaxCoarse = 256, kMaxLevels = 10, kPowerIts = 20;

static std::vector<std::vector<int32_t>> strong_graph(const HCsr& A) {
  std::vector<double> d(A.n);
  for (int64_t i = 0; i < A.n; ++i) d[i] = A.at(i, i);
  std::vector<std::vector<int32_t>> S(A.n);
  for (int64_t i = 0; i < A.n; ++i)
    for (int32_t t = A.rp[i]; t < A.rp[i + 1]; ++t) {
      int32_t j = A.ci[t];
      if (j != i && std::fabs(A.v[t]) >= kTheta * std::sqrt(std::fabs(d[i] * d[j]))) S[i].push_back(j);
    }
  for (auto& s : S) std::sort(s.begin(), s.end());
  return S;
}

static int32_t aggregate(const HCsr& A, std::vector<int32_t>& agg) {
  auto S = strong_graph(A);
  const int64_t n = A.n;
  agg.assign(n, -1);
  int32_t na = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    bool free_nb = true;
    for (int32_t j : S[i]) free_nb &= agg[j] < 0;
    if (!free_nb) continue;
    agg[i] = na;
    for (int32_t j : S[i]) agg[j] = na;
    ++na;
  }
  std::vector<int32_t> first = agg;
  for (int64_t i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    for (int32_t j : S[i])
      if (first[j] >= 0) {
        agg[i] = first[j];
        break;
      }
  }
  for (int64_t i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    agg[i] = na;
    for (int32_t j : S[i])
      if (agg[j] < 0) agg[j] = na;
    ++na;
  }
  return na;
}

static sg_status setup_amg(AmgHier& H, const HCsr& A0c) {
  H.lev.clear();
  HCsr A = A0c;
  std::vector<HCsr> As, Ps;
  std::vector<std::vector<int32_t>> aggs;
  for (;;) {
    As.push_back(A);
    if (A.n <= kMaxCoarse || int(As.size()) >= kMaxLevels) break;
    std::vector<int32_t> agg;
    int32_t na = aggregate(A, agg);
    if (na >= A.n) break;
    std::vector<double> size(na, 0.0);
    for (int32_t a : agg) size[a] += 1.0;
    HCsr Pt;
    Pt.n = A.n;
    Pt.m = na;
    Pt.rp.resize(A.n + 1);
    for (int64_t i = 0; i < A.n; ++i) {
      Pt.rp[i] = int32_t(i);
      Pt.ci.push_back(agg[i]);
      Pt.v.push_back(1.0 / std::sqrt(size[agg[i]]));
    }
    Pt.rp[A.n] = int32_t(A.n);
    // spectral radius of D^{-1} A by power iteration from x_i = 1 + (i mod 3)
    std::vector<double> x(A.n), y(A.n), dinv(A.n);
    for (int64_t i = 0; i < A.n; ++i) dinv[i] = 1.0 / A.at(i, i);
    double nx = 0.0;
    for (int64_t i = 0; i < A.n; ++i) {
      x[i] = 1.0 + double(i % 3);
      nx += x[i] * x[i];
    }
    nx = std::sqrt(nx);
    for (auto& v : x) v /= nx;
    double rho = 0.0;
    for (int it = 0; it < kPowerIts; ++it) {
      double s = 0.0;
      for (int64_t i = 0; i < A.n; ++i) {
        double acc = 0.0;
        for (int32_t t = A.rp[i]; t < A.rp[i + 1]; ++t) acc += A.v[t] * x[A.ci[t]];
        y[i] = dinv[i] * acc;
        s += y[i] * y[i];
      }
      rho = std::sqrt(s);
      for (int64_t i = 0; i < A.n; ++i) x[i] = y[i] / rho;
    }
    const double omega = 4.0 / (3.0 * rho);
    // P = Pt - omega D^{-1} A Pt
    HCsr AP = matmul(A, Pt);
    for (int64_t i = 0; i < AP.n; ++i)
      for (int32_t t = AP.rp[i]; t < AP.rp[i + 1]; ++t) AP.v[t] *= -omega * dinv[i];
    // add Pt (its entries are inside AP's pattern: the diagonal of A is nonzero)
    for (int64_t i = 0; i < A.n; ++i) {
      int32_t c = agg[i];
      bool found = false;
      for (int32_t t = AP.rp[i]; t < AP.rp[i + 1]; ++t)
        if (AP.ci[t] == c) {
          AP.v[t] += Pt.v[i];
          found = true;
        }
      if (!found) {
        set_error("AMG setup: tentative prolongator entry outside A P_t");
        return SG_ERR_ARG;
      }
    }
    HCsr P = AP;
    HCsr Rm = transpose(P);
    HCsr Anext = matmul(Rm, matmul(A, P));
    Ps.push_back(P);
    aggs.push_back(agg);
    A = Anext;
  }
  H.lev.resize(As.size());
  for (size_t l = 0; l < As.size(); ++l) {
    AmgLevel& L = H.lev[l];
    L.n = As[l].n;
    L.ld = round_up(L.n, 32);
    SG_TRY(L.A.upload(As[l].n, As[l].m, As[l].rp, As[l].ci, As[l].v));
    std::vector<double> dl1(L.n, 0.0);
    for (int64_t i = 0; i < L.n; ++i)
      for (int32_t t = As[l].rp[i]; t < As[l].rp[i + 1]; ++t) dl1[i] += std::fabs(As[l].v[t]);
    std::vector<double> di(L.n);
    std::vector<float> di32(L.n);
    for (int64_t i = 0; i < L.n; ++i) {
      di[i] = 1.0 / dl1[i];
      di32[i] = float(di[i]);
    }
    SG_TRY(L.dinv64.alloc(std::max<size_t>(1, L.n) * 8));
    SG_TRY(L.dinv32.alloc(std::max<size_t>(1, L.n) * 4));
    SG_CUDA(cudaMemcpy(L.dinv64.ptr, di.data(), L.n * 8, cudaMemcpyHostToDevice));
    SG_CUDA(cudaMemcpy(L.dinv32.ptr, di32.data(), L.n * 4, cudaMemcpyHostToDevice));
    if (l + 1 < As.size()) {
      HCsr Rm = transpose(Ps[l]);
      SG_TRY(L.Pm.upload(Ps[l].n, Ps[l].m, Ps[l].rp, Ps[l].ci, Ps[l].v));
      SG_TRY(L.R.upload(Rm.n, Rm.m, Rm.rp, Rm.ci, Rm.v));
      L.agg = aggs[l];
    }
  }
  // coarsest: explicit inverse from a dense Cholesky factor (FP64)
  const HCsr& Ac = As.back();
  const int nc = int(Ac.n);
  std::vector<double> D(size_t(nc) * nc, 0.0);
  for (int i = 0; i < nc; ++i)
    for (int32_t t = Ac.rp[i]; t < Ac.rp[i + 1]; ++t) D[size_t(i) * nc + Ac.ci[t]] = Ac.v[t];
  chol_lower(D, nc);
  std::vector<double> Li = lower_inverse(D, nc);
  std::vector<double> inv(size_t(nc) * nc, 0.0);  // L^{-T} L^{-1}
  for (int i = 0; i < nc; ++i)
    for (int j = 0; j < nc; ++j) {
      double s = 0.0;
      for (int k = std::max(i, j); k < nc; ++k) s += Li[size_t(k) * nc + i] * Li[size_t(k) * nc + j];
      inv[size_t(i) * nc + j] = s;
    }
  SG_TRY(H.coarsest_inv64.alloc(inv.size() * 8));
  SG_CUDA(cudaMemcpy(H.coarsest_inv64.ptr, inv.data(), inv.size() * 8, cudaMemcpyHostToDevice));
  return SG_OK;
}

sg_status amg_setup_fine(const sg_problem* pr, AmgHier& h) {
  HCsr A;
  A.n = pr->n;
  A.m = pr->n;
  A.rp = pr->rowptr;
  A.ci = pr->colidx;
  A.v = pr->a0;
  return setup_amg(h, A);
}

sg_status precond_setup_host(sg_problem* pr, Precond& pc) {
  SG_TRY(setup_ras(pr, pc));
  CoarsePlan plan;
  HCsr Ac0;
  SG_TRY(setup_coarse(pr, pc, plan, Ac0));
  SG_TRY(setup_amg(pc.amg, Ac0));
  SG_TRY(precond_setup_coarse_plan(pr, pc, plan));
  return SG_OK;
}

}  // namespace sg
