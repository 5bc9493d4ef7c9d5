// Host-side setup of the SG system (Sec. 2.1): KL modes of the separable
// exponential kernel, multi-index sets, Hermite triple products, the shared
// CSR pattern of the stiffness matrices, the load vector and the mean
// stiffness matrix A_0 (kept on the host for the preconditioner setup).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <tuple>

#include "sg_internal.h"

namespace sg {

// ---------------------------------------------------------------------------
// Karhunen-Loeve modes (Sec. 2.1, Eqs. KLE and CovarKer2DNLP).  The paper
// cites, but does not print, the analytic eigenpairs; this is the standard
// 1D solution on [-a, a], a = 1/2, for the kernel exp(-|s - t| / b):
//   even:  theta tan(theta) = a / b,   theta in (k pi, k pi + pi/2)
//   odd:   theta cot(theta) = -a / b,  theta in (k pi + pi/2, (k+1) pi)
//   omega = theta / a,  lambda = 2 b / (1 + b^2 omega^2),
//   phi_even(s) = cos(omega s) / sqrt(a + sin(2 omega a) / (2 omega)),
//   phi_odd(s)  = sin(omega s) / sqrt(a - sin(2 omega a) / (2 omega)).
// Roots are bracketed until the bracket ends are adjacent doubles.
// ---------------------------------------------------------------------------
namespace {

struct Mode1 {
  double lam, omega;
  int odd;
};

constexpr double kHalf = 0.5;
constexpr double kPi = 3.14159265358979323846;

double bisect_root(const std::function<double(double)>& f, double lo, double hi, bool rising) {
  for (;;) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) return lo;
    double v = f(mid);
    bool below = rising ? (v < 0.0) : !(v < 0.0);
    if (below)
      lo = mid;
    else
      hi = mid;
  }
}

std::vector<Mode1> kl_modes_1d(double b, int count) {
  const double a = kHalf, c = 1.0 / b;
  std::vector<Mode1> out;
  for (int m = 0; m < count; ++m) {
    int k = m / 2;
    double theta;
    if (m % 2 == 0) {
      theta = bisect_root([&](double t) { return t * std::tan(t) - a * c; }, k * kPi,
                          k * kPi + 0.5 * kPi, true);
    } else {
      theta = bisect_root([&](double t) { return t / std::tan(t) + a * c; }, k * kPi + 0.5 * kPi,
                          (k + 1) * kPi, false);
    }
    double w = theta / a;
    out.push_back({2.0 * b / (1.0 + b * b * w * w), w, m % 2});
  }
  return out;
}

double kl_phi_1d(const Mode1& m, double s) {
  const double a = kHalf;
  if (!m.odd) return std::cos(m.omega * s) / std::sqrt(a + std::sin(2.0 * m.omega * a) / (2.0 * m.omega));
  return std::sin(m.omega * s) / std::sqrt(a - std::sin(2.0 * m.omega * a) / (2.0 * m.omega));
}

// 1D Hermite triple product <He_a He_b He_c> (linearisation formula).
int64_t he_triple(int a, int b, int c) {
  if ((a + b + c) & 1) return 0;
  int s = (a + b + c) / 2;
  if (s < a || s < b || s < c) return 0;
  auto fact = [](int v) {
    int64_t f = 1;
    for (int i = 2; i <= v; ++i) f *= i;
    return f;
  };
  return fact(a) * fact(b) * fact(c) / (fact(s - a) * fact(s - b) * fact(s - c));
}

double alpha_fact(const int32_t* alpha, int L) {
  double f = 1.0;
  for (int i = 0; i < L; ++i)
    for (int v = 2; v <= alpha[i]; ++v) f *= v;
  return f;
}

}  // namespace

// Total-degree multi-index set, degree ascending and lexicographically
// descending within one degree (compositions of d generated largest-first).
int64_t he_triple_1d(int a, int b, int c) { return he_triple(a, b, c); }

std::vector<int32_t> multi_indices(int L, int p) {
  std::vector<int32_t> out;
  std::vector<int32_t> cur(std::max(L, 1), 0);
  std::function<void(int, int)> rec = [&](int pos, int left) {
    if (pos == L - 1) {
      cur[pos] = left;
      out.insert(out.end(), cur.begin(), cur.begin() + L);
      return;
    }
    for (int v = left; v >= 0; --v) {
      cur[pos] = v;
      rec(pos + 1, left - v);
    }
  };
  if (L == 0) return out;  // a single empty index: caller handles L == 0
  for (int d = 0; d <= p; ++d) rec(0, d);
  return out;
}

sg_status build_host(sg_problem* pr, const sg_kl_desc* kl) {
  const int N = pr->N, L = pr->L;
  pr->E = 2LL * N * N;
  pr->n = int64_t(N - 1) * (N - 1);
  const double h = 1.0 / N;

  // -- multi-index sets and sizes
  if (L > 0) {
    pr->mi_out = multi_indices(L, pr->p);
    pr->mi_in = multi_indices(L, pr->q);
    pr->P = int(pr->mi_out.size() / L);
    pr->K = int(pr->mi_in.size() / L);
  } else {
    pr->P = 1;
    pr->K = 1;
  }

  // -- Gaussian field modes at triangle centroids
  pr->gfield.assign(size_t(L) * pr->E, 0.0);
  if (L > 0) {
    if (kl->user_modes) {
      std::memcpy(pr->gfield.data(), kl->user_modes, sizeof(double) * L * pr->E);
    } else {
      auto mx = kl_modes_1d(kl->bx, L);
      auto my = kl_modes_1d(kl->by, L);
      std::vector<std::tuple<double, int, int>> cand;
      for (int m = 0; m < L; ++m)
        for (int nn = 0; nn < L; ++nn)
          // sigma^2 (lambda_m lambda_n): the product of the two 1D values is
          // commutative, so the equal pairs (m, n), (n, m) of b_x = b_y stay
          // exactly equal and the (m, n) tie-break decides their order
          cand.emplace_back(-(kl->sigma2 * (mx[m].lam * my[nn].lam)), m, nn);
      std::sort(cand.begin(), cand.end());
      for (int i = 0; i < L; ++i) {
        double lam = -std::get<0>(cand[i]);
        const Mode1& ax = mx[std::get<1>(cand[i])];
        const Mode1& ay = my[std::get<2>(cand[i])];
        double sl = std::sqrt(lam);
        for (int cj = 0; cj < N; ++cj)
          for (int ci = 0; ci < N; ++ci) {
            // lower triangle (i,j),(i+1,j),(i+1,j+1); upper (i,j),(i+1,j+1),(i,j+1)
            double xl = double(3 * ci + 2) / 3.0 * h, yl = double(3 * cj + 1) / 3.0 * h;
            double xu = double(3 * ci + 1) / 3.0 * h, yu = double(3 * cj + 2) / 3.0 * h;
            int64_t e = 2LL * (int64_t(cj) * N + ci);
            pr->gfield[size_t(i) * pr->E + e] = sl * kl_phi_1d(ax, xl - kHalf) * kl_phi_1d(ay, yl - kHalf);
            pr->gfield[size_t(i) * pr->E + e + 1] = sl * kl_phi_1d(ax, xu - kHalf) * kl_phi_1d(ay, yu - kHalf);
          }
      }
    }
  }

  // -- triple products <psi_k psi_a psi_b>, ordered k, a, b
  pr->kab.clear();
  pr->num.clear();
  pr->g.clear();
  if (L == 0) {
    pr->kab = {0, 0, 0};
    pr->num = {1};
    pr->g = {1.0};
  } else {
    const int P = pr->P, K = pr->K;
    std::vector<double> fin(K), fout(P);
    for (int k = 0; k < K; ++k) fin[k] = alpha_fact(&pr->mi_in[size_t(k) * L], L);
    for (int a = 0; a < P; ++a) fout[a] = alpha_fact(&pr->mi_out[size_t(a) * L], L);
    for (int k = 0; k < K; ++k)
      for (int a = 0; a < P; ++a)
        for (int b = 0; b < P; ++b) {
          int64_t v = 1;
          for (int i = 0; i < L && v; ++i)
            v *= he_triple(pr->mi_in[size_t(k) * L + i], pr->mi_out[size_t(a) * L + i],
                           pr->mi_out[size_t(b) * L + i]);
          if (!v) continue;
          pr->kab.insert(pr->kab.end(), {k, a, b});
          pr->num.push_back(v);
          pr->g.push_back(double(v) / std::sqrt(fin[k] * fout[a] * fout[b]));
        }
  }
  pr->T = int64_t(pr->num.size());

  // -- mean coefficient c_0 = exp(g0 + 1/2 sum g_i^2) per triangle, A_0 on
  //    the host and the shared pattern (A_0's nonzeros).
  std::vector<double> c0(pr->E);
  for (int64_t e = 0; e < pr->E; ++e) {
    double s = 0.0;
    for (int i = 0; i < L; ++i) s += pr->gfield[size_t(i) * pr->E + e] * pr->gfield[size_t(i) * pr->E + e];
    c0[e] = std::exp(pr->g0 + 0.5 * s);
  }
  const int m = N - 1;
  auto lo = [&](int ci, int cj) { return c0[2LL * (int64_t(cj) * N + ci)]; };
  auto up = [&](int ci, int cj) { return c0[2LL * (int64_t(cj) * N + ci) + 1]; };
  pr->rowptr.assign(pr->n + 1, 0);
  pr->colidx.clear();
  pr->a0.clear();
  for (int j = 1; j <= m; ++j)
    for (int i = 1; i <= m; ++i) {
      int64_t r = int64_t(j - 1) * m + (i - 1);
      // stencil slots in ascending column order: south, west, centre, east, north
      double vs = -0.5 * (up(i, j - 1) + lo(i - 1, j - 1));
      double vw = -0.5 * (lo(i - 1, j) + up(i - 1, j - 1));
      double vc = 0.5 * lo(i, j) + 0.5 * up(i, j) + lo(i - 1, j) + up(i, j - 1) + 0.5 * lo(i - 1, j - 1) +
                  0.5 * up(i - 1, j - 1);
      double ve = -0.5 * (lo(i, j) + up(i, j - 1));
      double vn = -0.5 * (up(i, j) + lo(i - 1, j));
      auto push = [&](bool inside, int64_t col, double v) {
        if (inside && v != 0.0) {
          pr->colidx.push_back(int32_t(col));
          pr->a0.push_back(v);
        }
      };
      push(j > 1, r - m, vs);
      push(i > 1, r - 1, vw);
      push(true, r, vc);
      push(i < m, r + 1, ve);
      push(j < m, r + m, vn);
      pr->rowptr[r + 1] = int32_t(pr->colidx.size());
    }
  pr->nnzA = int64_t(pr->colidx.size());
  pr->b.assign(pr->n, h * h);
  return SG_OK;
}

}  // namespace sg

// ---------------------------------------------------------------------------
// Fourfold products of the nonlinear problem (Sec. 2.2, t_ijkl of Eq.
// stonlp_system).  1D: He_a He_b = sum_m (<He_a He_b He_m> / m!) He_m, so
// <He_a He_b He_c He_d> = sum_m (<He_a He_b He_m> / m!) <He_m He_c He_d>;
// every factor is an integer.  Multi-dimensional values are products over
// the dimensions.  Integers are formed in 128 bits and must fit 64.
// ---------------------------------------------------------------------------
namespace {

using i128 = __int128;

i128 fact128(int v) {
  i128 f = 1;
  for (int i = 2; i <= v; ++i) f *= i;
  return f;
}

// <He_a He_b He_c> with a = y + z, b = x + z, c = x + y: a! b! c! / (x! y! z!)
i128 he_triple128(int a, int b, int c) {
  if ((a + b + c) & 1) return 0;
  const int s = (a + b + c) / 2;
  if (s < a || s < b || s < c) return 0;
  return fact128(a) * fact128(b) * fact128(c) / (fact128(s - a) * fact128(s - b) * fact128(s - c));
}

const i128 kI64Max = i128(INT64_MAX);

}  // namespace

extern "C" sg_status sg_fourfold_products(int L, int p, int q, int64_t* count, int32_t* ijkl, int64_t* num,
                                          double* t) {
  using sg::set_error;
  SG_ARG(count, "sg_fourfold_products: NULL count");
  SG_ARG(L >= 1 && L <= 12 && p >= 0 && p <= 8 && q >= 0 && q <= 16,
         "sg_fourfold_products: need 1 <= L <= 12, 0 <= p <= 8, 0 <= q <= 16");
  // 1D table q1[a][b][c][d], a <= q (input degree), b, c, d <= p
  const int Q = q + 1, R = p + 1;
  std::vector<int64_t> q1(size_t(Q) * R * R * R, 0);
  for (int a = 0; a <= q; ++a)
    for (int b = 0; b <= p; ++b)
      for (int c = 0; c <= p; ++c)
        for (int d = 0; d <= p; ++d) {
          i128 tot = 0;
          for (int m = 0; m <= a + b; ++m) {
            const i128 tab = he_triple128(a, b, m);
            if (tab == 0) continue;
            tot += tab / fact128(m) * he_triple128(m, c, d);
          }
          if (tot > kI64Max || tot < -kI64Max) {
            set_error("sg_fourfold_products: a 1D fourfold moment exceeds 64 bits");
            return SG_ERR_UNSUPPORTED;
          }
          q1[((size_t(a) * R + b) * R + c) * R + d] = int64_t(tot);
        }
  const std::vector<int32_t> in = sg::multi_indices(L, q), out = sg::multi_indices(L, p);
  const int64_t K = int64_t(in.size()) / L, P = int64_t(out.size()) / L;
  auto fact_of = [&](const int32_t* al) {
    double f = 1.0;
    for (int d = 0; d < L; ++d)
      for (int v = 2; v <= al[d]; ++v) f *= v;
    return f;
  };
  const bool fill = ijkl || num || t;
  const int64_t cap = *count;
  int64_t n = 0;
  for (int64_t i = 0; i < K; ++i)
    for (int64_t j = 0; j < P; ++j)
      for (int64_t k = 0; k < P; ++k)
        for (int64_t l = 0; l < P; ++l) {
          i128 v = 1;
          for (int d = 0; d < L && v != 0; ++d) {
            const int64_t f = q1[((size_t(in[i * L + d]) * R + out[j * L + d]) * R + out[k * L + d]) * R +
                                 out[l * L + d]];
            v *= f;
            if (v > kI64Max || v < -kI64Max) {
              set_error("sg_fourfold_products: a fourfold product exceeds 64 bits");
              return SG_ERR_UNSUPPORTED;
            }
          }
          if (v == 0) continue;
          if (fill) {
            if (n >= cap) {
              set_error("sg_fourfold_products: *count is smaller than the number of products");
              return SG_ERR_ARG;
            }
            if (ijkl) {
              ijkl[4 * n] = int32_t(i);
              ijkl[4 * n + 1] = int32_t(j);
              ijkl[4 * n + 2] = int32_t(k);
              ijkl[4 * n + 3] = int32_t(l);
            }
            if (num) num[n] = int64_t(v);
            if (t)
              t[n] = double(int64_t(v)) / std::sqrt(fact_of(&in[i * L]) * fact_of(&out[j * L]) *
                                                    fact_of(&out[k * L]) * fact_of(&out[l * L]));
          }
          ++n;
        }
  *count = n;
  return SG_OK;
}
