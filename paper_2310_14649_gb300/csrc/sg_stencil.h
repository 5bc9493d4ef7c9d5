// The five-point P1 stencil of a piecewise-constant coefficient on the
// structured "/" mesh (Sec. 2.1: A(c) = sum_e c_e K_e with K_e the unit P1
// element stiffness).  Shared by the assembly of the linear problem's A_k
// and by the nonlinear problem's per-step operators.
#pragma once

#include <cstdint>

namespace sg {

// Row (i, j) (interior node, 1 <= i, j <= N-1) of A(c) for one coefficient
// field c over the 2 N^2 triangles (element 2 (j N + i) is the lower and
// 2 (j N + i) + 1 the upper triangle of cell (i, j)).  Slots in ascending
// column order: south, west, centre, east, north; entries outside the
// interior are 0.  The hypotenuse couplings vanish on this mesh.
template <typename T, typename C>
__host__ __device__ inline void p1_stencil(const C* c, int N, int i, int j, T v[5]) {
  const int m = N - 1;
  auto lo = [&](int ci, int cj) { return T(c[2LL * (int64_t(cj) * N + ci)]); };
  auto up = [&](int ci, int cj) { return T(c[2LL * (int64_t(cj) * N + ci) + 1]); };
  v[0] = (j > 1) ? T(-0.5) * (up(i, j - 1) + lo(i - 1, j - 1)) : T(0);
  v[1] = (i > 1) ? T(-0.5) * (lo(i - 1, j) + up(i - 1, j - 1)) : T(0);
  v[2] = T(0.5) * lo(i, j) + T(0.5) * up(i, j) + lo(i - 1, j) + up(i, j - 1) + T(0.5) * lo(i - 1, j - 1) +
         T(0.5) * up(i - 1, j - 1);
  v[3] = (i < m) ? T(-0.5) * (lo(i, j) + up(i, j - 1)) : T(0);
  v[4] = (j < m) ? T(-0.5) * (up(i, j) + lo(i - 1, j)) : T(0);
}

}  // namespace sg
