// Batched solves with the fine mean matrix A_0 (sg_train.cu).
#pragma once

#include "sg_kernels.h"

namespace sg {

// z = A_0^{-1} b for up to nb columns at once: conjugate gradients
// preconditioned by one smoothed-aggregation V(1,1) cycle of A_0, FP64.
struct MeanSolver {
  AmgHier H;
  int nb = 0;
  int64_t n = 0, ld = 0;
  DevBuf x, r, p, q, z, scal;
  std::vector<DevBuf> lev;
  AmgWork<double> w;

  sg_status init(const sg_problem* pr, int cols);
  // B, Z: FP32 columns (ldb, ldz rows); stops when every column has
  // ||b - A_0 z|| <= rtol ||b|| or after max_it iterations
  sg_status solve(const float* B, int64_t ldb, float* Z, int64_t ldz, int cols, double rtol, int max_it,
                  double* relres_max, int* its, cudaStream_t st);
};

}  // namespace sg
