// Learned smoother (sg_cnn.cu): network state and its operations.
#pragma once

#include "sg_solver.h"

namespace sg {

struct MeanSolver;

constexpr int kTcWaitDefault = 1 << 22;  // mbarrier polls before a tcgen05 kernel reports a timeout

int64_t cnn_param_count();          // parameters in the oracle layout
int64_t cnn_param_count_padded();   // parameters in the padded kernel layout

struct Cnn {
  bool ready = false, trained = false;
  int H = 0, W = 0, cap = 0, adam_t = 0;
  int64_t woff[5] = {}, boff[5] = {};
  DevBuf params, grads, adam_m, adam_v;  // FP32, padded layout
  DevBuf wf[5], wr[5];                   // BF16 forward and flipped weights
  DevBuf logd;                           // log(diag(A_0) / 4) per node
  DevBuf act[5], gbuf[2], out, ztgt;     // activations, gradients, FP32 output, targets
  DevBuf sumsq, lossbuf;                 // per-image scalars
  MeanSolver* mean = nullptr;            // batched A_0 solves (training targets)
  int loss_kind = 0;                     // 0 energy norm of A_0, 1 relative L2 error
  bool use_tc = true;                    // forward on tcgen05 (false: mma.sync)
  DevBuf wtc[5];                         // BF16 weights in the tcgen05 plane layout
  DevBuf wtcr[5];                        // flipped, transposed weights (input gradient), same layout
  DevBuf tcerr;                          // set by a tcgen05 kernel whose wait timed out
  int wait_limit = kTcWaitDefault;       // mbarrier polls of a tcgen05 completion wait
  DevCsr A0;                             // fine mean matrix (energy loss)
  DevBuf ebuf, aebuf, azbuf;             // error, A_0 error, A_0 target (energy loss)
  Cnn() = default;
  Cnn(const Cnn&) = delete;
  Cnn& operator=(const Cnn&) = delete;
  ~Cnn();

  sg_status init(const std::vector<double>& logdiag, int H, int W, const std::vector<int32_t>& rowptr,
                 const std::vector<int32_t>& colidx, const std::vector<double>& a0);
  sg_status reserve(int nimg);
  sg_status set_weights(const float* host_oracle_layout, cudaStream_t st);
  sg_status get_weights(float* host_oracle_layout, bool grad, cudaStream_t st);
  sg_status pack(cudaStream_t st);
  sg_status forward(int nimg, cudaStream_t st);
  sg_status backward(int nimg, cudaStream_t st);
  template <typename T>
  sg_status pack_input(const T* R, int64_t ld, int nimg, cudaStream_t st);
  template <typename T>
  sg_status unpack_output(T* Z, int64_t ld, int nimg, cudaStream_t st);
  // targets in network units from residual-unit targets (after pack_input)
  sg_status scale_targets(const float* Z, int64_t ld, int nimg, cudaStream_t st);
  sg_status loss_and_grad(int nimg, double* host_loss, cudaStream_t st);
  sg_status adam(float lr, cudaStream_t st);
};

// z = S_cnn r on the P mode images of R (ld rows each): the network per
// mode, then omega_cnn G~^{-1} across modes at every node when transform
template <typename T>
sg_status cnn_smooth(sg_problem* pr, const Precond& pc, const T* R, int64_t ld, T* Z, bool transform,
                     cudaStream_t st);
// the preconditioner attached to a problem (after sg_precond_setup)
Precond& precond_of(sg_problem* pr);
// tcgen05 forward convolution (sg_conv_tc.cu)
sg_status conv_tc_attrs();
sg_status conv_tc_pack(const float* Wsrc, int ci_pad, int co_pad, void* out, bool rev, cudaStream_t st);
sg_status conv_tc_wgrad(int l, const void* X, const void* G, float* dW, float* db, int H, int W, int nimg, int* err,
                        int wait_limit, cudaStream_t st);
sg_status conv_tc_dgrad(int l, const void* G, const void* Wr, const void* mask, void* Yb, int H, int W, int nimg,
                        int* err, int wait_limit, cudaStream_t st);
sg_status conv_tc_layer(int l, const void* X, const void* Wp, const float* b, void* Yb, float* Yf, int H, int W,
                        int nimg, int* err, int wait_limit, cudaStream_t st);
// selects the learned smoother with damping omega (estimated when <= 0)
sg_status learned_smoother_enable(sg_problem* pr, double omega, cudaStream_t st);
// He-normal weights (std sqrt(2 / fan_in)), zero biases, in the oracle
// layout, from a splitmix64 stream and the Box-Muller transform
std::vector<float> cnn_he_init(uint64_t seed);

}  // namespace sg
