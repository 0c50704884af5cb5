// flow_internal.h -- host-side declarations of the flow proposal (flow_kernels.cu, flow_api.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "flow.cuh"
#include "gwns_internal.h"

namespace gwns {

// Points per tile of the flow gradient: a tile fills the top half of the 128-row MMA operands (the
// rest are masked rows), so that twice as many CTAs share the survivors -- the kernel is bound by
// its per-layer latency, not by the tensor pipe.
constexpr int kGradRows = 64;

// Device buffers of one event's flow (all owned by the handle).
struct FlowHost {
  int enabled = 0;
  int n_layers = 0, n_params = 0, every = 1, epochs = 20;
  double p_flow = 0.0, lr = 1e-3;
  FlowDev* d_flow = nullptr;       // the FlowDev the kernels read (standardise/Adam update it)
  unsigned char* d_img = nullptr;  // [L][kImgLayer]
  float* d_bias = nullptr;         // [L][kBiasLayer]
  float* d_master = nullptr;       // [n_params]
  float* d_m = nullptr;            // [n_params]
  float* d_v = nullptr;            // [n_params]
  float* d_partial = nullptr;      // [tiles_cap][n_params]
  double* d_loss_part = nullptr;   // [tiles_cap]
  float* d_zsave = nullptr;        // [tiles_cap][L][128][16]
  float* d_grad = nullptr;         // [n_params] (gradient-only calls)
  int tiles_cap = 0;
  double* d_tab_u = nullptr;       // [k][stride][D] proposal table of the sampler's walks
  double* d_tab_lq = nullptr;      // [k][stride]
  int stride = 0;
  int32_t* d_train = nullptr;      // 1 when this batch retrains the flow (written by a kernel)
};

cudaError_t flow_kernel_setup();
cudaError_t launch_flow_logq(const FlowDev* d_flow, const double* d_u, int n, double* d_logq, int32_t* d_err,
                             int n_sm, cudaStream_t s);
// Proposal table of a walk batch; scalars from d_task when it is not null.
cudaError_t launch_flow_table(const FlowDev* d_flow, const WalkTask* d_task, int n_walk, int n_steps,
                              int64_t walker_offset, int64_t iteration, uint64_t key0, uint64_t key1, int stride,
                              double* d_tab_u, double* d_tab_lq, int32_t* d_err, int n_sm, cudaStream_t s);
cudaError_t launch_flow_grad(FlowDev* d_flow, const double* d_u, int n, const int32_t* d_active, int bump_t,
                             float* d_partial, double* d_loss_part, float* d_zsave, int32_t* d_err, cudaStream_t s);
cudaError_t launch_flow_adam(FlowDev* d_flow, unsigned char* d_img, float* d_bias, float* d_master, float* d_m,
                             float* d_v, const float* d_partial, int n, const int32_t* d_active, float* d_grad_out,
                             int n_params, cudaStream_t s);
cudaError_t launch_flow_pack(const FlowDev* d_flow, unsigned char* d_img, float* d_bias, const float* d_master,
                             int n_params, cudaStream_t s);
cudaError_t launch_flow_init(FlowDev* d_flow, float* d_master, float* d_m, float* d_v, int n_params, uint64_t key0,
                             uint64_t key1, cudaStream_t s);
cudaError_t launch_flow_standardise(FlowDev* d_flow, const double* d_u, int n, const int32_t* d_active,
                                    cudaStream_t s);

}  // namespace gwns
