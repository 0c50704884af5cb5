// flow.cuh -- the normalising-flow proposal's device data and the one-point density that the
// walk evaluates on CUDA cores.
//
// The flow (a reading: the paper only motivates flow proposals, Sec. 5) is an L-layer
// RealNVP affine-coupling flow (Dinh, Sohl-Dickstein & Bengio 2017) on the unit cube:
//   z0 = (logit(u) - mu) / sigma;  layer l conditions on the dimensions d with (d + l) even:
//   a = m_l z, h1 = tanh(W1 a + b1), h2 = tanh(W2 h1 + b2), [s_raw | t] = W3 h2 + b3,
//   s = S tanh(s_raw / S) (S = 2), z_d <- z_d exp(s_d) + t_d on the other dimensions;
//   log q(u) = log N(z_L) + sum of s - sum log sigma - sum log(u (1 - u)).
// Matrix products take bf16 operands (weights and the activations a, h1, h2) with FP32
// accumulation; everything else is FP32.
//
// Device storage of one flow (per event):
//   img   [L][kImgLayer] bytes: the bf16 weight images in the tensor-core operand layout
//         (tc.cuh): W1 [128 x 16], W2 [128 x 128], W3 [32 x 128] as B operands of the forward
//         products, then W1T [16 x 128], W2T [128 x 128], W3T [128 x 32] for the backward ones.
//         Output rows of W3 are padded: s_d in row d, t_d in row 16 + d.
//   bias  [L][288] FP32: b1 [128], b2 [128], b3 padded like W3's rows [32].
//   master, adam_m, adam_v [n_params] FP32 in the flat order W1, b1, W2, b2, W3, b3 per layer
//         (W3 and b3 with rows s_0..s_{D-1}, t_0..t_{D-1}).
#pragma once

#include <cstdint>
#include <cuda_bf16.h>

#include "gwns_model.cuh"
#include "tc.cuh"

namespace gwns {

constexpr int kFlowP = 16;          // padded dimensions (D <= 16)
constexpr int kFlowH = 128;         // hidden width
constexpr int kFlowO = 32;          // padded conditioner outputs [s (16) | t (16)]
constexpr int kFlowMaxLayers = 16;
constexpr float kFlowS = 2.0f;      // soft clamp of the log-scale

constexpr uint32_t kImgW1 = 0, kImgW2 = 4096, kImgW3 = 36864, kImgFwd = 45056;
constexpr uint32_t kImgW1T = 45056, kImgW2T = 49152, kImgW3T = 81920, kImgLayer = 90112;
constexpr int kBiasB1 = 0, kBiasB2 = 128, kBiasB3 = 256, kBiasLayer = 288;

// Read-mostly flow state of one event, in device memory.
struct FlowDev {
  int n_layers, n_dim, n_params;
  float p_flow;                       // probability of a flow step in the walk
  float mu[kFlowP], sigma[kFlowP];    // standardisation of logit(u)
  float log_sigma_sum;
  int adam_t;                         // Adam steps taken (the gradient kernel advances it)
  float lr;
  const unsigned char* img;           // [L][kImgLayer]
  const float* bias;                  // [L][kBiasLayer]
};

__host__ __device__ inline int flow_layer_params(int D) {
  return kFlowH * D + kFlowH + kFlowH * kFlowH + kFlowH + 2 * D * kFlowH + 2 * D;
}
// flat offsets inside one layer's parameter block
__host__ __device__ inline int flow_off_b1(int D) { return kFlowH * D; }
__host__ __device__ inline int flow_off_w2(int D) { return kFlowH * D + kFlowH; }
__host__ __device__ inline int flow_off_b2(int D) { return kFlowH * D + kFlowH + kFlowH * kFlowH; }
__host__ __device__ inline int flow_off_w3(int D) { return kFlowH * D + 2 * kFlowH + kFlowH * kFlowH; }
__host__ __device__ inline int flow_off_b3(int D) { return kFlowH * D + 2 * kFlowH + kFlowH * kFlowH + 2 * D * kFlowH; }

__device__ __forceinline__ bool flow_cond(int l, int d) { return ((d + l) & 1) == 0; }

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// tanh of the flow's activations (one definition for every kernel that evaluates the flow).
__device__ __forceinline__ float flow_tanh(float x) { return tanhf(x); }

// z0 and -log(u (1 - u)) of one coordinate (FP32 logarithms; 1 - u formed in FP64).
__device__ __forceinline__ void flow_pre_map(const FlowDev& F, int d, double u, float& z0, float& jac) {
  const float lu = logf((float)u), l1u = logf((float)(1.0 - u));
  z0 = (lu - l1u - F.mu[d]) / F.sigma[d];
  jac = -(lu + l1u);
}

// unpacks 8 bf16 values of a 16-byte image chunk
__device__ __forceinline__ void bf16x8(const uint4& q, float* f) {
  const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    f[2 * i] = __uint_as_float(w[i] << 16);
    f[2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
  }
}

struct FlowScratch {
  float z[kFlowP];
  float a[kFlowP];
  float h1[kFlowH];
  float h2[kFlowH];
  float o[kFlowO];
  float red[4];
};

// log q(u) at one point, evaluated by the whole 128-thread CTA on CUDA cores with the same
// bf16 roundings as the tensor-core path (its accumulation order differs).  u: [D] FP64 in
// shared or global memory.  Every thread returns the value.  Contains __syncthreads.
static __device__ __noinline__ float flow_logq_cta(const FlowDev& F, const double* u, FlowScratch& S) {
  const int tid = threadIdx.x, D = F.n_dim, L = F.n_layers;
  float jac = 0.0f, sdet = 0.0f;
  if (tid < kFlowP) {
    float z0 = 0.0f;
    if (tid < D) flow_pre_map(F, tid, u[tid], z0, jac);
    S.z[tid] = z0;
  }
  __syncthreads();
  for (int l = 0; l < L; ++l) {
    const unsigned char* img = F.img + (size_t)l * kImgLayer;
    const float* bias = F.bias + (size_t)l * kBiasLayer;
    if (tid < kFlowP) S.a[tid] = (tid < D && flow_cond(l, tid)) ? bf16_round(S.z[tid]) : 0.0f;
    __syncthreads();
    {  // hidden layer 1: unit tid
      float acc = bias[kBiasB1 + tid], w[8];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        bf16x8(*(const uint4*)(img + kImgW1 + tc::image_offset(128, tid, 8 * c)), w);
#pragma unroll
        for (int i = 0; i < 8; ++i) acc = fmaf(w[i], S.a[8 * c + i], acc);
      }
      S.h1[tid] = bf16_round(flow_tanh(acc));
    }
    __syncthreads();
    {  // hidden layer 2: unit tid
      float acc = bias[kBiasB2 + tid], w[8];
#pragma unroll 4
      for (int c = 0; c < 16; ++c) {
        bf16x8(*(const uint4*)(img + kImgW2 + tc::image_offset(128, tid, 8 * c)), w);
#pragma unroll
        for (int i = 0; i < 8; ++i) acc = fmaf(w[i], S.h1[8 * c + i], acc);
      }
      S.h2[tid] = bf16_round(flow_tanh(acc));
    }
    __syncthreads();
    {  // outputs: output tid / 4, quarter tid % 4 of its 128 inputs
      const int o = tid >> 2, q = tid & 3;
      float acc = 0.0f, w[8];
#pragma unroll
      for (int c = 4 * q; c < 4 * q + 4; ++c) {
        bf16x8(*(const uint4*)(img + kImgW3 + tc::image_offset(32, o, 8 * c)), w);
#pragma unroll
        for (int i = 0; i < 8; ++i) acc = fmaf(w[i], S.h2[8 * c + i], acc);
      }
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      if (q == 0) S.o[o] = acc + bias[kBiasB3 + o];
    }
    __syncthreads();
    if (tid < D && !flow_cond(l, tid)) {
      const float s = kFlowS * flow_tanh(S.o[tid] / kFlowS);
      S.z[tid] = S.z[tid] * expf(s) + S.o[16 + tid];
      sdet += s;
    }
    __syncthreads();
  }
  float c = 0.0f;
  if (tid < D) c = -0.5f * S.z[tid] * S.z[tid] + sdet + jac;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
  if ((tid & 31) == 0) S.red[tid >> 5] = c;
  __syncthreads();
  const float tot = S.red[0] + S.red[1] + S.red[2] + S.red[3];
  __syncthreads();
  return tot - 0.5f * (float)D * 1.8378770664093453f - F.log_sigma_sum;
}

// Standard normal base point of walk step `step` of walker `wid`, dimension pair block c:
// Box-Muller on Philox block (step, wid, it, 16 + c): words (0, 1) -> x[4c], x[4c+1],
// words (2, 3) -> x[4c+2], x[4c+3].
__device__ __forceinline__ void flow_base_normals(uint64_t step, uint64_t wid, uint64_t it, int c, uint64_t key0,
                                                  uint64_t key1, float* x4) {
  Philox4 B = philox4x64(step, wid, it, 16ull + (uint64_t)c, key0, key1);
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const float u1 = (float)rand_open_unit(B.v[2 * p]);
    const float u2 = (float)rand_open_unit(B.v[2 * p + 1]);
    const float r = sqrtf(-2.0f * logf(u1));
    float sn, cs;
    sincospif(2.0f * u2, &sn, &cs);
    x4[2 * p] = r * cs;
    x4[2 * p + 1] = r * sn;
  }
}

}  // namespace gwns
