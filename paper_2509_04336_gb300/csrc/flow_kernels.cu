// flow_kernels.cu -- tensor-core (tcgen05) kernels of the flow proposal: the batched
// forward map (log q), the inverse map (proposal tables), the maximum-likelihood gradient,
// Adam with the bf16 weight-image update, standardisation and initialisation.
//
// Work layout.  A tile is 128 points; thread t of the 128-thread CTA owns point t of the
// tile (its row of every activation and of every TMEM accumulator).  One coupling layer is
// three products with bf16 operands staged in shared memory and FP32 accumulators in TMEM:
//     G1 [128 x 128] = a  [128 x 16]  * W1^T      (K = 16,  one MMA)
//     G2 [128 x 128] = h1 [128 x 128] * W2^T      (K = 128, eight MMAs)
//     G3 [128 x 32]  = h2 [128 x 128] * W3^T      (K = 128, eight MMAs)
// issued by thread 0 (tcgen05.mma, kind::f16), completed through tcgen05.commit on an
// mbarrier, and read back with tcgen05.ld for the FP32 epilogues (bias, tanh, coupling).
// Weights arrive by one bulk copy (cp.async.bulk) per layer, double-buffered in the apply
// kernel so the next layer's copy overlaps this layer's work.
//
// The gradient kernel recomputes each layer's activations in the backward pass (from the
// layer inputs it saved on the way forward) and forms, per tile,
//     dh2 = g_o W3,   dh1 = g_p2 W2,   g_a = g_p1 W1          (data gradients)
//     dW3 = g_o^T h2, dW2 = g_p2^T h1, dW1 = g_p1^T a          (weight gradients, K = points)
// all on the tensor cores, the weight gradients from transposed operand images written by
// the epilogues.  Bias gradients are column sums (warp butterfly + shared memory).  Per-tile
// partial gradients go to global memory; the Adam kernel sums them in a fixed order.
#include <cuda_bf16.h>

#include "api_internal.h"
#include "flow.cuh"
#include "flow_internal.h"

namespace gwns {
namespace {

constexpr int kFT = 128;

// apply kernel shared memory (bytes): two weight buffers, two bias buffers, a, h
constexpr uint32_t kBiasBytes = kBiasLayer * 4;   // 1152
constexpr uint32_t kApWF0 = 0, kApWF1 = 45056, kApB0 = 90112, kApB1 = 91264, kApXA = 92416, kApHA = 96512;
constexpr uint32_t kApBar = 129280;
constexpr uint32_t kApBytes = kApBar + 64;
// gradient kernel shared memory (bytes)
constexpr uint32_t kGrXA = 0, kGrHA = 4096, kGrHB = 36864, kGrG3 = 69632, kGrWF = 77824, kGrW1T = 122880;
constexpr uint32_t kGrW3T = 126976, kGrCS = 135168, kGrBias = 137216, kGrBar = 138368;
constexpr uint32_t kGrBytes = kGrBar + 64;
static_assert(kGrBytes <= 232448, "gradient kernel shared memory");

constexpr uint32_t kTmemCols = 256;
constexpr float kLn2Pi = 1.8378770664093453f;

// ------------------------------------------------------------------ operand staging helpers
__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  __nv_bfloat162 p = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&p);
}
// 16 values of row r, columns c0 .. c0+15, into a 128-row image
__device__ __forceinline__ void st_row16(unsigned char* img, int r, int c0, const float* v) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint4 q;
    q.x = pack_bf16x2(v[8 * h + 0], v[8 * h + 1]);
    q.y = pack_bf16x2(v[8 * h + 2], v[8 * h + 3]);
    q.z = pack_bf16x2(v[8 * h + 4], v[8 * h + 5]);
    q.w = pack_bf16x2(v[8 * h + 6], v[8 * h + 7]);
    *reinterpret_cast<uint4*>(img + tc::image_offset(128, r, c0 + 8 * h)) = q;
  }
}
__device__ __forceinline__ void ld_row16(const unsigned char* img, int r, int c0, float* v) {
  bf16x8(*reinterpret_cast<const uint4*>(img + tc::image_offset(128, r, c0)), v);
  bf16x8(*reinterpret_cast<const uint4*>(img + tc::image_offset(128, r, c0 + 8)), v + 8);
}

// Sum over the warp's 32 lanes of column `lane` of the lanes' 32-column vectors v (the
// butterfly halves the columns a lane carries at each of the five exchanges).
template <int S>
__device__ __forceinline__ void colsum_step(float* v, int lane) {
  const bool up = (lane & S) != 0;
#pragma unroll
  for (int i = 0; i < S; ++i) {
    const float send = up ? v[i] : v[i + S];
    const float keep = up ? v[i + S] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, S);
  }
}
__device__ __forceinline__ float warp_colsum32(float* v, int lane) {
  colsum_step<16>(v, lane);
  colsum_step<8>(v, lane);
  colsum_step<4>(v, lane);
  colsum_step<2>(v, lane);
  colsum_step<1>(v, lane);
  return v[0];
}

// ------------------------------------------------------------------ MMA sequencing
struct Tc {
  uint32_t tmem, lane_base;
  uint64_t* mbar;   // MMA completion
  uint32_t mphase;  // parity of the next completion
  int* abort;
  int pend;         // thread 0: a committed MMA group not yet observed complete
  uint32_t pend_par;

  // D (+)= A B^T over K = 16 ksteps; A: 128-row image, B: N-row image (both K-major).
  __device__ void gemm(uint32_t dcol, const unsigned char* A, const unsigned char* B, int N, int ksteps) const {
    const uint32_t a0 = tc::smem_addr(A), b0 = tc::smem_addr(B);
    const uint32_t albo = tc::image_lbo(128), blbo = tc::image_lbo(N);
    const uint32_t id = tc::idesc_bf16(128, N);
    for (int k = 0; k < ksteps; ++k)
      tc::mma_bf16(tmem + dcol, tc::sdesc(a0 + 2u * k * albo, albo, 128), tc::sdesc(b0 + 2u * k * blbo, blbo, 128),
                   id, k > 0 ? 1u : 0u);
  }
  // D (+)= A^T B over K = 16 ksteps of the tile's points: A and B are 128-row images read
  // MN-major (their columns are D's rows and columns).
  __device__ void gemm_mn(uint32_t dcol, const unsigned char* A, const unsigned char* B, int N, int ksteps) const {
    const uint32_t a0 = tc::smem_addr(A), b0 = tc::smem_addr(B);
    const uint32_t lbo = 128, sbo = tc::image_lbo(128);
    const uint32_t id = tc::idesc_bf16_mn(128, N, true, true);
    for (int k = 0; k < ksteps; ++k)
      tc::mma_bf16(tmem + dcol, tc::sdesc(a0 + 256u * k, lbo, sbo), tc::sdesc(b0 + 256u * k, lbo, sbo), id,
                   k > 0 ? 1u : 0u);
  }
  __device__ void commit() {
    tc::mma_commit(mbar);
    pend = 1;
    pend_par = mphase;
  }
  // all threads: operands written -> visible to the tensor core, then barrier
  __device__ static void publish() {
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
  }
  // all threads: wait for the committed group; false (for every thread) on timeout
  __device__ bool wait() {
    const bool ok = tc::mbar_wait(mbar, mphase);
    mphase ^= 1u;
    if (!ok) *abort = 1;
    tc::fence_after_sync();
    __syncthreads();
    if (threadIdx.x == 0 && ok) pend = 0;
    return *abort == 0;
  }
  __device__ void ld16(uint32_t col, float* v) const { tc::tmem_ld16(tmem + lane_base + col, v); }
};

// ------------------------------------------------------------------ forward / inverse
struct ApplyArgs {
  const FlowDev* flow;
  int inverse;
  // forward: n_rows points u [n][D] -> logq [n]
  int n_rows;
  const double* u_in;
  double* logq_out;
  // inverse: the proposal table of a walk batch, rows (walker w, step t) for w < n_walk and
  // t < *n_steps; base normals from Philox (t, walker_offset + w, iteration, 16 + c).
  // Scalars come from `task` when it is set (graph replays), else from the fields below.
  const WalkTask* task;
  int n_walk, n_steps;
  int64_t walker_offset, iteration;
  uint64_t key0, key1;
  int stride;             // table steps per walker
  double* tab_u;          // [n_walk][stride][D]
  double* tab_lq;         // [n_walk][stride]
  int32_t* err;
};

__global__ void __launch_bounds__(kFT, 1) flow_apply_kernel(ApplyArgs A) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const FlowDev& F = *A.flow;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int D = F.n_dim, L = F.n_layers;
  int n_walk = A.n_walk, n_steps = A.n_steps;
  int64_t wofs = A.walker_offset, iter = A.iteration;
  uint64_t k0 = A.key0, k1 = A.key1;
  if (A.inverse && A.task) {
    if (A.task->done) return;
    n_walk = A.task->n;
    n_steps = A.task->n_steps;
    wofs = A.task->walker_offset;
    iter = A.task->iteration;
    k0 = A.task->key0;
    k1 = A.task->key1;
  }
  const int64_t n_rows = A.inverse ? (int64_t)n_walk * (int64_t)min(n_steps, A.stride) : (int64_t)A.n_rows;
  const int64_t n_tiles = (n_rows + kFT - 1) / kFT;
  if ((int64_t)blockIdx.x >= n_tiles) return;
  const int my_tiles = (int)((n_tiles - 1 - blockIdx.x) / gridDim.x + 1);
  const int steps_eff = A.inverse ? min(n_steps, A.stride) : 1;

  unsigned char* WF[2] = {sm + kApWF0, sm + kApWF1};
  unsigned char* XA = sm + kApXA;
  unsigned char* HA = sm + kApHA;
  float* BS[2] = {reinterpret_cast<float*>(sm + kApB0), reinterpret_cast<float*>(sm + kApB1)};
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + kApBar);   // [0], [1] weights, [2] MMA
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kApBar + 32);
  int* abort = reinterpret_cast<int*>(sm + kApBar + 36);
  if (warp == 0) {
    tc::tmem_alloc(tslot, kTmemCols);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&bars[0], 1);
    tc::mbar_init(&bars[1], 1);
    tc::mbar_init(&bars[2], 1);
    *abort = 0;
    tc::mbar_init_fence();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  Tc T{*tslot, (uint32_t)(warp * 32) << 16, &bars[2], 0u, abort, 0, 0u};

  const int total = my_tiles * L;
  uint32_t wpar[2] = {0u, 0u};
  int wpend[2] = {0, 0};
  auto layer_of = [&](int s) { const int l = s % L; return A.inverse ? L - 1 - l : l; };
  auto issue = [&](int s) {   // thread 0
    const int b = s & 1;
    tc::mbar_expect_tx(&bars[b], kImgFwd);
    tc::bulk_g2s(WF[b], F.img + (size_t)layer_of(s) * kImgLayer, kImgFwd, &bars[b]);
    wpend[b] = 1;
  };
  if (tid == 0) issue(0);

  bool ok = true;
  int s = 0;
  for (int ti = 0; ti < my_tiles && ok; ++ti) {
    const int64_t row = ((int64_t)blockIdx.x + (int64_t)ti * gridDim.x) * kFT + tid;
    const bool valid = row < n_rows;
    float z[kFlowP];
    float jac = 0.0f, logn = 0.0f, logdet = 0.0f;
    int64_t w_i = 0, t_i = 0;
#pragma unroll
    for (int d = 0; d < kFlowP; ++d) z[d] = 0.0f;
    if (valid) {
      if (!A.inverse) {
#pragma unroll
        for (int d = 0; d < kFlowP; ++d)
          if (d < D) {
            float zd, jd;
            flow_pre_map(F, d, A.u_in[row * D + d], zd, jd);
            z[d] = zd;
            jac += jd;
          }
      } else {
        w_i = row / steps_eff;
        t_i = row - w_i * steps_eff;
#pragma unroll
        for (int c = 0; c < kFlowP / 4; ++c)
          if (4 * c < D) {
            float x4[4];
            flow_base_normals((uint64_t)t_i, (uint64_t)(wofs + w_i), (uint64_t)iter, c, k0, k1, x4);
#pragma unroll
            for (int i = 0; i < 4; ++i)
              if (4 * c + i < D) z[4 * c + i] = x4[i];
          }
#pragma unroll
        for (int d = 0; d < kFlowP; ++d) logn -= 0.5f * z[d] * z[d];
      }
    }
    for (int li = 0; li < L && ok; ++li, ++s) {
      const int l = layer_of(s);
      const int b = s & 1;
      // this step's biases (the buffer of step s - 1 is still being read until the barrier)
      float* bias = BS[b];
      for (int i = tid; i < kBiasLayer; i += kFT) bias[i] = __ldg(F.bias + (size_t)l * kBiasLayer + i);
      if (tid == 0 && s + 1 < total) issue(s + 1);
      {
        float a[kFlowP];
#pragma unroll
        for (int d = 0; d < kFlowP; ++d) a[d] = (d < D && flow_cond(l, d)) ? z[d] : 0.0f;
        st_row16(XA, tid, 0, a);
      }
      Tc::publish();
      if (tid == 0) {
        tc::fence_after_sync();
        if (!tc::mbar_wait(&bars[b], wpar[b])) {
          *abort = 1;
        } else {
          wpar[b] ^= 1u;
          wpend[b] = 0;
          T.gemm(0, XA, WF[b] + kImgW1, 128, 1);
          T.commit();
        }
      }
      __syncthreads();
      if (*abort) { ok = false; break; }
      if (!(ok = T.wait())) break;
      // h1 = tanh(G1 + b1)
#pragma unroll 1
      for (int c0 = 0; c0 < kFlowH; c0 += 16) {
        float v[16];
        T.ld16(c0, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = flow_tanh(v[i] + bias[kBiasB1 + c0 + i]);
        st_row16(HA, tid, c0, v);
      }
      Tc::publish();
      if (tid == 0) {
        tc::fence_after_sync();
        T.gemm(0, HA, WF[b] + kImgW2, 128, 8);
        T.commit();
      }
      if (!(ok = T.wait())) break;
      // h2 = tanh(G2 + b2), written over h1 (G2 has completed)
#pragma unroll 1
      for (int c0 = 0; c0 < kFlowH; c0 += 16) {
        float v[16];
        T.ld16(c0, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = flow_tanh(v[i] + bias[kBiasB2 + c0 + i]);
        st_row16(HA, tid, c0, v);
      }
      Tc::publish();
      if (tid == 0) {
        tc::fence_after_sync();
        T.gemm(128, HA, WF[b] + kImgW3, 32, 8);
        T.commit();
      }
      if (!(ok = T.wait())) break;
      {
        float sr[16], tt[16];
        T.ld16(128, sr);
        T.ld16(144, tt);
#pragma unroll
        for (int d = 0; d < kFlowP; ++d)
          if (d < D && !flow_cond(l, d)) {
            const float sc = kFlowS * flow_tanh((sr[d] + bias[kBiasB3 + d]) / kFlowS);
            const float sh = tt[d] + bias[kBiasB3 + 16 + d];
            z[d] = A.inverse ? (z[d] - sh) * expf(-sc) : z[d] * expf(sc) + sh;
            logdet += sc;
          }
      }
    }
    if (!ok) break;
    if (valid) {
      if (!A.inverse) {
        float lq = logdet + jac - F.log_sigma_sum - 0.5f * (float)D * kLn2Pi;
#pragma unroll
        for (int d = 0; d < kFlowP; ++d) lq -= 0.5f * z[d] * z[d];
        A.logq_out[row] = (double)lq;
      } else {
        float j2 = 0.0f;
        double* uo = A.tab_u + ((size_t)w_i * A.stride + t_i) * D;
#pragma unroll
        for (int d = 0; d < kFlowP; ++d)
          if (d < D) {
            const float wv = F.sigma[d] * z[d] + F.mu[d];
            const float e = expf(-fabsf(wv));
            const float small = e / (1.0f + e);   // min(u, 1 - u)
            uo[d] = wv <= 0.0f ? (double)small : 1.0 - (double)small;
            j2 += fabsf(wv) + 2.0f * log1pf(e);   // -log(u (1 - u))
          }
        A.tab_lq[(size_t)w_i * A.stride + t_i] =
            (double)(logn - 0.5f * (float)D * kLn2Pi + logdet + j2 - F.log_sigma_sum);
      }
    }
  }
  if (!ok && tid == 0) {
    // bounded drain of the copies and MMAs still in flight
    for (int b = 0; b < 2; ++b)
      if (wpend[b]) tc::mbar_wait(&bars[b], wpar[b]);
    if (T.pend) tc::mbar_wait(&bars[2], T.pend_par);
    atomicExch(A.err, 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(T.tmem, kTmemCols);
}

// ------------------------------------------------------------------ gradient
struct GradArgs {
  FlowDev* flow;
  const double* u;         // [n][D]
  int n;
  const int32_t* active;   // optional: skip unless *active != 0
  int bump_t;              // advance Adam's step counter (training) or not (gradient only)
  float* partial;          // [n_tiles][n_params]
  double* loss_part;       // [n_tiles]
  float* zsave;            // [n_tiles][L][128][16]
  int32_t* err;
};

__global__ void __launch_bounds__(kFT, 1) flow_grad_kernel(GradArgs G) {
  extern __shared__ __align__(1024) unsigned char sm[];
  if (G.active && *G.active == 0) return;
  FlowDev& F = *G.flow;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int D = F.n_dim, L = F.n_layers, NP = F.n_params, LP = flow_layer_params(D);
  const int tile = blockIdx.x;
  const int row = tile * kGradRows + tid;
  const bool valid = tid < kGradRows && row < G.n;
  if (G.bump_t && tile == 0 && tid == 0) F.adam_t += 1;

  unsigned char *XA = sm + kGrXA, *HA = sm + kGrHA, *HB = sm + kGrHB, *G3 = sm + kGrG3;
  unsigned char *WF = sm + kGrWF, *W1T = sm + kGrW1T, *W3T = sm + kGrW3T;
  float* CS = reinterpret_cast<float*>(sm + kGrCS);             // [4 warps][128]
  float* bias = reinterpret_cast<float*>(sm + kGrBias);         // this layer's b1 | b2 | b3
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + kGrBar);   // [0] weights, [1] W2T, [2] MMA
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kGrBar + 32);
  int* abort = reinterpret_cast<int*>(sm + kGrBar + 36);
  float* part = G.partial + (size_t)tile * NP;
  float* zs = G.zsave + (size_t)tile * L * kFT * kFlowP;

  if (warp == 0) {
    tc::tmem_alloc(tslot, kTmemCols);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    for (int i = 0; i < 3; ++i) tc::mbar_init(&bars[i], 1);
    *abort = 0;
    tc::mbar_init_fence();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  Tc T{*tslot, (uint32_t)(warp * 32) << 16, &bars[2], 0u, abort, 0, 0u};
  uint32_t wpar = 0u, w2par = 0u;
  int wpend = 0, w2pend = 0;
  bool ok = true;

  // column sums of a [128 rows x 32 cols] block held one row per thread -> out[32]
  auto colsum32 = [&](float* v, float* out) {
    const float c = warp_colsum32(v, lane);
    CS[warp * 128 + lane] = c;
    __syncthreads();
    if (tid < 32) out[tid] = CS[tid] + CS[128 + tid] + CS[256 + tid] + CS[384 + tid];
    __syncthreads();
  };
  // this layer's biases into shared memory (the previous readers passed a barrier)
  auto stage_bias = [&](int l) {
    for (int i = tid; i < kBiasLayer; i += kFT) bias[i] = __ldg(F.bias + (size_t)l * kBiasLayer + i);
  };

  // ---- forward pass: layer inputs saved, log q for the loss
  float z[kFlowP], jac = 0.0f, logdet = 0.0f;
#pragma unroll
  for (int d = 0; d < kFlowP; ++d) z[d] = 0.0f;
  if (valid) {
#pragma unroll
    for (int d = 0; d < kFlowP; ++d)
      if (d < D) {
        float zd, jd;
        flow_pre_map(F, d, G.u[(size_t)row * D + d], zd, jd);
        z[d] = zd;
        jac += jd;
      }
  }
  for (int l = 0; l < L && ok; ++l) {
    float4* zsl = reinterpret_cast<float4*>(zs + ((size_t)l * kFT + tid) * kFlowP);
#pragma unroll
    for (int q = 0; q < 4; ++q) zsl[q] = make_float4(z[4 * q], z[4 * q + 1], z[4 * q + 2], z[4 * q + 3]);
    if (tid == 0) {
      tc::mbar_expect_tx(&bars[0], kImgFwd);
      tc::bulk_g2s(WF, F.img + (size_t)l * kImgLayer, kImgFwd, &bars[0]);
      wpend = 1;
    }
    stage_bias(l);
    {
      float a[kFlowP];
#pragma unroll
      for (int d = 0; d < kFlowP; ++d) a[d] = (d < D && flow_cond(l, d)) ? z[d] : 0.0f;
      st_row16(XA, tid, 0, a);
    }
    Tc::publish();
    if (tid == 0) {
      tc::fence_after_sync();
      if (!tc::mbar_wait(&bars[0], wpar)) {
        *abort = 1;
      } else {
        wpar ^= 1u;
        wpend = 0;
        T.gemm(0, XA, WF + kImgW1, 128, 1);
        T.commit();
      }
    }
    __syncthreads();
    if (*abort) { ok = false; break; }
    if (!(ok = T.wait())) break;
#pragma unroll 1
    for (int c0 = 0; c0 < kFlowH; c0 += 16) {
      float v[16];
      T.ld16(c0, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = flow_tanh(v[i] + bias[kBiasB1 + c0 + i]);
      st_row16(HA, tid, c0, v);
    }
    Tc::publish();
    if (tid == 0) {
      tc::fence_after_sync();
      T.gemm(0, HA, WF + kImgW2, 128, 8);
      T.commit();
    }
    if (!(ok = T.wait())) break;
#pragma unroll 1
    for (int c0 = 0; c0 < kFlowH; c0 += 16) {
      float v[16];
      T.ld16(c0, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = flow_tanh(v[i] + bias[kBiasB2 + c0 + i]);
      st_row16(HB, tid, c0, v);
    }
    Tc::publish();
    if (tid == 0) {
      tc::fence_after_sync();
      T.gemm(128, HB, WF + kImgW3, 32, 8);
      T.commit();
    }
    if (!(ok = T.wait())) break;
    {
      float sr[16], tt[16];
      T.ld16(128, sr);
      T.ld16(144, tt);
#pragma unroll
      for (int d = 0; d < kFlowP; ++d)
        if (d < D && !flow_cond(l, d)) {
          const float sc = kFlowS * flow_tanh((sr[d] + bias[kBiasB3 + d]) / kFlowS);
          z[d] = z[d] * expf(sc) + tt[d] + bias[kBiasB3 + 16 + d];
          logdet += sc;
        }
    }
    tc::fence_before_sync();
    __syncthreads();   // WF and the biases are reloaded by the next layer
  }
  // loss part: sum over the tile's points of -log q
  float g[kFlowP];
  if (ok) {
    float nll = 0.0f;
    if (valid) {
      nll = -(logdet + jac - F.log_sigma_sum - 0.5f * (float)D * kLn2Pi);
#pragma unroll
      for (int d = 0; d < kFlowP; ++d) nll += 0.5f * z[d] * z[d];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) nll += __shfl_xor_sync(0xffffffffu, nll, off);
    if (lane == 0) CS[warp] = nll;
    __syncthreads();
    if (tid == 0) G.loss_part[tile] = (double)CS[0] + (double)CS[1] + (double)CS[2] + (double)CS[3];
    __syncthreads();
  }
#pragma unroll
  for (int d = 0; d < kFlowP; ++d) g[d] = valid ? z[d] : 0.0f;

  // ---- backward pass
  for (int l = L - 1; l >= 0 && ok; --l) {
    const unsigned char* img = F.img + (size_t)l * kImgLayer;
    float* pl = part + (size_t)l * LP;
    float zin[kFlowP];
    {
      const float4* zsl = reinterpret_cast<const float4*>(zs + ((size_t)l * kFT + tid) * kFlowP);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 v = zsl[q];
        zin[4 * q] = v.x; zin[4 * q + 1] = v.y; zin[4 * q + 2] = v.z; zin[4 * q + 3] = v.w;
      }
    }
    if (tid == 0) {
      tc::mbar_expect_tx(&bars[0], kImgFwd + 4096 + 8192);
      tc::bulk_g2s(WF, img, kImgFwd, &bars[0]);
      tc::bulk_g2s(W1T, img + kImgW1T, 4096, &bars[0]);
      tc::bulk_g2s(W3T, img + kImgW3T, 8192, &bars[0]);
      wpend = 1;
    }
    stage_bias(l);
    {
      float a[kFlowP];
#pragma unroll
      for (int d = 0; d < kFlowP; ++d) a[d] = (d < D && flow_cond(l, d)) ? zin[d] : 0.0f;
      st_row16(XA, tid, 0, a);
    }
    Tc::publish();
    if (tid == 0) {
      tc::fence_after_sync();
      if (!tc::mbar_wait(&bars[0], wpar)) {
        *abort = 1;
      } else {
        wpar ^= 1u;
        wpend = 0;
        T.gemm(0, XA, WF + kImgW1, 128, 1);
        T.commit();
      }
    }
    __syncthreads();
    if (*abort) { ok = false; break; }
    if (!(ok = T.wait())) break;
    // h1 -> HA
#pragma unroll 1
    for (int c0 = 0; c0 < kFlowH; c0 += 16) {
      float v[16];
      T.ld16(c0, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = flow_tanh(v[i] + bias[kBiasB1 + c0 + i]);
      st_row16(HA, tid, c0, v);
    }
    Tc::publish();
    if (tid == 0) {
      tc::fence_after_sync();
      T.gemm(0, HA, WF + kImgW2, 128, 8);
      T.commit();
    }
    if (!(ok = T.wait())) break;
    if (tid == 0) {   // W2 has been consumed: bring W2T into its slot
      tc::mbar_expect_tx(&bars[1], 32768);
      tc::bulk_g2s(WF + kImgW2, img + kImgW2T, 32768, &bars[1]);
      w2pend = 1;
    }
    // h2 -> HB
#pragma unroll 1
    for (int c0 = 0; c0 < kFlowH; c0 += 16) {
      float v[16];
      T.ld16(c0, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = flow_tanh(v[i] + bias[kBiasB2 + c0 + i]);
      st_row16(HB, tid, c0, v);
    }
    Tc::publish();
    if (tid == 0) {
      tc::fence_after_sync();
      T.gemm(128, HB, WF + kImgW3, 32, 8);
      T.commit();
    }
    if (!(ok = T.wait())) break;
    // coupling backward: g_o = [d/ds_raw | d/dt] -> G3; db3; direct part of dz_in
    float gdir[kFlowP];
    {
      float sr[16], tt[16], go[32];
      T.ld16(128, sr);
      T.ld16(144, tt);
#pragma unroll
      for (int d = 0; d < kFlowP; ++d) {
        go[d] = 0.0f;
        go[16 + d] = 0.0f;
        gdir[d] = g[d];
        if (d < D && !flow_cond(l, d)) {
          const float th = flow_tanh((sr[d] + bias[kBiasB3 + d]) / kFlowS);
          const float e = expf(kFlowS * th);
          const float gs = valid ? (g[d] * zin[d] * e - 1.0f) : 0.0f;
          go[d] = gs * (1.0f - th * th);
          go[16 + d] = g[d];
          gdir[d] = g[d] * e;
        }
      }
      st_row16(G3, tid, 0, go);
      st_row16(G3, tid, 16, go + 16);
      float cs[32];
      colsum32(go, cs);   // go is consumed
      if (tid < kFlowO) {
        const int o = tid;
        const int op = o < 16 ? (o < D ? o : -1) : (o - 16 < D ? D + o - 16 : -1);
        if (op >= 0) pl[flow_off_b3(D) + op] = cs[o];
      }
    }
    Tc::publish();
    if (tid == 0) {
      tc::fence_after_sync();
      T.gemm(0, G3, W3T, 128, 2);         // dh2 = g_o W3
      T.gemm_mn(128, HB, G3, 32, 8);      // dW3^T = h2^T g_o
      T.commit();
    }
    if (!(ok = T.wait())) break;
    {
      // dW3[o'][j] for hidden unit j = tid
      float v[16];
#pragma unroll 1
      for (int c0 = 0; c0 < kFlowO; c0 += 16) {
        T.ld16(128 + c0, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int o = c0 + i;
          const int op = o < 16 ? (o < D ? o : -1) : (o - 16 < D ? D + o - 16 : -1);
          if (op >= 0) pl[flow_off_w3(D) + op * kFlowH + tid] = v[i];
        }
      }
    }
    // g_p2 = dh2 (1 - h2^2) -> G2 over HB; db2
#pragma unroll 1
    for (int c0 = 0; c0 < kFlowH; c0 += 32) {
      float gp[32], h[16];
      T.ld16(c0, gp);
      T.ld16(c0 + 16, gp + 16);
      ld_row16(HB, tid, c0, h);
#pragma unroll
      for (int i = 0; i < 16; ++i) gp[i] *= 1.0f - h[i] * h[i];
      ld_row16(HB, tid, c0 + 16, h);
#pragma unroll
      for (int i = 0; i < 16; ++i) gp[16 + i] *= 1.0f - h[i] * h[i];
      st_row16(HB, tid, c0, gp);
      st_row16(HB, tid, c0 + 16, gp + 16);
      float cs[32];
      colsum32(gp, cs);
      if (tid < 32) pl[flow_off_b2(D) + c0 + tid] = cs[tid];
    }
    Tc::publish();
    if (tid == 0) {
      tc::fence_after_sync();
      if (!tc::mbar_wait(&bars[1], w2par)) {
        *abort = 1;
      } else {
        w2par ^= 1u;
        w2pend = 0;
        T.gemm(0, HB, WF + kImgW2, 128, 8);     // dh1 = g_p2 W2 (W2T image in the W2 slot)
        T.gemm_mn(128, HB, HA, 128, 8);         // dW2 = g_p2^T h1
        T.commit();
      }
    }
    __syncthreads();
    if (*abort) { ok = false; break; }
    if (!(ok = T.wait())) break;
    {
      // dW2[j][k] for output unit j = tid
      float v[16];
#pragma unroll 1
      for (int c0 = 0; c0 < kFlowH; c0 += 16) {
        T.ld16(128 + c0, v);
        float* dst = pl + flow_off_w2(D) + tid * kFlowH + c0;   // layer blocks are not 16-byte aligned
#pragma unroll
        for (int i = 0; i < 16; ++i) dst[i] = v[i];
      }
    }
    // g_p1 = dh1 (1 - h1^2) -> G1 over HA; db1
#pragma unroll 1
    for (int c0 = 0; c0 < kFlowH; c0 += 32) {
      float gp[32], h[16];
      T.ld16(c0, gp);
      T.ld16(c0 + 16, gp + 16);
      ld_row16(HA, tid, c0, h);
#pragma unroll
      for (int i = 0; i < 16; ++i) gp[i] *= 1.0f - h[i] * h[i];
      ld_row16(HA, tid, c0 + 16, h);
#pragma unroll
      for (int i = 0; i < 16; ++i) gp[16 + i] *= 1.0f - h[i] * h[i];
      st_row16(HA, tid, c0, gp);
      st_row16(HA, tid, c0 + 16, gp + 16);
      float cs[32];
      colsum32(gp, cs);
      if (tid < 32) pl[flow_off_b1(D) + c0 + tid] = cs[tid];
    }
    Tc::publish();
    if (tid == 0) {
      tc::fence_after_sync();
      T.gemm(128, HA, W1T, 16, 8);       // g_a = g_p1 W1
      T.gemm_mn(192, HA, XA, 16, 8);     // dW1 = g_p1^T a
      T.commit();
    }
    if (!(ok = T.wait())) break;
    {
      float v[16];
      T.ld16(192, v);   // dW1[j][d] for hidden unit j = tid
#pragma unroll
      for (int d = 0; d < kFlowP; ++d)
        if (d < D) pl[tid * D + d] = v[d];
      T.ld16(128, v);   // g_a of this point
#pragma unroll
      for (int d = 0; d < kFlowP; ++d) g[d] = gdir[d] + ((d < D && flow_cond(l, d)) ? v[d] : 0.0f);
    }
    tc::fence_before_sync();
    __syncthreads();   // slots and biases are reloaded by the next layer
  }
  if (!ok && tid == 0) {
    if (wpend) tc::mbar_wait(&bars[0], wpar);
    if (w2pend) tc::mbar_wait(&bars[1], w2par);
    if (T.pend) tc::mbar_wait(&bars[2], T.pend_par);
    atomicExch(G.err, 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(T.tmem, kTmemCols);
}

// ------------------------------------------------------------------ weights
// Writes parameter i (flat order) into the bf16 images and the bias table.
__device__ void pack_param(const FlowDev& F, unsigned char* img_all, float* bias_all, int i, float w) {
  const int D = F.n_dim, LP = flow_layer_params(D);
  const int l = i / LP, r = i - l * LP;
  unsigned char* img = img_all + (size_t)l * kImgLayer;
  float* bias = bias_all + (size_t)l * kBiasLayer;
  const __nv_bfloat16 wb = __float2bfloat16_rn(w);
  if (r < flow_off_b1(D)) {
    const int j = r / D, d = r - j * D;
    *reinterpret_cast<__nv_bfloat16*>(img + kImgW1 + tc::image_offset(128, j, d)) = wb;
    *reinterpret_cast<__nv_bfloat16*>(img + kImgW1T + tc::image_offset(16, d, j)) = wb;
  } else if (r < flow_off_w2(D)) {
    bias[kBiasB1 + (r - flow_off_b1(D))] = w;
  } else if (r < flow_off_b2(D)) {
    const int q = r - flow_off_w2(D), j = q / kFlowH, k = q - j * kFlowH;
    *reinterpret_cast<__nv_bfloat16*>(img + kImgW2 + tc::image_offset(128, j, k)) = wb;
    *reinterpret_cast<__nv_bfloat16*>(img + kImgW2T + tc::image_offset(128, k, j)) = wb;
  } else if (r < flow_off_w3(D)) {
    bias[kBiasB2 + (r - flow_off_b2(D))] = w;
  } else if (r < flow_off_b3(D)) {
    const int q = r - flow_off_w3(D), op = q / kFlowH, k = q - op * kFlowH;
    const int o = op < D ? op : 16 + (op - D);
    *reinterpret_cast<__nv_bfloat16*>(img + kImgW3 + tc::image_offset(32, o, k)) = wb;
    *reinterpret_cast<__nv_bfloat16*>(img + kImgW3T + tc::image_offset(128, k, o)) = wb;
  } else {
    const int op = r - flow_off_b3(D);
    bias[kBiasB3 + (op < D ? op : 16 + (op - D))] = w;
  }
}

struct AdamArgs {
  FlowDev* flow;
  unsigned char* img;
  float* bias;
  float* master;
  float* m;
  float* v;
  const float* partial;    // [n_tiles][n_params]
  int n_tiles;
  float inv_n;
  const int32_t* active;
  float* grad_out;         // gradient-only mode: write the mean gradient here, no update
};

__global__ void flow_adam_kernel(AdamArgs A) {
  if (A.active && *A.active == 0) return;
  const FlowDev& F = *A.flow;
  const int NP = F.n_params;
  const float t = (float)F.adam_t;
  const float c1 = 1.0f / (1.0f - powf(0.9f, t)), c2 = 1.0f / (1.0f - powf(0.999f, t));
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NP; i += gridDim.x * blockDim.x) {
    float gs = 0.0f;
    for (int k = 0; k < A.n_tiles; ++k) gs += A.partial[(size_t)k * NP + i];
    const float g = gs * A.inv_n;
    if (A.grad_out) {
      A.grad_out[i] = g;
      continue;
    }
    if (!isfinite(g)) continue;   // a non-finite component leaves its parameter and moments
    const float m = 0.9f * A.m[i] + 0.1f * g;
    const float v = 0.999f * A.v[i] + 0.001f * g * g;
    A.m[i] = m;
    A.v[i] = v;
    const float w = A.master[i] - F.lr * (m * c1) / (sqrtf(v * c2) + 1e-8f);
    A.master[i] = w;
    pack_param(F, A.img, A.bias, i, w);
  }
}

__global__ void flow_pack_kernel(const FlowDev* F, unsigned char* img, float* bias, const float* master) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < F->n_params; i += gridDim.x * blockDim.x)
    pack_param(*F, img, bias, i, master[i]);
}

// Initial weights: W1, W2 uniform on (-1, 1) / sqrt(fan_in) from Philox block
// (l, mat, e / 4, 5), word e % 4; W3 and biases zero; Adam state zero.
__global__ void flow_init_kernel(FlowDev* F, float* master, float* m, float* v, uint64_t key0, uint64_t key1) {
  const int D = F->n_dim, LP = flow_layer_params(D);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < F->n_params; i += gridDim.x * blockDim.x) {
    const int l = i / LP, r = i - l * LP;
    float w = 0.0f;
    int mat = -1, e = 0, fan = 1;
    if (r < flow_off_b1(D)) { mat = 0; e = r; fan = D; }
    else if (r >= flow_off_w2(D) && r < flow_off_b2(D)) { mat = 1; e = r - flow_off_w2(D); fan = kFlowH; }
    if (mat >= 0) {
      Philox4 B = philox4x64((uint64_t)l, (uint64_t)mat, (uint64_t)(e >> 2), 5ull, key0, key1);
      w = (float)((2.0 * rand_open_unit(B.v[e & 3]) - 1.0) / sqrt((double)fan));
    }
    master[i] = w;
    m[i] = 0.0f;
    v[i] = 0.0f;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) F->adam_t = 0;
}

// mu, sigma of logit(u) over the training points (FP64 sums of the FP32 logits).
__global__ void flow_standardise_kernel(FlowDev* F, const double* u, int n, const int32_t* active) {
  if (active && *active == 0) return;
  __shared__ double red[256];
  __shared__ float s_mu;
  const int D = F->n_dim;
  float lss = 0.0f;
  for (int d = 0; d < D; ++d) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double x = u[(size_t)i * D + d];
      acc += (double)(logf((float)x) - logf((float)(1.0 - x)));
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
      __syncthreads();
    }
    const double mean = red[0] / n;
    __syncthreads();
    acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double x = u[(size_t)i * D + d];
      const double y = (double)(logf((float)x) - logf((float)(1.0 - x))) - mean;
      acc += y * y;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      double sd = sqrt(red[0] / n);
      if (!(sd > 0.0)) sd = 1.0;
      F->mu[d] = (float)mean;
      F->sigma[d] = (float)sd;
      s_mu = logf((float)sd);
    }
    __syncthreads();
    lss += s_mu;
    __syncthreads();
  }
  if (threadIdx.x == 0) F->log_sigma_sum = lss;
}

}  // namespace

// ------------------------------------------------------------------ launchers
cudaError_t flow_kernel_setup() {
  cudaError_t e = cudaFuncSetAttribute(flow_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kApBytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(flow_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGrBytes);
}

cudaError_t launch_flow_logq(const FlowDev* d_flow, const double* d_u, int n, double* d_logq, int32_t* d_err,
                             int n_sm, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  ApplyArgs A{};
  A.flow = d_flow;
  A.inverse = 0;
  A.n_rows = n;
  A.u_in = d_u;
  A.logq_out = d_logq;
  A.err = d_err;
  const int tiles = (n + kFT - 1) / kFT;
  flow_apply_kernel<<<tiles < n_sm ? tiles : n_sm, kFT, kApBytes, s>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_flow_table(const FlowDev* d_flow, const WalkTask* d_task, int n_walk, int n_steps,
                              int64_t walker_offset, int64_t iteration, uint64_t key0, uint64_t key1, int stride,
                              double* d_tab_u, double* d_tab_lq, int32_t* d_err, int n_sm, cudaStream_t s) {
  ApplyArgs A{};
  A.flow = d_flow;
  A.inverse = 1;
  A.task = d_task;
  A.n_walk = n_walk;
  A.n_steps = n_steps;
  A.walker_offset = walker_offset;
  A.iteration = iteration;
  A.key0 = key0;
  A.key1 = key1;
  A.stride = stride;
  A.tab_u = d_tab_u;
  A.tab_lq = d_tab_lq;
  A.err = d_err;
  flow_apply_kernel<<<n_sm, kFT, kApBytes, s>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_flow_grad(FlowDev* d_flow, const double* d_u, int n, const int32_t* d_active, int bump_t,
                             float* d_partial, double* d_loss_part, float* d_zsave, int32_t* d_err, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  GradArgs G{d_flow, d_u, n, d_active, bump_t, d_partial, d_loss_part, d_zsave, d_err};
  flow_grad_kernel<<<(n + kGradRows - 1) / kGradRows, kFT, kGrBytes, s>>>(G);
  return cudaGetLastError();
}

cudaError_t launch_flow_adam(FlowDev* d_flow, unsigned char* d_img, float* d_bias, float* d_master, float* d_m,
                             float* d_v, const float* d_partial, int n, const int32_t* d_active, float* d_grad_out,
                             int n_params, cudaStream_t s) {
  AdamArgs A{d_flow, d_img, d_bias, d_master, d_m, d_v, d_partial, (n + kGradRows - 1) / kGradRows, 1.0f / (float)n,
             d_active, d_grad_out};
  const int blocks = (n_params + 255) / 256;
  flow_adam_kernel<<<blocks < 1024 ? blocks : 1024, 256, 0, s>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_flow_pack(const FlowDev* d_flow, unsigned char* d_img, float* d_bias, const float* d_master,
                             int n_params, cudaStream_t s) {
  const int blocks = (n_params + 255) / 256;
  flow_pack_kernel<<<blocks < 1024 ? blocks : 1024, 256, 0, s>>>(d_flow, d_img, d_bias, d_master);
  return cudaGetLastError();
}

cudaError_t launch_flow_init(FlowDev* d_flow, float* d_master, float* d_m, float* d_v, int n_params, uint64_t key0,
                             uint64_t key1, cudaStream_t s) {
  const int blocks = (n_params + 255) / 256;
  flow_init_kernel<<<blocks < 1024 ? blocks : 1024, 256, 0, s>>>(d_flow, d_master, d_m, d_v, key0, key1);
  return cudaGetLastError();
}

cudaError_t launch_flow_standardise(FlowDev* d_flow, const double* d_u, int n, const int32_t* d_active,
                                    cudaStream_t s) {
  flow_standardise_kernel<<<1, 256, 0, s>>>(d_flow, d_u, n, d_active);
  return cudaGetLastError();
}

}  // namespace gwns
