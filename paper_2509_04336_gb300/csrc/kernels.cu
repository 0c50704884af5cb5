// kernels.cu -- likelihood, waveform and acceptance-walk kernels (sm_103a).
//
// Thread layout: one CTA of kThreads threads owns one walker (likelihood evaluation).
// Thread 0 computes the walker's per-theta constants (prior transform, TaylorF2
// coefficients, antenna patterns) into shared memory; all threads then stream the
// active frequency bins (stride kThreads) and accumulate S_det; a warp-shuffle tree
// and a cross-warp pass in shared memory reduce the sums.
#include <cstdio>

#include "gwns_internal.h"

namespace gwns {

namespace {

constexpr int kWarps = kThreads / 32;

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Reduce NDET complex sums over the CTA; thread 0 receives FP64 totals.
template <int NDET>
__device__ inline void reduce_f64(AccF64& acc, double (*red)[2 * kMaxDet], double* s_re, double* s_im) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int det = 0; det < NDET; ++det) {
    double r = acc.re[det], i = acc.im[det];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      r += __shfl_down_sync(0xffffffffu, r, off);
      i += __shfl_down_sync(0xffffffffu, i, off);
    }
    if (lane == 0) { red[warp][2 * det] = r; red[warp][2 * det + 1] = i; }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int det = 0; det < NDET; ++det) {
      double r = 0.0, i = 0.0;
      for (int w = 0; w < kWarps; ++w) { r += red[w][2 * det]; i += red[w][2 * det + 1]; }
      s_re[det] = r; s_im[det] = i;
    }
  }
}

// Compensated FP32 tree: every level adds (sum, error) pairs with an error-free two-sum.
template <int NDET>
__device__ inline void reduce_mixed(AccF32& acc, double (*red)[2 * kMaxDet], double* s_re, double* s_im) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int det = 0; det < NDET; ++det) {
#pragma unroll
    for (int part = 0; part < 2; ++part) {
      float s = part ? acc.im[det] : acc.re[det];
      float c = -(part ? acc.cim[det] : acc.cre[det]);   // Kahan keeps the negated error
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        float so = __shfl_down_sync(0xffffffffu, s, off);
        float co = __shfl_down_sync(0xffffffffu, c, off);
        float t, e;
        two_sum(s, so, t, e);
        s = t;
        c = c + co + e;
      }
      if (lane == 0) red[warp][2 * det + part] = (double)s + (double)c;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int det = 0; det < NDET; ++det) {
      double r = 0.0, i = 0.0;
      for (int w = 0; w < kWarps; ++w) { r += red[w][2 * det]; i += red[w][2 * det + 1]; }
      s_re[det] = r; s_im[det] = i;
    }
  }
}

// S_det sums of one walker over its active bins, reduced to thread 0.
template <int PREC, int NDET>
__device__ inline void walker_sums(const EventDev& ev, const WalkerParams& P, double (*red)[2 * kMaxDet],
                                   double* s_re, double* s_im) {
  if (PREC == 0) {
    AccF64 acc; acc.zero();
    for (int k = threadIdx.x; k < P.k_end; k += kThreads) bin_accumulate_f64<NDET>(ev, P, k, acc);
    reduce_f64<NDET>(acc, red, s_re, s_im);
  } else {
    AccF32 acc; acc.zero();
    for (int k = threadIdx.x; k < P.k_end; k += kThreads) bin_accumulate_mixed<NDET>(ev, P, k, acc);
    reduce_mixed<NDET>(acc, red, s_re, s_im);
  }
}

__device__ inline bool theta_ok(const double* th) {
  for (int i = 0; i < kParams; ++i) if (!isfinite(th[i])) return false;
  return th[0] > 0.0 && th[1] > 0.0 && th[4] > 0.0;
}

// ---------------------------------------------------------------- likelihood batch
template <int PREC, int NDET>
__global__ void __launch_bounds__(kThreads) likelihood_kernel(const EventDev* __restrict__ evp,
                                                               const double* __restrict__ theta, int n,
                                                               double* __restrict__ lnl, int32_t* status) {
  __shared__ WalkerParams P;
  __shared__ double red[kWarps][2 * kMaxDet];
  __shared__ double s_re[kMaxDet], s_im[kMaxDet];
  __shared__ int ok;
  const EventDev& ev = *evp;
  const int w = blockIdx.x;
  if (threadIdx.x == 0) {
    double th[kParams];
    for (int i = 0; i < kParams; ++i) th[i] = theta[(size_t)w * kParams + i];
    ok = theta_ok(th);
    if (ok) {
      double sd, cd;
      sincos(th[10], &sd, &cd);
      taylorf2_setup(ev, th, cos(th[5]), sd, cd, P);
    } else {
      P.k_end = 0;
    }
  }
  __syncthreads();
  walker_sums<PREC, NDET>(ev, P, red, s_re, s_im);
  if (threadIdx.x == 0) {
    if (ok) {
      lnl[w] = assemble_lnl(ev, P, s_re, s_im);
    } else {
      lnl[w] = __longlong_as_double(0x7ff8000000000000ll);
      atomicOr(status, 1);
    }
  }
}

// ln L of unit-cube points u [n][D] (prior transform, then the likelihood).  Used for the
// initial live points; non-finite results are stored as -inf so that they die first.
template <int PREC, int NDET>
__global__ void __launch_bounds__(kThreads) unit_likelihood_kernel(const EventDev* __restrict__ evp,
                                                                    const double* __restrict__ u, int n,
                                                                    double* __restrict__ lnl) {
  __shared__ WalkerParams P;
  __shared__ double red[kWarps][2 * kMaxDet];
  __shared__ double s_re[kMaxDet], s_im[kMaxDet];
  const EventDev& ev = *evp;
  const int w = blockIdx.x;
  if (threadIdx.x == 0) {
    double th[kParams], ci, sd, cd;
    unit_to_theta(ev, u + (size_t)w * ev.n_dim, th, &ci, &sd, &cd);
    taylorf2_setup(ev, th, ci, sd, cd, P);
  }
  __syncthreads();
  walker_sums<PREC, NDET>(ev, P, red, s_re, s_im);
  if (threadIdx.x == 0) {
    double v = assemble_lnl(ev, P, s_re, s_im);
    lnl[w] = isfinite(v) ? v : -INFINITY;
  }
}

// Physical theta [n][11] of unit-cube points u [n][D].
__global__ void unit_to_theta_kernel(const EventDev* __restrict__ evp, const double* __restrict__ u, int64_t n,
                                     double* __restrict__ theta) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const EventDev& ev = *evp;
  double th[kParams], ci, sd, cd;
  unit_to_theta(ev, u + i * ev.n_dim, th, &ci, &sd, &cd);
  for (int k = 0; k < kParams; ++k) theta[i * kParams + k] = th[k];
}

// ---------------------------------------------------------------- waveform (FP64)
template <int NDET>
__global__ void __launch_bounds__(256) waveform_kernel(const EventDev* __restrict__ evp,
                                                       const double* __restrict__ theta, int n_bins,
                                                       double* __restrict__ h_re, double* __restrict__ h_im) {
  __shared__ WalkerParams P;
  const EventDev& ev = *evp;
  const int w = blockIdx.y;
  if (threadIdx.x == 0) {
    double th[kParams];
    for (int i = 0; i < kParams; ++i) th[i] = theta[(size_t)w * kParams + i];
    double sd, cd;
    sincos(th[10], &sd, &cd);
    taylorf2_setup(ev, th, cos(th[5]), sd, cd, P);
  }
  __syncthreads();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_bins) return;
#pragma unroll
  for (int det = 0; det < NDET; ++det) {
    double re = 0.0, im = 0.0;
    if (k < P.k_end) {
      const double* g = ev.basis64 + (size_t)k * kBasis;
      double phi = P.phase0;
      for (int j = 0; j < kBasis; ++j) phi = fma(P.C[j], g[j], phi);
      double f = ev.f_min + ev.df * (double)k;
      double ph = fma(P.tau[det], f, phi);
      double r = ph - rint(ph);
      double s, c;
      sincospi(2.0 * r, &s, &c);
      double a = pow(f, -7.0 / 6.0);
      // K P exp(-2 pi i r)
      re = a * (P.kp_re[det] * c + P.kp_im[det] * s);
      im = a * (P.kp_im[det] * c - P.kp_re[det] * s);
    }
    size_t o = ((size_t)w * NDET + det) * n_bins + k;
    h_re[o] = re;
    h_im[o] = im;
  }
}

// ---------------------------------------------------------------- acceptance walk
// One CTA per walker.  Thread 0 draws the DE move (Philox blocks (t, id, it, 0|1)),
// applies periodic wrapping and the bounds test, transforms to theta and computes the
// per-walker constants; the CTA evaluates ln L; thread 0 applies the strict L > L* test.
template <int PREC, int NDET>
__global__ void __launch_bounds__(kThreads) walk_kernel(const EventDev* __restrict__ evs, WalkTask* tasks,
                                                         const int32_t* __restrict__ blk_task,
                                                         const int32_t* __restrict__ blk_local) {
  __shared__ WalkerParams P;
  __shared__ double red[kWarps][2 * kMaxDet];
  __shared__ double s_re[kMaxDet], s_im[kMaxDet];
  __shared__ double u[kMaxDim], prop[kMaxDim];
  __shared__ int inside;
  const WalkTask& T = tasks[blk_task[blockIdx.x]];
  const int j = blk_local[blockIdx.x];
  const EventDev& ev = evs[T.event];
  if (T.done) return;
  const int D = ev.n_dim;
  const int n_steps = T.n_steps;
  const double lnl_star = T.lnl_star;
  const uint64_t it = (uint64_t)T.iteration;
  const uint64_t wid = (uint64_t)(T.walker_offset + j);
  const uint64_t n_s = (uint64_t)T.n_s;
  if (threadIdx.x < D) u[threadIdx.x] = T.u0[(size_t)j * D + threadIdx.x];
  double lnl = T.lnl0[j];
  int n_acc = 0, n_like = 0;
  int64_t n_bins = 0;
  const double de_scale = 2.38 / sqrt(2.0 * (double)D);
  __syncthreads();
  for (int t = 0; t < n_steps; ++t) {
    if (threadIdx.x == 0) {
      Philox4 A = philox4x64((uint64_t)t, wid, it, 0ull, T.key0, T.key1);
      uint64_t a = rand_index(A.v[0], n_s);
      uint64_t b = rand_index(A.v[1], n_s - 1);
      b += (b >= a) ? 1ull : 0ull;
      double s;
      if ((A.v[2] >> 63) == 1ull) {
        s = 1.0;
      } else {
        Philox4 B = philox4x64((uint64_t)t, wid, it, 1ull, T.key0, T.key1);
        double prod = __dmul_rn(__dmul_rn(__dmul_rn(rand_open_unit(B.v[0]), rand_open_unit(B.v[1])),
                                          rand_open_unit(B.v[2])), rand_open_unit(B.v[3]));
        s = __dmul_rn(de_scale, __dmul_rn(-0.25, log(prod)));
      }
      const double* ua = T.surv + a * D;
      const double* ub = T.surv + b * D;
      int in = 1;
      for (int d = 0; d < D; ++d) {
        double x = __dadd_rn(u[d], __dmul_rn(s, __dsub_rn(ua[d], ub[d])));
        if (ev.prior[ev.dim_param[d]].periodic) x = __dsub_rn(x, floor(x));
        if (!(x >= 0.0 && x <= 1.0)) in = 0;
        prop[d] = x;
      }
      inside = in;
      if (in) {
        double th[kParams], ci, sd, cd;
        unit_to_theta(ev, prop, th, &ci, &sd, &cd);
        taylorf2_setup(ev, th, ci, sd, cd, P);
      }
    }
    __syncthreads();
    if (inside) {
      walker_sums<PREC, NDET>(ev, P, red, s_re, s_im);
      if (threadIdx.x == 0) {
        double v = assemble_lnl(ev, P, s_re, s_im);
        ++n_like;
        n_bins += P.k_end;
        if (v > lnl_star) {
          for (int d = 0; d < D; ++d) u[d] = prop[d];
          lnl = v;
          ++n_acc;
        }
      }
    }
    __syncthreads();
  }
  if (threadIdx.x < D) T.u_out[(size_t)j * D + threadIdx.x] = u[threadIdx.x];
  if (threadIdx.x == 0) {
    T.lnl_out[j] = lnl;
    T.n_acc[j] = n_acc;
    T.n_like[j] = n_like;
    if (T.n_bins) T.n_bins[j] = n_bins;
  }
}

}  // namespace

cudaError_t launch_likelihood(int precision, int n_det, const EventDev* d_ev, const double* d_theta, int n,
                              double* d_lnl, int32_t* d_status, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
#define GWNS_LIK(P, N) likelihood_kernel<P, N><<<n, kThreads, 0, s>>>(d_ev, d_theta, n, d_lnl, d_status)
  if (precision == 0) {
    if (n_det == 1) GWNS_LIK(0, 1); else if (n_det == 2) GWNS_LIK(0, 2);
    else if (n_det == 3) GWNS_LIK(0, 3); else GWNS_LIK(0, 4);
  } else {
    if (n_det == 1) GWNS_LIK(1, 1); else if (n_det == 2) GWNS_LIK(1, 2);
    else if (n_det == 3) GWNS_LIK(1, 3); else GWNS_LIK(1, 4);
  }
#undef GWNS_LIK
  return cudaGetLastError();
}

cudaError_t launch_unit_likelihood(int precision, int n_det, const EventDev* d_ev, const double* d_u, int n,
                                   double* d_lnl, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
#define GWNS_UL(P, N) unit_likelihood_kernel<P, N><<<n, kThreads, 0, s>>>(d_ev, d_u, n, d_lnl)
  if (precision == 0) {
    if (n_det == 1) GWNS_UL(0, 1); else if (n_det == 2) GWNS_UL(0, 2);
    else if (n_det == 3) GWNS_UL(0, 3); else GWNS_UL(0, 4);
  } else {
    if (n_det == 1) GWNS_UL(1, 1); else if (n_det == 2) GWNS_UL(1, 2);
    else if (n_det == 3) GWNS_UL(1, 3); else GWNS_UL(1, 4);
  }
#undef GWNS_UL
  return cudaGetLastError();
}

cudaError_t launch_unit_to_theta(const EventDev* d_ev, const double* d_u, int64_t n, double* d_theta,
                                 cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  unit_to_theta_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(d_ev, d_u, n, d_theta);
  return cudaGetLastError();
}

cudaError_t launch_waveform(int n_det, const EventDev* d_ev, const double* d_theta, int n, int n_bins,
                            double* d_hre, double* d_him, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  dim3 grid((n_bins + 255) / 256, n);
#define GWNS_WF(N) waveform_kernel<N><<<grid, 256, 0, s>>>(d_ev, d_theta, n_bins, d_hre, d_him)
  if (n_det == 1) GWNS_WF(1); else if (n_det == 2) GWNS_WF(2); else if (n_det == 3) GWNS_WF(3); else GWNS_WF(4);
#undef GWNS_WF
  return cudaGetLastError();
}

cudaError_t launch_walk(int precision, int n_det, const EventDev* d_evs, WalkTask* d_tasks,
                        const int32_t* d_blk_task, const int32_t* d_blk_local, int n_blocks, cudaStream_t s) {
  if (n_blocks <= 0) return cudaSuccess;
#define GWNS_WALK(P, N) walk_kernel<P, N><<<n_blocks, kThreads, 0, s>>>(d_evs, d_tasks, d_blk_task, d_blk_local)
  if (precision == 0) {
    if (n_det == 1) GWNS_WALK(0, 1); else if (n_det == 2) GWNS_WALK(0, 2);
    else if (n_det == 3) GWNS_WALK(0, 3); else GWNS_WALK(0, 4);
  } else {
    if (n_det == 1) GWNS_WALK(1, 1); else if (n_det == 2) GWNS_WALK(1, 2);
    else if (n_det == 3) GWNS_WALK(1, 3); else GWNS_WALK(1, 4);
  }
#undef GWNS_WALK
  return cudaGetLastError();
}

}  // namespace gwns
