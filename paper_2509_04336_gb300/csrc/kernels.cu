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

// Per-SM arrival counters of walk CTAs.  A CTA's position modulo kThreads/32 picks the warp
// that runs its per-proposal setup, so the CTAs sharing an SM spread that FP64-heavy work
// over different sub-partitions (warp w of a CTA runs on sub-partition w mod 4).
__device__ unsigned int g_walk_sm_arrivals[256];

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
// PREC: 0 = FP64, 1 = mixed with FP64 phase, 2 = mixed with float-float phase.
template <int PREC, int NDET>
__device__ inline void walker_sums(const EventDev& ev, const WalkerParams& P, double (*red)[2 * kMaxDet],
                                   double* s_re, double* s_im) {
  if (PREC == 0) {
    AccF64 acc; acc.zero();
    for (int k = threadIdx.x; k < P.k_end; k += kThreads) bin_accumulate_f64<NDET>(ev, P, k, acc);
    reduce_f64<NDET>(acc, red, s_re, s_im);
  } else {
    AccF32 acc; acc.zero();
    if (PREC == 1) {
      for (int k = threadIdx.x; k < P.k_end; k += kThreads) bin_accumulate_mixed<NDET>(ev, P, k, acc);
    } else {
      for (int k = threadIdx.x; k < P.k_end; k += kThreads) bin_accumulate_ff<NDET>(ev, P, k, acc);
    }
    reduce_mixed<NDET>(acc, red, s_re, s_im);
  }
}

// Warp-level version: the 32 lanes of one warp evaluate one walker; lane 0 receives the sums.
template <int PREC, int NDET>
__device__ inline void warp_sums(const EventDev& ev, const WalkerParams& P, double* s_re, double* s_im) {
  const int lane = threadIdx.x & 31;
  if (PREC == 0) {
    AccF64 acc; acc.zero();
    for (int k = lane; k < P.k_end; k += 32) bin_accumulate_f64<NDET>(ev, P, k, acc);
#pragma unroll
    for (int det = 0; det < NDET; ++det) {
      double r = acc.re[det], i = acc.im[det];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        r += __shfl_down_sync(0xffffffffu, r, off);
        i += __shfl_down_sync(0xffffffffu, i, off);
      }
      s_re[det] = r; s_im[det] = i;
    }
  } else {
    AccF32 acc; acc.zero();
    if (PREC == 1) {
      for (int k = lane; k < P.k_end; k += 32) bin_accumulate_mixed<NDET>(ev, P, k, acc);
    } else {
      for (int k = lane; k < P.k_end; k += 32) bin_accumulate_ff<NDET>(ev, P, k, acc);
    }
#pragma unroll
    for (int det = 0; det < NDET; ++det) {
#pragma unroll
      for (int part = 0; part < 2; ++part) {
        float sv = part ? acc.im[det] : acc.re[det];
        float c = -(part ? acc.cim[det] : acc.cre[det]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          float so = __shfl_down_sync(0xffffffffu, sv, off);
          float co = __shfl_down_sync(0xffffffffu, c, off);
          float t, e;
          two_sum(sv, so, t, e);
          sv = t;
          c = c + co + e;
        }
        double v = (double)sv + (double)c;
        if (part) s_im[det] = v; else s_re[det] = v;
      }
    }
  }
}

// Warp-level sums for the mixed paths left as compensated float pairs (sum, error) in
// lane 0, so that the FP64 conversion and ln L assembly can run later for all proposals at
// once, one lane per proposal.
template <int PREC, int NDET>
__device__ inline void warp_sums_f32(const EventDev& ev, const WalkerParams& P, float* out /*[4 * NDET]*/) {
  const int lane = threadIdx.x & 31;
  AccF32 acc; acc.zero();
  if (PREC == 1) {
    for (int k = lane; k < P.k_end; k += 32) bin_accumulate_mixed<NDET>(ev, P, k, acc);
  } else {
    for (int k = lane; k < P.k_end; k += 32) bin_accumulate_ff<NDET>(ev, P, k, acc);
  }
#pragma unroll
  for (int det = 0; det < NDET; ++det) {
#pragma unroll
    for (int part = 0; part < 2; ++part) {
      float sv = part ? acc.im[det] : acc.re[det];
      float c = -(part ? acc.cim[det] : acc.cre[det]);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        float so = __shfl_down_sync(0xffffffffu, sv, off);
        float co = __shfl_down_sync(0xffffffffu, c, off);
        float t, e;
        two_sum(sv, so, t, e);
        sv = t;
        c = c + co + e;
      }
      if (lane == 0) { out[4 * det + 2 * part] = sv; out[4 * det + 2 * part + 1] = c; }
    }
  }
}

__device__ inline bool theta_ok(const double* th) {
  for (int i = 0; i < kParams; ++i) if (!isfinite(th[i])) return false;
  return th[0] > 0.0 && th[1] > 0.0 && th[4] > 0.0;
}

// Per-walker constants of one proposal: the FP64 path uses the plain FP64 setup, the
// mixed paths the lean one (FP64 only where the phase needs it).
template <int PREC>
__device__ inline void setup_from_unit(const EventDev& ev, const double* u, WalkerParams& P) {
  if (PREC == 0) {
    double th[kParams], ci, sd, cd;
    unit_to_theta(ev, u, th, &ci, &sd, &cd);
    taylorf2_setup(ev, th, ci, sd, cd, P);
  } else {
    LeanTheta t;
    unit_to_lean(ev, u, t);
    taylorf2_setup_lean(ev, t, P);
    if (PREC == 2) make_ff(ev, P);
  }
}

template <int PREC>
__device__ inline void setup_from_theta(const EventDev& ev, const double* th, WalkerParams& P) {
  if (PREC == 0) {
    double sd, cd;
    sincos(th[10], &sd, &cd);
    taylorf2_setup(ev, th, cos(th[5]), sd, cd, P);
  } else {
    LeanTheta t;
    theta_to_lean(th, t);
    taylorf2_setup_lean(ev, t, P);
    if (PREC == 2) make_ff(ev, P);
  }
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
      setup_from_theta<PREC>(ev, th, P);
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
    setup_from_unit<PREC>(ev, u + (size_t)w * ev.n_dim, P);
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
// One CTA per walker, persistent over the walk.  A round looks ahead over the next W steps:
//  1. the DE draws of a step depend only on its Philox counter (step, walker, iteration,
//     tag), not on the chain, so every thread screens one candidate step in FP32 from the
//     current position; the candidates that may lie in the cube are compacted into one warp,
//     which redoes their draws and proposals exactly in FP64 and compacts the in-bounds ones,
//     in step order, into at most m = task.spec slots;
//  2. that warp computes the per-proposal constants (the FP64-heavy part) on full lanes, and
//     the CTA evaluates the slots' likelihoods, one warp per proposal (the whole CTA per
//     proposal when there are fewer than kWarps of them);
//  3. thread 0 replays the steps in order: out-of-bounds steps reject without a likelihood
//     call, the first in-bounds proposal with ln L > ln L* is taken and ends the round.
//     Candidates after it were built from a position the chain has left and are redrawn
//     from the new one in the next round.
// The chain, the accepted and likelihood-call counts and every ln L are those of the walk
// that takes one step at a time.  The setup warp rotates over the CTAs of an SM (an arrival
// counter), so their FP64 work lands on different sub-partitions.
template <int PREC, int NDET>
__global__ void __launch_bounds__(kThreads) walk_kernel(const EventDev* __restrict__ evs, WalkTask* tasks,
                                                         const int32_t* __restrict__ blk_task,
                                                         const int32_t* __restrict__ blk_local) {
  __shared__ WalkerParams P[kSpecMax];
  __shared__ double prop[kSpecMax][kMaxDim];
  __shared__ int cstep[kSpecMax];
  __shared__ int mstep[32];
  __shared__ double lnl_p[kSpecMax];
  __shared__ float part_sums[kSpecMax][4 * kMaxDet];
  __shared__ double u[kMaxDim];
  __shared__ float u32[kMaxDim];
  __shared__ double red[kWarps][2 * kMaxDet];
  __shared__ double s_re[kMaxDet], s_im[kMaxDet];
  __shared__ int wcount[kWarps];
  __shared__ int s_next, s_setup_warp, s_nin, s_end;
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
  const int m = T.spec < 1 ? 1 : (T.spec > kSpecMax ? kSpecMax : T.spec);
  const int window = min(kThreads, max(32, 4 * m));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x < D) {
    u[threadIdx.x] = T.u0[(size_t)j * D + threadIdx.x];
    u32[threadIdx.x] = (float)u[threadIdx.x];
  }
  if (threadIdx.x == 0) {
    unsigned int smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    s_setup_warp = (int)(atomicAdd(&g_walk_sm_arrivals[smid & 255u], 1u) % (unsigned)kWarps);
  }
  double lnl = T.lnl0[j];
  int n_acc = 0, n_like = 0;
  int64_t n_bins = 0, n_spec = 0;
  const double de_scale = 2.38 / sqrt(2.0 * (double)D);
  const float de_scale32 = (float)de_scale;
  __syncthreads();
  const int sw = s_setup_warp;
  int t = 0;
  while (t < n_steps) {
    const int W = min(window, n_steps - t);
    // 1a. every thread screens one candidate step in FP32: a float proposal lies within
    //     ~1e-6 of the FP64 one, so a coordinate more than 1e-5 outside [0, 1] rejects
    //     the step for certain; the rest are "maybe in bounds"
    int maybe = 0;
    const int step = t + (int)threadIdx.x;
    if ((int)threadIdx.x < W) {
      Philox4 A = philox4x64((uint64_t)step, wid, it, 0ull, T.key0, T.key1);
      uint64_t a = rand_index(A.v[0], n_s);
      uint64_t b = rand_index(A.v[1], n_s - 1);
      b += (b >= a) ? 1ull : 0ull;
      float sc = 1.0f;
      if ((A.v[2] >> 63) == 0ull) {
        Philox4 B = philox4x64((uint64_t)step, wid, it, 1ull, T.key0, T.key1);
        // log2 U_i = log2((x_i >> 12) + 1/2) - 52, each factor's integer rounded to float
        // (relative error 6e-8, no truncation, no underflow of the product)
        float l2 = __log2f(__ull2float_rn(B.v[0] >> 12) + 0.5f) + __log2f(__ull2float_rn(B.v[1] >> 12) + 0.5f) +
                   __log2f(__ull2float_rn(B.v[2] >> 12) + 0.5f) + __log2f(__ull2float_rn(B.v[3] >> 12) + 0.5f) -
                   208.0f;
        sc = de_scale32 * (-0.25f * 0.6931471805599453f * l2);
      }
      // |x32 - x64| stays below ~1e-7 (1 + |s|) plus the log2 error times |s|: a margin of
      // 1e-5 (1 + |s|) never rejects a step that the exact FP64 test accepts
      const float margin = 1e-5f * (1.0f + fabsf(sc));
      maybe = 1;
      if (T.surv32) {
        const float* ua = T.surv32 + a * D;
        const float* ub = T.surv32 + b * D;
#pragma unroll
        for (int d = 0; d < kMaxDim; ++d) {
          if (d < D && !ev.prior[ev.dim_param[d]].periodic) {
            float x = u32[d] + sc * (ua[d] - ub[d]);
            if (!(x >= -margin && x <= 1.0f + margin)) maybe = 0;
          }
        }
      } else {
        const double* ua = T.surv + a * D;
        const double* ub = T.surv + b * D;
#pragma unroll
        for (int d = 0; d < kMaxDim; ++d) {
          if (d < D && !ev.prior[ev.dim_param[d]].periodic) {
            float x = u32[d] + sc * ((float)ua[d] - (float)ub[d]);
            if (!(x >= -margin && x <= 1.0f + margin)) maybe = 0;
          }
        }
      }
    }
    unsigned mask = __ballot_sync(0xffffffffu, maybe);
    if (lane == 0) wcount[warp] = __popc(mask);
    __syncthreads();
    int before = 0, total = 0;
#pragma unroll
    for (int w2 = 0; w2 < kWarps; ++w2) {
      int cw = wcount[w2];
      before += (w2 < warp) ? cw : 0;
      total += cw;
    }
    const int mslot = before + __popc(mask & ((1u << lane) - 1u));
    if (maybe && mslot < 32) mstep[mslot] = step;
    const int nmaybe = min(total, 32);
    __syncthreads();
    // 1b. the setup warp redoes the maybe-in-bounds steps exactly (FP64, as the walk is
    //     defined) and compacts the in-bounds ones into at most m slots
    if (warp == sw) {
      int in = 0;
      double pr[kMaxDim];
      const int st = lane < nmaybe ? mstep[lane] : 0;
      if (lane < nmaybe) {
        Philox4 A = philox4x64((uint64_t)st, wid, it, 0ull, T.key0, T.key1);
        uint64_t a = rand_index(A.v[0], n_s);
        uint64_t b = rand_index(A.v[1], n_s - 1);
        b += (b >= a) ? 1ull : 0ull;
        double sc;
        if ((A.v[2] >> 63) == 1ull) {
          sc = 1.0;
        } else {
          Philox4 B = philox4x64((uint64_t)st, wid, it, 1ull, T.key0, T.key1);
          double prod = __dmul_rn(__dmul_rn(__dmul_rn(rand_open_unit(B.v[0]), rand_open_unit(B.v[1])),
                                            rand_open_unit(B.v[2])), rand_open_unit(B.v[3]));
          sc = __dmul_rn(de_scale, __dmul_rn(-0.25, log(prod)));
        }
        const double* ua = T.surv + a * D;
        const double* ub = T.surv + b * D;
        in = 1;
#pragma unroll
        for (int d = 0; d < kMaxDim; ++d) {
          if (d < D) {
            double x = __dadd_rn(u[d], __dmul_rn(sc, __dsub_rn(ua[d], ub[d])));
            if (ev.prior[ev.dim_param[d]].periodic) x = __dsub_rn(x, floor(x));
            // 0 <= x <= 1 on the bit pattern (integer pipe): +0 .. 1.0 are the patterns up
            // to 0x3FF0000000000000; negative values and NaN compare above.  x is never -0.
            if ((unsigned long long)__double_as_longlong(x) > 0x3FF0000000000000ull) in = 0;
            pr[d] = x;
          }
        }
      }
      const unsigned im = __ballot_sync(0xffffffffu, in);
      const int slot = __popc(im & ((1u << lane) - 1u));
      if (in && slot < m) {
#pragma unroll
        for (int d = 0; d < kMaxDim; ++d)
          if (d < D) prop[slot][d] = pr[d];
        cstep[slot] = st;
      }
      const int nin_w = min(__popc(im), m);
      // steps covered by this round: up to the m-th in-bounds proposal, else up to the last
      // screened maybe-step, else the whole window
      const unsigned mth = __ballot_sync(0xffffffffu, in && slot == m - 1);
      int end;
      if (__popc(im) > m) end = __shfl_sync(0xffffffffu, st, __ffs(mth) - 1);
      else if (total > 32) end = __shfl_sync(0xffffffffu, st, 31);
      else end = t + W - 1;
      if (lane == 0) { s_nin = nin_w; s_end = end; }
      __syncwarp();
      if (lane < nin_w) setup_from_unit<PREC>(ev, prop[lane], P[lane]);
    }
    __syncthreads();
    const int nin = s_nin;
    // 2. likelihoods
    if (PREC != 0 && nin >= kWarps) {
      for (int i = warp; i < nin; i += kWarps) warp_sums_f32<PREC, NDET>(ev, P[i], part_sums[i]);
      __syncthreads();
      if (warp == sw && lane < nin) {
        double sr[kMaxDet], si[kMaxDet];
#pragma unroll
        for (int det = 0; det < NDET; ++det) {
          sr[det] = (double)part_sums[lane][4 * det] + (double)part_sums[lane][4 * det + 1];
          si[det] = (double)part_sums[lane][4 * det + 2] + (double)part_sums[lane][4 * det + 3];
        }
        lnl_p[lane] = assemble_lnl(ev, P[lane], sr, si);
      }
    } else if (nin >= kWarps) {
      for (int i = warp; i < nin; i += kWarps) {
        double sr[kMaxDet], si[kMaxDet];
        warp_sums<PREC, NDET>(ev, P[i], sr, si);
        if (lane == 0) lnl_p[i] = assemble_lnl(ev, P[i], sr, si);
      }
    } else {
      for (int i = 0; i < nin; ++i) {
        walker_sums<PREC, NDET>(ev, P[i], red, s_re, s_im);
        if (threadIdx.x == 0) lnl_p[i] = assemble_lnl(ev, P[i], s_re, s_im);
        __syncthreads();
      }
    }
    __syncthreads();
    // 3. the steps in order
    if (threadIdx.x == 0) {
      int nxt = s_end + 1;
      for (int i = 0; i < nin; ++i) {
        ++n_like;
        n_bins += P[i].k_end;
        if (lnl_p[i] > lnl_star) {
          for (int d = 0; d < D; ++d) { u[d] = prop[i][d]; u32[d] = (float)prop[i][d]; }
          lnl = lnl_p[i];
          ++n_acc;
          nxt = cstep[i] + 1;
          break;
        }
      }
      n_spec += nin;
      s_next = nxt;
    }
    __syncthreads();
    t = s_next;
  }
  if (threadIdx.x < D) T.u_out[(size_t)j * D + threadIdx.x] = u[threadIdx.x];
  if (threadIdx.x == 0) {
    T.lnl_out[j] = lnl;
    T.n_acc[j] = n_acc;
    T.n_like[j] = n_like;
    if (T.n_bins) T.n_bins[j] = n_bins;
    if (T.n_spec) T.n_spec[j] = n_spec;
  }
}

}  // namespace

// Instantiate a kernel macro K(P, N) for the precision and detector count of a call.
#define GWNS_DISPATCH(K)                                                          \
  if (precision == 0) {                                                           \
    if (n_det == 1) K(0, 1); else if (n_det == 2) K(0, 2);                        \
    else if (n_det == 3) K(0, 3); else K(0, 4);                                   \
  } else if (precision == 1) {                                                    \
    if (n_det == 1) K(1, 1); else if (n_det == 2) K(1, 2);                        \
    else if (n_det == 3) K(1, 3); else K(1, 4);                                   \
  } else {                                                                        \
    if (n_det == 1) K(2, 1); else if (n_det == 2) K(2, 2);                        \
    else if (n_det == 3) K(2, 3); else K(2, 4);                                   \
  }

cudaError_t launch_likelihood(int precision, int n_det, const EventDev* d_ev, const double* d_theta, int n,
                              double* d_lnl, int32_t* d_status, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
#define GWNS_LIK(P, N) likelihood_kernel<P, N><<<n, kThreads, 0, s>>>(d_ev, d_theta, n, d_lnl, d_status)
  GWNS_DISPATCH(GWNS_LIK)
#undef GWNS_LIK
  return cudaGetLastError();
}

cudaError_t launch_unit_likelihood(int precision, int n_det, const EventDev* d_ev, const double* d_u, int n,
                                   double* d_lnl, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
#define GWNS_UL(P, N) unit_likelihood_kernel<P, N><<<n, kThreads, 0, s>>>(d_ev, d_u, n, d_lnl)
  GWNS_DISPATCH(GWNS_UL)
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
  GWNS_DISPATCH(GWNS_WALK)
#undef GWNS_WALK
  return cudaGetLastError();
}

}  // namespace gwns
