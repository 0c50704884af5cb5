// kernels_impl.cuh -- likelihood, waveform and acceptance-walk kernels (sm_103a).
// Included by kernels_p{0,1,2}.cu, one translation unit per precision (parallel builds).
//
// Template parameters of every kernel: PREC (0 FP64, 1 mixed with FP64 phase, 2 mixed with
// float-float phase), NDET (detectors, 1..4) and WF (0 TaylorF2, 1 IMRPhenomD form).
// Per-bin sums per detector: Re and Im of S_det = sum_k a_k z_k exp(-2 pi i Phi_det(f_k)), and
// for the IMRPhenomD form the template power sum_k a_k^2 4 df f^-7/3 / S (TaylorF2 takes it
// from prefix sums).  Threads accumulate disjoint bin subsets (FP64, or FP32 with Kahan
// compensation), then warp-shuffle trees (error-free two-sums in FP32) reduce them.
#pragma once

#include <cstdio>
#include <type_traits>

#include "flow.cuh"
#include "gwns_internal.h"

namespace gwns {

namespace {

// Per-SM arrival counters of walk CTAs.  A CTA's position modulo kThreads/32 picks the warp
// that runs its per-proposal setup, so the CTAs sharing an SM spread that FP64-heavy work
// over different sub-partitions (warp w of a CTA runs on sub-partition w mod 4).
__device__ unsigned int g_walk_sm_arrivals[256];

constexpr int kWarps = kThreads / 32;
constexpr int kMaxVals = 3 * kMaxDet;   // (re, im, hh) per detector

// (x >> 12) + 1/2 as a float (relative error ~1e-7) from two 32-bit conversions: a 64-bit
// integer conversion runs on the FP64 pipe.
__device__ __forceinline__ float top52_half_f(uint64_t x) {
  const uint64_t v = x >> 12;
  return fmaf(__uint2float_rn((uint32_t)(v >> 20)), 1048576.0f, __uint2float_rn((uint32_t)(v & 0xFFFFFull)) + 0.5f);
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// The watchdog of a walk's thread 0: a host-set abort flag (read at the start of a round, so that
// the load's latency overlaps the round) and the task's time budget (nanoseconds since the CTA
// started).
__device__ __forceinline__ int walk_abort_flag(const WalkTask& T) {
  return T.abort ? *(volatile const int32_t*)T.abort : 0;
}
__device__ __forceinline__ bool walk_should_stop(const WalkTask& T, uint64_t t0, int abort_flag) {
  return abort_flag != 0 || (T.budget_ns != 0ull && global_ns() - t0 > T.budget_ns);
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

template <int NDET, int WF>
struct NVals { static constexpr int value = (WF == 1 ? 3 : 2) * NDET; };

// Partial sums of the bins k = start, start + stride, ... of one walker (values laid out
// [det][re, im(, hh)]).  FP64 path: dv; mixed paths: (fv, fc) Kahan pairs, fc the negated error.
template <int PREC, int NDET, int WF>
__device__ inline void partials(const EventDev& ev, const WalkerParams& P, int start, int stride, double* dv,
                                float* fv, float* fc) {
  constexpr int NW = (WF == 1 ? 3 : 2);
  if (WF == 0) {
    if (PREC == 0) {
      AccF64 acc; acc.zero();
      for (int k = start; k < P.k_end; k += stride) bin_accumulate_f64<NDET>(ev, P, k, acc);
#pragma unroll
      for (int d = 0; d < NDET; ++d) { dv[NW * d] = acc.re[d]; dv[NW * d + 1] = acc.im[d]; }
    } else {
      AccF32 acc; acc.zero();
      if (PREC == 1) {
        for (int k = start; k < P.k_end; k += stride) bin_accumulate_mixed<NDET>(ev, P, k, acc);
      } else {
        for (int k = start; k < P.k_end; k += stride) bin_accumulate_ff<NDET>(ev, P, k, acc);
      }
#pragma unroll
      for (int d = 0; d < NDET; ++d) {
        fv[NW * d] = acc.re[d]; fc[NW * d] = -acc.cre[d];
        fv[NW * d + 1] = acc.im[d]; fc[NW * d + 1] = -acc.cim[d];
      }
    }
  } else {
    if (PREC == 0) {
      AccPD64 acc; acc.zero();
      for (int k = start; k < P.k_end; k += stride) pd_accumulate_f64<NDET>(ev, P, P.pd, k, acc);
#pragma unroll
      for (int d = 0; d < NDET; ++d) { dv[NW * d] = acc.re[d]; dv[NW * d + 1] = acc.im[d]; dv[NW * d + 2] = acc.hh[d]; }
    } else {
      AccPD32 acc; acc.zero();
      if (PREC == 1) {
        for (int k = start; k < P.k_end; k += stride) pd_accumulate_mixed<NDET>(ev, P, P.pd, k, acc);
      } else {
        for (int k = start; k < P.k_end; k += stride) pd_accumulate_ff<NDET>(ev, P, P.pd, k, acc);
      }
#pragma unroll
      for (int d = 0; d < NDET; ++d) {
        fv[NW * d] = acc.re[d]; fc[NW * d] = -acc.cre[d];
        fv[NW * d + 1] = acc.im[d]; fc[NW * d + 1] = -acc.cim[d];
        fv[NW * d + 2] = acc.hh[d]; fc[NW * d + 2] = -acc.chh[d];
      }
    }
  }
}

// Warp reductions: lane 0 receives the totals.
template <int NV>
__device__ __forceinline__ void warp_reduce_f64(double* dv) {
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double r = dv[i];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) r += __shfl_down_sync(0xffffffffu, r, off);
    dv[i] = r;
  }
}

// Compensated all-lane sums of NV values by recursive halving: at the exchange with offset
// S each lane keeps half of the values it still carries (the upper half when bit S of its
// lane is set) and adds its partner's copy of that half, so V = NV rounded up to a power of
// two values need V - 1 pair exchanges before the last value is reduced over the remaining
// lanes (instead of NV * 5).  Every addition is an error-free two-sum whose error joins the
// compensation.  On return lane l holds the total (s, c) of value index
// vbits(l) = bits 4, 3, ... of l read as the binary digits of the index (most significant
// first), for log2 V digits.
template <int V, int S>
__device__ __forceinline__ void halve_step(float* s, float* c, int lane) {
  const bool up = (lane & S) != 0;
#pragma unroll
  for (int i = 0; i < V / 2; ++i) {
    const float ss = up ? s[i] : s[i + V / 2], sc = up ? c[i] : c[i + V / 2];
    const float ks = up ? s[i + V / 2] : s[i], kc = up ? c[i + V / 2] : c[i];
    const float os = __shfl_xor_sync(0xffffffffu, ss, S), oc = __shfl_xor_sync(0xffffffffu, sc, S);
    float t, e;
    two_sum(ks, os, t, e);
    s[i] = t;
    c[i] = kc + oc + e;
  }
}
template <int S>
__device__ __forceinline__ void fold_step(float& s, float& c) {
  const float os = __shfl_xor_sync(0xffffffffu, s, S), oc = __shfl_xor_sync(0xffffffffu, c, S);
  float t, e;
  two_sum(s, os, t, e);
  s = t;
  c = c + oc + e;
}
template <int NV>
struct Pow2Vals { static constexpr int value = NV <= 2 ? 2 : NV <= 4 ? 4 : NV <= 8 ? 8 : 16; };
// (s, c) of the value this lane ends with; *index receives that value's index.
template <int NV>
__device__ __forceinline__ void warp_halving_sums(const float* fv, const float* fc, int lane, float& s_out,
                                                  float& c_out, int& index) {
  constexpr int V = Pow2Vals<NV>::value;
  float s[V], c[V];
#pragma unroll
  for (int i = 0; i < V; ++i) { s[i] = i < NV ? fv[i] : 0.0f; c[i] = i < NV ? fc[i] : 0.0f; }
  halve_step<V, 16>(s, c, lane);
  if (V >= 4) halve_step<V / 2, 8>(s, c, lane);
  if (V >= 8) halve_step<V / 4, 4>(s, c, lane);
  if (V >= 16) halve_step<V / 8, 2>(s, c, lane);
  float rs = s[0], rc = c[0];
  if (V <= 8) fold_step<2>(rs, rc);
  if (V <= 4) fold_step<4>(rs, rc);
  if (V <= 2) fold_step<8>(rs, rc);
  fold_step<1>(rs, rc);
  int idx = 0;
  idx = (idx << 1) | ((lane >> 4) & 1);
  if (V >= 4) idx = (idx << 1) | ((lane >> 3) & 1);
  if (V >= 8) idx = (idx << 1) | ((lane >> 2) & 1);
  if (V >= 16) idx = (idx << 1) | ((lane >> 1) & 1);
  s_out = rs;
  c_out = rc;
  index = idx;
}

// The same halving in FP64 (plain additions): lane l ends with the total of value index
// vbits(l), as above.
template <int V, int S>
__device__ __forceinline__ void halve_step_f64(double* s, int lane) {
  const bool up = (lane & S) != 0;
#pragma unroll
  for (int i = 0; i < V / 2; ++i) {
    const double send = up ? s[i] : s[i + V / 2], keep = up ? s[i + V / 2] : s[i];
    s[i] = keep + __shfl_xor_sync(0xffffffffu, send, S);
  }
}
template <int S>
__device__ __forceinline__ void fold_step_f64(double& s) {
  s = s + __shfl_xor_sync(0xffffffffu, s, S);
}
template <int NV>
__device__ __forceinline__ void warp_halving_f64(const double* dv, int lane, double& out, int& index) {
  constexpr int V = Pow2Vals<NV>::value;
  double s[V];
#pragma unroll
  for (int i = 0; i < V; ++i) s[i] = i < NV ? dv[i] : 0.0;
  halve_step_f64<V, 16>(s, lane);
  if (V >= 4) halve_step_f64<V / 2, 8>(s, lane);
  if (V >= 8) halve_step_f64<V / 4, 4>(s, lane);
  if (V >= 16) halve_step_f64<V / 8, 2>(s, lane);
  double r = s[0];
  if (V <= 8) fold_step_f64<2>(r);
  if (V <= 4) fold_step_f64<4>(r);
  if (V <= 2) fold_step_f64<8>(r);
  fold_step_f64<1>(r);
  int idx = (lane >> 4) & 1;
  if (V >= 4) idx = (idx << 1) | ((lane >> 3) & 1);
  if (V >= 8) idx = (idx << 1) | ((lane >> 2) & 1);
  if (V >= 16) idx = (idx << 1) | ((lane >> 1) & 1);
  out = r;
  index = idx;
}

// One proposal's sum has one order whichever threads evaluate it, so that its ln L does not
// depend on the round it was drawn in or on the kernel that evaluates it: chunk w (w = 0..3) is
// the bins 32 w + l + 128 m (m = 0, 1, ...) summed in order on lane l, the lanes' values are
// reduced by the halving tree (compensated in the mixed paths, then converted to FP64), and
// the four chunk totals are added in the order of w in FP64.  The whole CTA forms chunk w on
// warp w; a warp that evaluates a proposal alone forms the four chunks in turn.
//
// chunk_total: this warp's chunk total of every value into out[0 .. NV) (shared memory).
template <int PREC, int NV>
__device__ __forceinline__ void chunk_total(const double* dv, const float* fv, const float* fc, int lane,
                                            double* out) {
  constexpr int group = 32 / Pow2Vals<NV>::value;
  int q;
  if (PREC == 0) {
    double r;
    warp_halving_f64<NV>(dv, lane, r, q);
    if ((lane & (group - 1)) == 0 && q < NV) out[q] = r;
  } else {
    float rs, rc;
    warp_halving_sums<NV>(fv, fc, lane, rs, rc, q);
    if ((lane & (group - 1)) == 0 && q < NV) out[q] = (double)rs + (double)rc;
  }
}
// value q of the four chunk totals ct[w][q], added in chunk order
template <int NV>
__device__ __forceinline__ double chunks_sum(const double (*ct)[NV], int q) {
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) t = t + ct[w][q];
  return t;
}
// The four chunks of one proposal on one warp: totals into ct[0 .. kWarps)[0 .. NV).
template <int PREC, int NDET, int WF>
__device__ inline void warp_chunks(const EventDev& ev, const WalkerParams& P, int lane,
                                   double (*ct)[NVals<NDET, WF>::value]) {
  constexpr int NV = NVals<NDET, WF>::value;
#pragma unroll 1
  for (int w = 0; w < kWarps; ++w) {
    double dv[NV];
    float fv[NV], fc[NV];
    partials<PREC, NDET, WF>(ev, P, 32 * w + lane, kThreads, dv, fv, fc);
    chunk_total<PREC, NV>(dv, fv, fc, lane, ct[w]);
  }
  __syncwarp();
}

// Sums of one walker over the whole CTA: totals in `out` (shared), visible to every thread on
// return; `ct` holds the warps' chunk totals.
template <int PREC, int NDET, int WF>
__device__ inline void cta_sums(const EventDev& ev, const WalkerParams& P, double (*ct)[NVals<NDET, WF>::value],
                                double* out) {
  constexpr int NV = NVals<NDET, WF>::value;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double dv[NV];
  float fv[NV], fc[NV];
  partials<PREC, NDET, WF>(ev, P, threadIdx.x, kThreads, dv, fv, fc);
  chunk_total<PREC, NV>(dv, fv, fc, lane, ct[warp]);
  __syncthreads();
  if (threadIdx.x < NV) out[threadIdx.x] = chunks_sum<NV>(ct, threadIdx.x);
  __syncthreads();
}

// ln L from reduced values laid out [det][re, im(, hh)]; the mixed paths' template-power sums
// are in units of the scaled FP32 weights.
template <int PREC, int NDET, int WF>
__device__ inline double lnl_from_vals(const EventDev& ev, const WalkerParams& P, const double* v) {
  constexpr int NW = (WF == 1 ? 3 : 2);
  if (PREC == 2) {   // the float-float path's scaled FP32 amplitudes
    double dh = 0.0, hh = (double)P.hh_f;
#pragma unroll
    for (int d = 0; d < NDET; ++d) {
      dh += (double)P.kpf_re[d] * v[NW * d] - (double)P.kpf_im[d] * v[NW * d + 1];
      if (WF == 1)
        hh += ((double)P.kpf_re[d] * P.kpf_re[d] + (double)P.kpf_im[d] * P.kpf_im[d]) * v[NW * d + 2] *
              (double)ev.hh_unscale_f;
    }
    dh = ldexp(dh, -kKpScaleExp);
    return ev.use_ratio ? dh - 0.5 * hh : -0.5 * (ev.dd_total - 2.0 * dh + hh);
  }
  double sr[kMaxDet], si[kMaxDet], sh[kMaxDet];
  const double hscale = PREC == 0 ? 1.0 : ev.gw32_unscale;
#pragma unroll
  for (int d = 0; d < NDET; ++d) {
    sr[d] = v[NW * d];
    si[d] = v[NW * d + 1];
    sh[d] = (WF == 1) ? v[NW * d + 2] * hscale : 0.0;
  }
  return assemble_lnl(ev, P, sr, si, WF == 1 ? sh : nullptr);
}

// ln L of the float-float TaylorF2 path in float-float arithmetic from the compensated
// per-detector sums ps = [det][re, im] x (sum, compensation): FP64 only converts the result.
template <int NDET, int WF>
__device__ inline double lnl_ff(const EventDev& ev, const WalkerParams& P, const float* ps) {
  constexpr int NS = (WF == 1 ? 6 : 4);   // floats per detector: (re, im(, hh)) x (sum, compensation)
  ff dh = ff_make(0.0f);
  float hh = P.hh_f;
#pragma unroll
  for (int d = 0; d < NDET; ++d) {
    const ff sr = fast_two_sum_ff(ps[NS * d], ps[NS * d + 1]);
    const ff si = fast_two_sum_ff(ps[NS * d + 2], ps[NS * d + 3]);
    dh = ff_add(dh, ff_sub(ff_mul_f(sr, P.kpf_re[d]), ff_mul_f(si, P.kpf_im[d])));
    if (WF == 1)
      hh += (P.kpf_re[d] * P.kpf_re[d] + P.kpf_im[d] * P.kpf_im[d]) * ((ps[NS * d + 4] + ps[NS * d + 5]) * ev.hh_unscale_f);
  }
  dh = ff_ldexp(dh, -kKpScaleExp);
  ff l;
  if (ev.use_ratio) {
    l = ff_add_f(dh, -0.5f * hh);
  } else {
    l = ff_add_f(ff_sub(ff_ldexp(dh, 1), ff{ev.dd_f[0], ev.dd_f[1]}), -hh);
    l = ff_ldexp(l, -1);
  }
  return (double)l.h + (double)l.l;
}

// ---------------------------------------------------------------- relative binning
// The float-float TaylorF2 phase at grid bin k [cycles, reduced to [-1/2, 1/2] plus a small
// low part], as the first half of bin_accumulate_ff computes it.
__device__ __forceinline__ float tf2_ff_r0(const EventDev& ev, const WalkerParams& p, int k) {
  const float2* g = ev.basis_ff + k;
  const size_t gs = (size_t)ev.n_bins;
  float q[kBasis];
  float sl = p.ph0l;
#pragma unroll
  for (int j = 0; j < kBasis; ++j) {
    const float2 gj = g[j * gs];
    q[j] = p.Ch[j] * gj.x;
    float e = fmaf(p.Ch[j], gj.x, -q[j]);
    e = fmaf(p.Ch[j], gj.y, e);
    sl += fmaf(p.Cl[j], gj.x, e);
  }
#pragma unroll
  for (int w = 1; w < kBasis; w <<= 1) {
#pragma unroll
    for (int j = 0; j + w < kBasis; j += 2 * w) {
      const float t = q[j] + q[j + w];
      const float bb = t - q[j];
      sl += (q[j] - (t - bb)) + (q[j + w] - bb);
      q[j] = t;
    }
  }
  const float t = p.ph0h + q[0];
  const float bb = t - p.ph0h;
  sl += (p.ph0h - (t - bb)) + (q[0] - bb);
  return (t - rintf(t)) + sl;
}

// The float-float IMRPhenomD-form phase [cycles] and amplitude shape at grid bin k, as the first
// half of pd_accumulate_ff computes them.
__device__ __forceinline__ void pd_ff_r0_amp(const EventDev& ev, const WalkerParams& p, const PhenomExtra& e,
                                             int k, float& r0, float& amp) {
  const float2* g = ev.basis_ff + k;
  const size_t gs = (size_t)ev.n_bins;
  const float ff = g[13 * gs].x;
  float sh, sl, extra = 0.f;
  if (k < e.k1) {
    sh = p.ph0h; sl = p.ph0l;
#pragma unroll
    for (int j = 0; j < 8; ++j) ff_term(sh, sl, p.Ch[j], p.Cl[j], g[j * gs]);
    ff_term(sh, sl, e.Cxh[0], e.Cxl[0], g[8 * gs]);
    ff_term(sh, sl, e.Cxh[1], e.Cxl[1], g[9 * gs]);
    ff_term(sh, sl, e.Cxh[2], e.Cxl[2], g[10 * gs]);
  } else if (k < e.k2) {
    sh = e.ph0_int_h; sl = e.ph0_int_l;
    ff_term(sh, sl, e.Cxh[3], e.Cxl[3], g[6 * gs]);
    ff_term(sh, sl, e.Cxh[4], e.Cxl[4], g[11 * gs]);
    ff_term(sh, sl, e.Cxh[5], e.Cxl[5], g[13 * gs]);
  } else {
    sh = e.ph0_mr_h; sl = e.ph0_mr_l;
    ff_term(sh, sl, e.Cxh[6], e.Cxl[6], g[1 * gs]);
    ff_term(sh, sl, e.Cxh[7], e.Cxl[7], g[12 * gs]);
    ff_term(sh, sl, e.Cxh[8], e.Cxl[8], g[13 * gs]);
    extra = e.at_scalef * atanf((e.Mf * ff - e.at_cf) * e.at_invf);
  }
  r0 = (sh - rintf(sh)) + sl + extra;
  amp = pd_amp_f32(e, k, ff, g[4 * gs].x);
}

// ln L of one proposal with the relative-binning likelihood (mode 2), evaluated by one warp
// (every lane returns it).  Coarse bins wholly below the proposal's cutoff whose right edge is
// a grid bin take the linear expansion of r = h / h0 between their edges (31 bins a pass; lane
// l holds edge base + l and reads its right neighbour by a shuffle); from the first other coarse
// bin up to the cutoff the active bins are summed exactly with the per-bin bodies.  *bins
// receives the grid bins the evaluation touched (edges plus the exact range).
template <int NDET, int WF>
__device__ double rb_lnl_warp(const EventDev& ev, const WalkerParams& P, int lane, int* bins = nullptr) {
  const int nb = ev.rb_nb;
  const int32_t* E = ev.rb_edges;
  const int k_end = P.k_end;
  const int kmax = min(k_end, ev.n_bins - 1);
  int lo = 0, hi = nb;   // n_full = the largest n with E[n] <= kmax (E[0] = 0)
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (E[mid] <= kmax) lo = mid;
    else hi = mid - 1;
  }
  const int n_full = lo;
  float dh = 0.f, dhc = 0.f, hh = 0.f, hhc = 0.f;
  const float df = ev.df_f[0];
  for (int base = 0; base < n_full; base += 31) {
    const int ei = base + lane;
    const bool have = ei <= n_full;
    float rre[NDET], rim[NDET];
#pragma unroll
    for (int det = 0; det < NDET; ++det) { rre[det] = 0.f; rim[det] = 0.f; }
    if (have) {
      const int k = E[ei];
      float r0, amp = 1.0f;
      if (WF == 0) r0 = tf2_ff_r0(ev, P, k);
      else pd_ff_r0_amp(ev, P, P.pd, k, r0, amp);
      const float kf = (float)k;
#pragma unroll
      for (int det = 0; det < NDET; ++det) {
        const float kb = kf * P.sbh[det];
        float ph = (r0 + P.sa[det]) + (kb - rintf(kb)) + kf * P.sbl[det];
        ph = ph - rintf(ph);
        float sn, cs;
        sincos_turn_sfu(ph, &sn, &cs);
        // h f^(7/6) 2^70 = amp (K P) exp(-2 pi i ph)
        const float hre = amp * (P.kpf_re[det] * cs + P.kpf_im[det] * sn);
        const float him = amp * (P.kpf_im[det] * cs - P.kpf_re[det] * sn);
        const float2 q = ev.rb_q0[(size_t)det * nb + ei];
        rre[det] = hre * q.x - him * q.y;
        rim[det] = hre * q.y + him * q.x;
      }
    }
    const int b = base + lane;
    const bool bin = lane < 31 && b < n_full;
    const float inv = bin ? 1.0f / ((float)(E[b + 1] - E[b]) * df) : 0.f;
#pragma unroll
    for (int det = 0; det < NDET; ++det) {
      const float nre = __shfl_down_sync(0xffffffffu, rre[det], 1);
      const float nim = __shfl_down_sync(0xffffffffu, rim[det], 1);
      if (bin) {
        const float r1re = (nre - rre[det]) * inv, r1im = (nim - rim[det]) * inv;
        const float2 a0 = ev.rb_a[((size_t)det * nb + b) * 2];
        const float2 a1 = ev.rb_a[((size_t)det * nb + b) * 2 + 1];
        const float4 bq = ev.rb_b[(size_t)det * nb + b];
        kahan_add(dh, dhc, a0.x * rre[det] - a0.y * rim[det] + a1.x * r1re - a1.y * r1im);
        kahan_add(hh, hhc, bq.x * (rre[det] * rre[det] + rim[det] * rim[det]) +
                               2.0f * bq.y * (rre[det] * r1re + rim[det] * r1im) +
                               bq.z * (r1re * r1re + r1im * r1im));
      }
    }
  }
  // exact part: the active bins from the first coarse bin not expanded
  const int kx = E[n_full];
  if (bins) *bins = n_full + 1 + max(k_end - kx, 0);
  double xdh = 0.0, xhh = 0.0;
  if (WF == 0) {
    AccF32 acc;
    acc.zero();
    for (int k = kx + lane; k < k_end; k += 32) bin_accumulate_ff<NDET>(ev, P, k, acc);
    float sdh = 0.f;
#pragma unroll
    for (int det = 0; det < NDET; ++det)
      sdh += P.kpf_re[det] * (acc.re[det] - acc.cre[det]) - P.kpf_im[det] * (acc.im[det] - acc.cim[det]);
    xdh = ldexp((double)sdh, -kKpScaleExp);
    if (lane == 0 && kx < k_end) {
      float hsum = 0.f;
      for (int det = 0; det < NDET; ++det) {
        const float* pre = ev.hhp32 + (size_t)det * ev.n_bins;
        const float seg = pre[k_end - 1] - (kx > 0 ? pre[kx - 1] : 0.f);
        hsum += (P.kpf_re[det] * P.kpf_re[det] + P.kpf_im[det] * P.kpf_im[det]) * seg;
      }
      xhh = (double)hsum;
    }
  } else {
    AccPD32 acc;
    acc.zero();
    for (int k = kx + lane; k < k_end; k += 32) pd_accumulate_ff<NDET>(ev, P, P.pd, k, acc);
    float sdh = 0.f, shh = 0.f;
#pragma unroll
    for (int det = 0; det < NDET; ++det) {
      sdh += P.kpf_re[det] * (acc.re[det] - acc.cre[det]) - P.kpf_im[det] * (acc.im[det] - acc.cim[det]);
      shh += (P.kpf_re[det] * P.kpf_re[det] + P.kpf_im[det] * P.kpf_im[det]) * acc.hh[det];
    }
    xdh = ldexp((double)sdh, -kKpScaleExp);
    xhh = (double)shh * (double)ev.hh_unscale_f;
  }
  double tdh = (double)dh - (double)dhc + xdh;
  double thh = (double)hh - (double)hhc + xhh;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    tdh += __shfl_xor_sync(0xffffffffu, tdh, off);
    thh += __shfl_xor_sync(0xffffffffu, thh, off);
  }
  return ev.use_ratio ? tdh - 0.5 * thh : -0.5 * (ev.dd_total - 2.0 * tdh + thh);
}

__device__ inline bool theta_ok(const double* th) {
  for (int i = 0; i < kParams; ++i) if (!isfinite(th[i])) return false;
  return th[0] > 0.0 && th[1] > 0.0 && th[4] > 0.0;
}

// Per-walker constants of one proposal: the FP64 path uses the plain FP64 setup, the mixed
// paths the lean one (FP64 only where the phase needs it).
template <int PREC, int WF>
__device__ inline void setup_from_unit(const EventDev& ev, const double* u, WalkerParams& P) {
  if (PREC == 0) {
    double th[kParams], ci, sd, cd;
    unit_to_theta(ev, u, th, &ci, &sd, &cd);
    taylorf2_setup<WF>(ev, th, ci, sd, cd, P);
  } else if (PREC == 2 && ev.ff_setup) {
    ff x[kMaxDim];
#pragma unroll
    for (int d = 0; d < kMaxDim; ++d) x[d] = d < ev.n_dim ? ff_from_double(u[d]) : ff_make(0.0f);
    if (WF == 0) taylorf2_setup_ff(ev, x, P);
    else phenomd_setup_ff(ev, x, P);
  } else {
    LeanTheta t;
    unit_to_lean(ev, u, t);
    taylorf2_setup_lean<WF>(ev, t, P);
    if (PREC == 2) make_ff<WF>(ev, P);
  }
}

template <int PREC, int WF>
__device__ inline void setup_from_theta(const EventDev& ev, const double* th, WalkerParams& P) {
  if (PREC == 0) {
    double sd, cd;
    sincos(th[10], &sd, &cd);
    taylorf2_setup<WF>(ev, th, cos(th[5]), sd, cd, P);
  } else {
    LeanTheta t;
    theta_to_lean(th, t);
    taylorf2_setup_lean<WF>(ev, t, P);
    if (PREC == 2) make_ff<WF>(ev, P);
  }
}

// ---------------------------------------------------------------- likelihood batch
template <int PREC, int NDET, int WF>
__global__ void __launch_bounds__(kThreads) likelihood_kernel(const EventDev* __restrict__ evp,
                                                               const double* __restrict__ theta, int n,
                                                               double* __restrict__ lnl, int32_t* status) {
  __shared__ WalkerParams P;
  __shared__ double red[kWarps][NVals<NDET, WF>::value];
  __shared__ double vals[kMaxVals];
  __shared__ int ok;
  const EventDev& ev = *evp;
  const int w = blockIdx.x;
  if (threadIdx.x == 0) {
    double th[kParams];
    for (int i = 0; i < kParams; ++i) th[i] = theta[(size_t)w * kParams + i];
    ok = theta_ok(th);
    if (ok) setup_from_theta<PREC, WF>(ev, th, P);
    else P.k_end = 0;
  }
  __syncthreads();
  if constexpr (PREC == 2) {
    if (ev.rb_nb > 0) {   // relative binning: warp 0 evaluates the proposal
      if (threadIdx.x < 32) {
        const double v = ok ? rb_lnl_warp<NDET, WF>(ev, P, threadIdx.x) : 0.0;
        if (threadIdx.x == 0) {
          if (ok) {
            lnl[w] = v;
          } else {
            lnl[w] = __longlong_as_double(0x7ff8000000000000ll);
            atomicOr(status, 1);
          }
        }
      }
      return;
    }
  }
  cta_sums<PREC, NDET, WF>(ev, P, red, vals);
  if (threadIdx.x == 0) {
    if (ok) {
      lnl[w] = lnl_from_vals<PREC, NDET, WF>(ev, P, vals);
    } else {
      lnl[w] = __longlong_as_double(0x7ff8000000000000ll);
      atomicOr(status, 1);
    }
  }
}

// ln L of unit-cube points u [n][D] (prior transform, then the likelihood).  Used for the
// initial live points; non-finite results are stored as -inf so that they die first.
template <int PREC, int NDET, int WF>
__global__ void __launch_bounds__(kThreads) unit_likelihood_kernel(const EventDev* __restrict__ evp,
                                                                    const double* __restrict__ u, int n,
                                                                    double* __restrict__ lnl) {
  __shared__ WalkerParams P;
  __shared__ double red[kWarps][NVals<NDET, WF>::value];
  __shared__ double vals[kMaxVals];
  const EventDev& ev = *evp;
  const int w = blockIdx.x;
  if (threadIdx.x == 0) setup_from_unit<PREC, WF>(ev, u + (size_t)w * ev.n_dim, P);
  __syncthreads();
  if constexpr (PREC == 2) {
    if (ev.rb_nb > 0) {
      if (threadIdx.x < 32) {
        const double v = rb_lnl_warp<NDET, WF>(ev, P, threadIdx.x);
        if (threadIdx.x == 0) lnl[w] = isfinite(v) ? v : -INFINITY;
      }
      return;
    }
  }
  cta_sums<PREC, NDET, WF>(ev, P, red, vals);
  if (threadIdx.x == 0) {
    double v = lnl_from_vals<PREC, NDET, WF>(ev, P, vals);
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
template <int NDET, int WF>
__global__ void __launch_bounds__(256) waveform_kernel(const EventDev* __restrict__ evp,
                                                       const double* __restrict__ theta, int n_bins,
                                                       double* __restrict__ h_re, double* __restrict__ h_im,
                                                       int no_cutoff) {
  __shared__ WalkerParams P;
  const EventDev& ev = *evp;
  const int w = blockIdx.y;
  if (threadIdx.x == 0) {
    double th[kParams];
    for (int i = 0; i < kParams; ++i) th[i] = theta[(size_t)w * kParams + i];
    setup_from_theta<0, WF>(ev, th, P);
    if (no_cutoff) P.k_end = n_bins;
  }
  __syncthreads();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_bins) return;
  const double f = ev.f_min + ev.df * (double)k;
  double phi = 0.0, amp = 0.0;
  if (k < P.k_end) {
    const double* g = ev.basis64 + (size_t)k * ev.n_basis;
    if (WF == 0) {
      phi = P.phase0;
      for (int j = 0; j < kBasis; ++j) phi = fma(P.C[j], g[j], phi);
      amp = 1.0;
    } else {
      const PhenomExtra& e = P.pd;
      if (k < e.k1) {
        phi = P.phase0;
        for (int j = 0; j < kBasis; ++j) phi = fma(P.C[j], g[j], phi);
        phi = fma(e.Cx[0], g[8], fma(e.Cx[1], g[9], fma(e.Cx[2], g[10], phi)));
      } else if (k < e.k2) {
        phi = fma(e.Cx[3], g[6], fma(e.Cx[4], g[11], fma(e.Cx[5], g[13], e.ph0_int)));
      } else {
        phi = fma(e.Cx[6], g[1], fma(e.Cx[7], g[12], fma(e.Cx[8], g[13], e.ph0_mr)));
        phi += e.at_scale * atan((e.M * f - e.at_c) * e.at_inv);
      }
      amp = pd_amp_f64(e, k, f, g[4]);
    }
  }
  const double a7 = pow(f, -7.0 / 6.0) * amp;
#pragma unroll
  for (int det = 0; det < NDET; ++det) {
    double re = 0.0, im = 0.0;
    if (k < P.k_end) {
      double ph = fma(P.tau[det], f, phi);
      double r = ph - rint(ph);
      double s, c;
      sincospi(2.0 * r, &s, &c);
      // a f^-7/6 K P exp(-2 pi i r)
      re = a7 * (P.kp_re[det] * c + P.kp_im[det] * s);
      im = a7 * (P.kp_im[det] * c - P.kp_re[det] * s);
    }
    size_t o = ((size_t)w * NDET + det) * n_bins + k;
    h_re[o] = re;
    h_im[o] = im;
  }
}

// ---------------------------------------------------------------- acceptance walk
// Modes 0 and 1 (FP64 phase); mode 2 runs walk_kernel_ff below.
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
// Flow steps (task.flow set): a step whose Philox tag-6 draw falls below p_flow proposes the
// precomputed flow sample of the proposal table instead of a DE move, and passes the screen
// iff ln U < ln q(u) - ln q(u') (an independence Metropolis-Hastings test taken before the
// likelihood); ln q of the current point is carried along and re-evaluated on CUDA cores
// after an accepted DE move.
template <int PREC, int NDET, int WF>
__global__ void __launch_bounds__(kThreads, 4) walk_kernel(const EventDev* __restrict__ evs, WalkTask* tasks,
                                                         const int32_t* __restrict__ blk_task,
                                                         const int32_t* __restrict__ blk_local) {
  constexpr int NV = NVals<NDET, WF>::value;
  __shared__ WalkerParams P[kSpecMax];
  __shared__ double prop[kSpecMax][kMaxDim];
  __shared__ int cstep[kSpecMax];
  __shared__ int mstep[32];
  __shared__ double lnl_p[kSpecMax];
  __shared__ double tot_p[kSpecMax][NV];
  __shared__ double ct[kWarps][kWarps][NV];
  __shared__ double u[kMaxDim];
  __shared__ float u32[kMaxDim];
  __shared__ int wcount[kWarps];
  __shared__ int s_next, s_setup_warp, s_nin, s_end, s_needq;
  __shared__ int s_isflow[kSpecMax];
  __shared__ float s_lqf[kSpecMax];
  __shared__ float s_logq;
  __shared__ FlowScratch fscr;
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
  int n_acc = 0, n_acc_flow = 0, n_like = 0;
  int64_t n_bins = 0, n_spec = 0;
  const uint64_t t0 = threadIdx.x == 0 ? global_ns() : 0ull;
  const double de_scale = 2.38 / sqrt(2.0 * (double)D);
  const float de_scale32 = (float)de_scale;
  __syncthreads();
  const int sw = s_setup_warp;
  const bool use_flow = T.flow != nullptr && T.p_flow > 0.0;
  const double p_flow = T.p_flow;
  if (use_flow) {
    const float lq = flow_logq_cta(*T.flow, u, fscr);
    if (threadIdx.x == 0) s_logq = lq;
    __syncthreads();
  }
  int t = 0;
  while (t < n_steps) {
    const int abort_flag = threadIdx.x == 0 ? walk_abort_flag(T) : 0;
    const int W = min(window, n_steps - t);
    // 1a. every thread screens one candidate step in FP32
    int maybe = 0;
    const int step = t + (int)threadIdx.x;
    bool fl = false;
    if (use_flow && (int)threadIdx.x < W) {
      Philox4 C = philox4x64((uint64_t)step, wid, it, 6ull, T.key0, T.key1);
      if (rand_open_unit(C.v[0]) < p_flow) {
        fl = true;
        const float lqf = (float)T.flq[(size_t)j * T.f_stride + step];
        maybe = logf((float)rand_open_unit(C.v[1])) < s_logq - lqf;
      }
    }
    if ((int)threadIdx.x < W && !fl) {
      Philox4 A = philox4x64((uint64_t)step, wid, it, 0ull, T.key0, T.key1);
      uint64_t a = rand_index(A.v[0], n_s);
      uint64_t b = rand_index(A.v[1], n_s - 1);
      b += (b >= a) ? 1ull : 0ull;
      float sc = 1.0f;
      if ((A.v[2] >> 63) == 0ull) {
        Philox4 B = philox4x64((uint64_t)step, wid, it, 1ull, T.key0, T.key1);
        // log2 U_i = log2((x_i >> 12) + 1/2) - 52, each factor's integer rounded to float
        // (relative error ~1e-7, no truncation, no underflow of the product)
        float l2 = __log2f(top52_half_f(B.v[0])) + __log2f(top52_half_f(B.v[1])) + __log2f(top52_half_f(B.v[2])) +
                   __log2f(top52_half_f(B.v[3])) - 208.0f;
        sc = de_scale32 * (-0.25f * 0.6931471805599453f * l2);
      }
      // |x32 - x64| stays below ~1e-7 (1 + |s|) plus the log2 error times |s|: a margin of
      // 1e-5 (1 + |s|) never rejects a step that the exact FP64 test accepts
      const float margin = 1e-5f * (1.0f + fabsf(sc));
      maybe = 1;
      if (T.survf) {
        const float2* ua = T.survf + a * D;
        const float2* ub = T.survf + b * D;
#pragma unroll
        for (int d = 0; d < kMaxDim; ++d) {
          if (d < D && !ev.prior[ev.dim_param[d]].periodic) {
            float x = u32[d] + sc * (ua[d].x - ub[d].x);
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
      int in = 0, isf = 0;
      float lqf = 0.0f;
      double pr[kMaxDim];
      const int st = lane < nmaybe ? mstep[lane] : 0;
      if (use_flow && lane < nmaybe) {
        Philox4 C = philox4x64((uint64_t)st, wid, it, 6ull, T.key0, T.key1);
        if (rand_open_unit(C.v[0]) < p_flow) {
          isf = 1;
          lqf = (float)T.flq[(size_t)j * T.f_stride + st];
          in = logf((float)rand_open_unit(C.v[1])) < s_logq - lqf;
          const double* fu = T.fu + ((size_t)j * T.f_stride + st) * D;
#pragma unroll
          for (int d = 0; d < kMaxDim; ++d)
            if (d < D) pr[d] = fu[d];
        }
      }
      if (lane < nmaybe && !isf) {
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
        s_isflow[slot] = isf;
        s_lqf[slot] = lqf;
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
      if (lane < nin_w) setup_from_unit<PREC, WF>(ev, prop[lane], P[lane]);
    }
    __syncthreads();
    const int nin = s_nin;
    // 2. likelihoods: the sums of proposal i into tot_p[i] (chunk totals in ct), then one lane
    //    per proposal assembles ln L (the FP64 part runs once per proposal, on one warp)
    if (nin >= kWarps) {
      // one warp per proposal, its four chunks in turn
      for (int i = warp; i < nin; i += kWarps) {
        warp_chunks<PREC, NDET, WF>(ev, P[i], lane, ct[warp]);
        if (lane < NV) tot_p[i][lane] = chunks_sum<NV>(ct[warp], lane);
        __syncwarp();
      }
    } else {
      // fewer proposals than warps: the whole CTA on each in turn, chunk w on warp w
      for (int i = 0; i < nin; ++i) {
        double dv[NV];
        float fv[NV], fc[NV];
        partials<PREC, NDET, WF>(ev, P[i], threadIdx.x, kThreads, dv, fv, fc);
        chunk_total<PREC, NV>(dv, fv, fc, lane, ct[0][warp]);
        __syncthreads();
        if (threadIdx.x < NV) tot_p[i][threadIdx.x] = chunks_sum<NV>(ct[0], threadIdx.x);
        __syncthreads();
      }
    }
    __syncthreads();
    if (warp == sw && lane < nin) lnl_p[lane] = lnl_from_vals<PREC, NDET, WF>(ev, P[lane], tot_p[lane]);
    __syncthreads();
    // 3. the steps in order
    if (threadIdx.x == 0) {
      int nxt = s_end + 1;
      s_needq = 0;
      for (int i = 0; i < nin; ++i) {
        ++n_like;
        n_bins += P[i].k_end;
        if (lnl_p[i] > lnl_star) {
          for (int d = 0; d < D; ++d) { u[d] = prop[i][d]; u32[d] = (float)prop[i][d]; }
          lnl = lnl_p[i];
          ++n_acc;
          nxt = cstep[i] + 1;
          if (use_flow) {
            if (s_isflow[i]) {
              s_logq = s_lqf[i];
              ++n_acc_flow;
            } else {
              s_needq = 1;
            }
          }
          break;
        }
      }
      n_spec += nin;
      if (walk_should_stop(T, t0, abort_flag)) {   // watchdog: end the walk after this round
        nxt = n_steps;
        if (T.status) atomicOr(T.status, 1);
      }
      s_next = nxt;
    }
    __syncthreads();
    t = s_next;
    if (use_flow && s_needq && t < n_steps) {
      const float lq = flow_logq_cta(*T.flow, u, fscr);
      if (threadIdx.x == 0) s_logq = lq;
      __syncthreads();
    }
  }
  if (threadIdx.x < D) T.u_out[(size_t)j * D + threadIdx.x] = u[threadIdx.x];
  if (threadIdx.x == 0) {
    T.lnl_out[j] = lnl;
    T.n_acc[j] = n_acc;
    if (T.n_acc_flow) T.n_acc_flow[j] = n_acc_flow;
    T.n_like[j] = n_like;
    if (T.n_bins) T.n_bins[j] = n_bins;
    if (T.n_spec) T.n_spec[j] = n_spec;
  }
}

// ---------------------------------------------------------------- float-float walk (mode 2)
__device__ __forceinline__ bool ff_in_unit(ff x) {
  // x normalised (|l| <= ulp(h) / 2, so h = 0 implies l = 0); NaN fails the first test
  return x.h >= 0.0f && (x.h < 1.0f || (x.h == 1.0f && x.l <= 0.0f));
}
// x - floor(x) of a float-float value (the periodic dimensions).
__device__ __forceinline__ ff ff_wrap_unit(ff x) {
  float fl = floorf(x.h);
  if (x.h == fl && x.l < 0.0f) fl -= 1.0f;
  return ff_add_f(x, -fl);
}

// The acceptance walk of mode 2.  The round of walk_kernel, restructured so that its serial
// part is short:
//  1. every thread forms the move of one candidate step of the window exactly, in float-float
//     arithmetic (the DE scale's logarithm, the survivors' float-float difference, the periodic
//     wrap, the bounds test) -- there is no FP32 screen and no one-warp recheck -- and a ballot
//     compacts the first m in-bounds moves;
//  2. the proposal constants of the round run on all four warps at once (tf2_split_first /
//     tf2_split_second, pd_split_first / pd_split_second: independent chains, then the
//     products; the IMRPhenomD form's continuity constants and its region boundaries and
//     amplitude shape on different warps);
//  3. the likelihoods: TaylorF2 one warp per proposal, the IMRPhenomD form the whole CTA per
//     proposal;
//  4. warp 0 assembles ln L of every proposal in float-float and finds the first acceptance
//     with one ballot.
// The DE move is the walk's, u' = u + gamma (u_a - u_b), with the position and the survivors as
// float pairs (~48 significant bits): the chain is the FP64 chain up to rounding at ~1e-14.
// A TaylorF2 round is padded to a multiple of four proposals: its warp-per-proposal likelihood
// phase takes as long for 1 or 5 proposals as for 4 or 8, and the padding only advances the
// chain further.  The IMRPhenomD form (thousands of bins a proposal) runs each proposal on the
// whole CTA instead.
template <int NDET, int WF, bool XF>
__global__ void __launch_bounds__(kThreads, 4) walk_kernel_ff(const EventDev* __restrict__ evs, WalkTask* tasks,
                                                            const int32_t* __restrict__ blk_task,
                                                            const int32_t* __restrict__ blk_local) {
  constexpr int NV = NVals<NDET, WF>::value;
  __shared__ WalkerParams P[kSpecMax];
  __shared__ ff propf[kSpecMax][kMaxDim];
  __shared__ std::conditional_t<WF == 0, TF2Part, PDPart> parts[kSpecMax];
  __shared__ int cstep[kSpecMax];
  __shared__ float part_sums[kSpecMax][2 * kMaxVals];
  __shared__ double s_rbl[kSpecMax];   // relative binning: ln L of each proposal
  __shared__ int s_rbk[kSpecMax];      // and the grid bins it touched
  // IMRPhenomD form: every warp's compensated sums of every proposal
  __shared__ float wsums[WF == 1 ? kSpecMax : 1][kWarps][2 * kMaxVals];
  __shared__ double u[kMaxDim];
  __shared__ ff uf[kMaxDim];
  __shared__ int wcount[kWarps];
  __shared__ int s_next, s_setup_warp, s_end, s_needq;
  __shared__ int s_isflow[kSpecMax];
  __shared__ float s_lqf[kSpecMax];
  __shared__ float s_logq;
  __shared__ FlowScratch fscr;
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
  int m = T.spec < 1 ? 1 : (T.spec > kSpecMax ? kSpecMax : T.spec);
  if (WF == 0) m = min((m + 3) & ~3, kSpecMax);
  const int window = min(kThreads, max(32, 4 * m));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool split = ev.ff_setup;
  if (threadIdx.x < D) {
    const double v = T.u0[(size_t)j * D + threadIdx.x];
    u[threadIdx.x] = v;
    uf[threadIdx.x] = ff_from_double(v);
  }
  if (threadIdx.x == 0) {
    unsigned int smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    s_setup_warp = (int)(atomicAdd(&g_walk_sm_arrivals[smid & 255u], 1u) % (unsigned)kWarps);
  }
  unsigned periodic = 0u;
#pragma unroll
  for (int d = 0; d < kMaxDim; ++d)
    if (d < D && ev.prior[ev.dim_param[d]].periodic) periodic |= 1u << d;
  double lnl = T.lnl0[j];
  int n_acc = 0, n_acc_flow = 0, n_like = 0;
  int64_t n_bins = 0, n_spec = 0;
  const uint64_t t0 = threadIdx.x == 0 ? global_ns() : 0ull;
  const ff de_scale = ff_from_double(2.38 / sqrt(2.0 * (double)D));
  __syncthreads();
  const int sw = s_setup_warp;
  const bool use_flow = XF && T.flow != nullptr && T.p_flow > 0.0;
  const double p_flow = T.p_flow;
  if (use_flow) {
    const float lq = flow_logq_cta(*T.flow, u, fscr);
    if (threadIdx.x == 0) s_logq = lq;
    __syncthreads();
  }
  int t = 0;
  while (t < n_steps) {
    const int abort_flag = threadIdx.x == 0 ? walk_abort_flag(T) : 0;
    const int W = min(window, n_steps - t);
    // 1. the exact move of one candidate step per thread
    const int step = t + (int)threadIdx.x;
    int in = 0, isf = 0;
    float lqf = 0.0f;
    ff xf[kMaxDim];
    if ((int)threadIdx.x < W) {
      // the step's Philox blocks: (tag 6: flow coin,) tag 0: survivors and scale coin,
      // tag 1: the scale's uniforms -- one inlined generator, called up to three times
      Philox4 A, B;
      bool draw_scale = false;
      int tag = use_flow ? 6 : 0;
#pragma unroll 1
      while (tag >= 0) {
        const Philox4 r = philox4x64((uint64_t)step, wid, it, (uint64_t)tag, T.key0, T.key1);
        if (tag == 6) {
          tag = 0;
          if (rand_open_unit(r.v[0]) < p_flow) {
            isf = 1;
            lqf = (float)T.flq[(size_t)j * T.f_stride + step];
            in = logf((float)rand_open_unit(r.v[1])) < s_logq - lqf;
            tag = -1;
          }
        } else if (tag == 0) {
          A = r;
          draw_scale = (r.v[2] >> 63) == 0ull;
          tag = draw_scale ? 1 : -1;
        } else {
          B = r;
          tag = -1;
        }
      }
      if (isf) {
        if (in) {
          const double* fu = T.fu + ((size_t)j * T.f_stride + step) * D;
#pragma unroll
          for (int d = 0; d < kMaxDim; ++d)
            if (d < D) xf[d] = ff_from_double(fu[d]);
        }
      } else {
        const uint64_t a = rand_index(A.v[0], n_s);
        uint64_t b = rand_index(A.v[1], n_s - 1);
        b += (b >= a) ? 1ull : 0ull;
        // both survivors' coordinates first (branch-free, all loads in flight at once)
        ff ua[kMaxDim], ub[kMaxDim];
        if (T.survf) {
#pragma unroll
          for (int d = 0; d < kMaxDim; ++d) {
            const int dd = d < D ? d : D - 1;
            const float2 pa = T.survf[a * D + dd], pb = T.survf[b * D + dd];
            ua[d] = ff{pa.x, pa.y};
            ub[d] = ff{pb.x, pb.y};
          }
        } else {
#pragma unroll
          for (int d = 0; d < kMaxDim; ++d) {
            const int dd = d < D ? d : D - 1;
            ua[d] = ff_from_double(T.surv[a * D + dd]);
            ub[d] = ff_from_double(T.surv[b * D + dd]);
          }
        }
        const ff sc = draw_scale ? ff_mul(ff_mul_f(ff_log_uniform_product(B.v), -0.25f), de_scale) : ff_make(1.0f);
        in = 1;
#pragma unroll
        for (int d = 0; d < kMaxDim; ++d) {
          ff x = ff_add(uf[d < D ? d : D - 1], ff_mul(sc, ff_sub(ua[d], ub[d])));
          const ff xw = ff_wrap_unit(x);
          if ((periodic >> d) & 1u) x = xw;
          if (d < D && !ff_in_unit(x)) in = 0;
          xf[d] = x;
        }
      }
    }
    const unsigned mask = __ballot_sync(0xffffffffu, in);
    if (lane == 0) wcount[warp] = __popc(mask);
    __syncthreads();
    int before = 0, total = 0;
#pragma unroll
    for (int w2 = 0; w2 < kWarps; ++w2) {
      const int cw = wcount[w2];
      before += (w2 < warp) ? cw : 0;
      total += cw;
    }
    const int slot = before + __popc(mask & ((1u << lane) - 1u));
    if (in && slot < m) {
#pragma unroll
      for (int d = 0; d < kMaxDim; ++d)
        if (d < D) propf[slot][d] = xf[d];
      cstep[slot] = step;
      s_isflow[slot] = isf;
      s_lqf[slot] = lqf;
      // the round covers the steps up to the m-th in-bounds one, else the whole window
      if (slot == m - 1 && total > m) s_end = step;
    }
    if (threadIdx.x == 0 && total <= m) s_end = t + W - 1;
    const int nin = min(total, m);
    __syncthreads();
    // 2. proposal constants
    if (nin > 0) {
      if (split) {
        if (lane < nin) {
          if constexpr (WF == 0) tf2_split_first(warp, ev, propf[lane], parts[lane], P[lane]);
          else pd_split_first(warp, ev, propf[lane], parts[lane], P[lane]);
        }
        __syncthreads();
        if (lane < nin) {
          if constexpr (WF == 0) tf2_split_second(warp, ev, parts[lane], P[lane]);
          else pd_split_second(warp, ev, parts[lane], P[lane]);
        }
      } else if (warp == sw && lane < nin) {
        if (ev.ff_setup) {
          if (WF == 0) taylorf2_setup_ff(ev, propf[lane], P[lane]);
          else phenomd_setup_ff(ev, propf[lane], P[lane]);
        } else {
          double pd[kMaxDim];
#pragma unroll
          for (int d = 0; d < kMaxDim; ++d) pd[d] = d < D ? (double)propf[lane][d].h + (double)propf[lane][d].l : 0.0;
          setup_from_unit<2, WF>(ev, pd, P[lane]);
        }
      }
      __syncthreads();
    }
    // 3. likelihoods
    constexpr int V = Pow2Vals<NV>::value;
    constexpr int group = 32 / V;
    const bool rb = XF && ev.rb_nb > 0;
    if (rb) {
      // relative binning (~10^2 coarse-bin edges a proposal): a warp per proposal
      for (int i = warp; i < nin; i += kWarps) {
        int nk;
        const double v = rb_lnl_warp<NDET, WF>(ev, P[i], lane, &nk);
        if (lane == 0) { s_rbl[i] = v; s_rbk[i] = nk; }
      }
      __syncthreads();
    } else if (WF == 1) {
      // IMRPhenomD form (thousands of bins a proposal): the whole CTA on each proposal in turn,
      // so that proposals of different lengths leave no warp waiting; warp 0 combines the four
      // warps' compensated sums below
      for (int i = 0; i < nin; ++i) {
        double dv[NV];
        float fv[NV], fc[NV];
        partials<2, NDET, WF>(ev, P[i], threadIdx.x, kThreads, dv, fv, fc);
        float rs, rc;
        int q;
        warp_halving_sums<NV>(fv, fc, lane, rs, rc, q);
        if ((lane & (group - 1)) == 0 && q < NV) { wsums[i][warp][2 * q] = rs; wsums[i][warp][2 * q + 1] = rc; }
      }
      __syncthreads();
    } else {
      for (int i = warp; i < nin; i += kWarps) {
        double dv[NV];
        float fv[NV], fc[NV];
        partials<2, NDET, WF>(ev, P[i], lane, 32, dv, fv, fc);
        float rs, rc;
        int q;
        warp_halving_sums<NV>(fv, fc, lane, rs, rc, q);
        if ((lane & (group - 1)) == 0 && q < NV) { part_sums[i][2 * q] = rs; part_sums[i][2 * q + 1] = rc; }
      }
      __syncthreads();
    }
    // 4. ln L of every proposal, then the steps in order: the first acceptance ends the round
    if (warp == 0) {
      double l = 0.0;
      if (lane < nin) {
        if (rb) {
          l = s_rbl[lane];
        } else if (WF == 1) {
          // (s, c) of the four warps, summed with error-free additions
          float ps[2 * NV];
#pragma unroll
          for (int q = 0; q < NV; ++q) {
            float sh = wsums[lane][0][2 * q], sl = wsums[lane][0][2 * q + 1];
#pragma unroll
            for (int w2 = 1; w2 < kWarps; ++w2) {
              float t, e;
              two_sum(sh, wsums[lane][w2][2 * q], t, e);
              sh = t;
              sl += wsums[lane][w2][2 * q + 1] + e;
            }
            ps[2 * q] = sh;
            ps[2 * q + 1] = sl;
          }
          l = lnl_ff<NDET, WF>(ev, P[lane], ps);
        } else {
          l = lnl_ff<NDET, WF>(ev, P[lane], part_sums[lane]);
        }
      }
      const unsigned am = __ballot_sync(0xffffffffu, lane < nin && l > lnl_star);
      const int c = am ? __ffs(am) - 1 : -1;
      const int used = c >= 0 ? c + 1 : nin;
      int kb = lane < used ? (rb ? s_rbk[lane] : P[lane].k_end) : 0;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) kb += __shfl_xor_sync(0xffffffffu, kb, off);
      if (c >= 0) {
        lnl = __shfl_sync(0xffffffffu, l, c);
        if (lane < D) {
          const ff x = propf[c][lane];
          uf[lane] = x;
          u[lane] = (double)x.h + (double)x.l;
        }
      }
      if (lane == 0) {
        n_like += used;
        n_bins += kb;
        n_spec += nin;
        int nxt = s_end + 1;
        s_needq = 0;
        if (c >= 0) {
          ++n_acc;
          nxt = cstep[c] + 1;
          if (use_flow) {
            if (s_isflow[c]) {
              s_logq = s_lqf[c];
              ++n_acc_flow;
            } else {
              s_needq = 1;
            }
          }
        }
        if (walk_should_stop(T, t0, abort_flag)) {   // watchdog: end the walk after this round
          nxt = n_steps;
          if (T.status) atomicOr(T.status, 1);
        }
        s_next = nxt;
      }
    }
    __syncthreads();
    t = s_next;
    if (use_flow && s_needq && t < n_steps) {
      const float lq = flow_logq_cta(*T.flow, u, fscr);
      if (threadIdx.x == 0) s_logq = lq;
      __syncthreads();
    }
  }
  if (threadIdx.x < D) T.u_out[(size_t)j * D + threadIdx.x] = u[threadIdx.x];
  if (threadIdx.x == 0) {
    T.lnl_out[j] = lnl;
    T.n_acc[j] = n_acc;
    if (T.n_acc_flow) T.n_acc_flow[j] = n_acc_flow;
    T.n_like[j] = n_like;
    if (T.n_bins) T.n_bins[j] = n_bins;
    if (T.n_spec) T.n_spec[j] = n_spec;
  }
}

// ---------------------------------------------------------------- hit-and-run slice sampling
// Any precision.  One CTA per walker (block b: walker blk_local[b] of task blk_task[b]); thread 0
// runs each move's slice logic and the whole CTA evaluates every in-bounds candidate's ln L (the
// likelihood of the handle's precision; relative binning on warp 0 when the event uses it).  A
// move (Neal 2003, stepping out and shrinkage, along a random line): direction d = C z / |z|
// (z standard normal, C = task.chol, the Cholesky factor of the survivors' covariance), bracket
// [lo, lo + 1] with lo = -U, stepping out by one unit at a time with a budget of kHrssMaxOut - 1
// split as J = floor(kHrssMaxOut V) to the left and the rest to the right while the bracket's
// end is inside the slice, then shrinkage draws until a point inside the slice (at most
// kHrssMaxShrink; then the walker stays).  A candidate outside the cube costs no likelihood
// call; periodic coordinates wrap.  Philox blocks (step, walker, iteration, tag): tags 32 + c
// the normals (Box-Muller on words (0, 1) and (2, 3)), 40 the bracket (U, V), 48 + j / 4 word
// j % 4 the j-th shrinkage uniform.  task.n_steps moves; n_acc receives the moves made,
// n_like the likelihood calls; the watchdog (task.abort, task.budget_ns) is checked before
// every move.
constexpr int kHrssMaxOut = 10;
constexpr int kHrssMaxShrink = 100;

template <int PREC, int NDET, int WF>
__global__ void __launch_bounds__(kThreads) hrss_kernel(const EventDev* __restrict__ evs, WalkTask* tasks,
                                                         const int32_t* __restrict__ blk_task,
                                                         const int32_t* __restrict__ blk_local) {
  __shared__ WalkerParams P;
  __shared__ double red[kWarps][NVals<NDET, WF>::value];
  __shared__ double vals[kMaxVals];
  __shared__ double x[kMaxDim], dvec[kMaxDim], pt[kMaxDim];
  __shared__ double s_rbl;
  __shared__ int s_eval, s_end, s_stop, s_rbk;
  const WalkTask& T = tasks[blk_task[blockIdx.x]];
  const int j = blk_local[blockIdx.x];
  const EventDev& ev = evs[T.event];
  if (T.done) return;
  const int D = ev.n_dim;
  const int n_steps = T.n_steps;
  const double lnl_star = T.lnl_star;
  const uint64_t it = (uint64_t)T.iteration;
  const uint64_t wid = (uint64_t)(T.walker_offset + j);
  const double* chol = T.chol;
  bool rb = false;
  if constexpr (PREC == 2) rb = ev.rb_nb > 0;
  if ((int)threadIdx.x < D) x[threadIdx.x] = T.u0[(size_t)j * D + threadIdx.x];
  double lnl = T.lnl0[j];
  int moves = 0, calls = 0;
  int64_t n_bins = 0;
  const uint64_t t0 = threadIdx.x == 0 ? global_ns() : 0ull;
  // thread 0's state of the current move: phase 0 steps out left, 1 right, 2 shrinks
  double lo = 0.0, hi = 0.0, tc = 0.0;
  int phase = 2, jl = 0, kr = 0, nsh = 0;
  __syncthreads();
  for (int t = 0; t < n_steps; ++t) {
    if (threadIdx.x == 0) {
      s_stop = walk_should_stop(T, t0, walk_abort_flag(T)) ? 1 : 0;
      if (s_stop && T.status) atomicOr(T.status, 1);
      double z[kMaxDim];
      for (int c = 0; 4 * c < D; ++c) {
        const Philox4 b = philox4x64((uint64_t)t, wid, it, 32ull + (uint64_t)c, T.key0, T.key1);
        for (int q = 0; q < 2; ++q) {
          const double r = sqrt(-2.0 * log(rand_open_unit(b.v[2 * q])));
          double sn, cs;
          sincospi(2.0 * rand_open_unit(b.v[2 * q + 1]), &sn, &cs);
          const int i0 = 4 * c + 2 * q;
          if (i0 < D) z[i0] = r * cs;
          if (i0 + 1 < D) z[i0 + 1] = r * sn;
        }
      }
      double nz = 0.0;
      for (int i = 0; i < D; ++i) nz += z[i] * z[i];
      nz = sqrt(nz);
      for (int i = 0; i < D; ++i) {
        double acc = 0.0;
        for (int k = 0; k <= i; ++k) acc += chol[i * D + k] * z[k];
        dvec[i] = acc / nz;
      }
      const Philox4 b = philox4x64((uint64_t)t, wid, it, 40ull, T.key0, T.key1);
      lo = -rand_open_unit(b.v[0]);
      hi = lo + 1.0;
      jl = (int)floor((double)kHrssMaxOut * rand_open_unit(b.v[1]));
      kr = kHrssMaxOut - 1 - jl;
      nsh = 0;
      phase = jl > 0 ? 0 : (kr > 0 ? 1 : 2);
    }
    __syncthreads();
    if (s_stop) break;
    // step-out evaluations <= kHrssMaxOut - 1, shrinkage draws <= kHrssMaxShrink
    for (int iter = 0; iter < kHrssMaxOut + kHrssMaxShrink; ++iter) {
      if (threadIdx.x == 0) {
        if (phase == 0) {
          tc = lo;
        } else if (phase == 1) {
          tc = hi;
        } else {
          const Philox4 b = philox4x64((uint64_t)t, wid, it, 48ull + (uint64_t)(nsh >> 2), T.key0, T.key1);
          tc = lo + (hi - lo) * rand_open_unit(b.v[nsh & 3]);
        }
        int inb = 1;
        for (int i = 0; i < D; ++i) {
          double v = x[i] + tc * dvec[i];
          if (ev.prior[ev.dim_param[i]].periodic) v -= floor(v);
          pt[i] = v;
          if (!(v >= 0.0 && v <= 1.0)) inb = 0;
        }
        s_eval = inb;
        if (inb) setup_from_unit<PREC, WF>(ev, pt, P);
      }
      __syncthreads();
      const int evaluate = s_eval;
      if (evaluate) {
        if (rb) {
          if constexpr (PREC == 2) {
            if (threadIdx.x < 32) {
              int kb = 0;
              const double v = rb_lnl_warp<NDET, WF>(ev, P, threadIdx.x, &kb);
              if (threadIdx.x == 0) { s_rbl = v; s_rbk = kb; }
            }
            __syncthreads();
          }
        } else {
          cta_sums<PREC, NDET, WF>(ev, P, red, vals);
        }
      }
      if (threadIdx.x == 0) {
        bool ins = false;
        double l = 0.0;
        if (evaluate) {
          l = rb ? s_rbl : lnl_from_vals<PREC, NDET, WF>(ev, P, vals);
          ++calls;
          n_bins += rb ? s_rbk : P.k_end;
          ins = l > lnl_star;
        }
        int end = 0;
        if (phase == 0) {
          if (ins) { lo -= 1.0; --jl; }
          if (!ins || jl == 0) phase = kr > 0 ? 1 : 2;
        } else if (phase == 1) {
          if (ins) { hi += 1.0; --kr; }
          if (!ins || kr == 0) phase = 2;
        } else if (ins) {
          for (int i = 0; i < D; ++i) x[i] = pt[i];
          lnl = l;
          ++moves;
          end = 1;
        } else {
          if (tc < 0.0) lo = tc;
          else hi = tc;
          if (++nsh == kHrssMaxShrink) end = 1;
        }
        s_end = end;
      }
      __syncthreads();
      if (s_end) break;
    }
  }
  if ((int)threadIdx.x < D) T.u_out[(size_t)j * D + threadIdx.x] = x[threadIdx.x];
  if (threadIdx.x == 0) {
    T.lnl_out[j] = lnl;
    T.n_acc[j] = moves;
    T.n_like[j] = calls;
    if (T.n_bins) T.n_bins[j] = n_bins;
    if (T.n_spec) T.n_spec[j] = calls;
  }
}

// ---------------------------------------------------------------- speculative HRSS (mode 2)
// The slice-sampling moves of hrss_kernel, with the candidate evaluations of a move batched into
// rounds that run like the float-float walk's: the candidates' points in FP64 on warp 0 (one lane
// each), their constants on the setup warps, their likelihoods one warp per candidate (TaylorF2,
// relative binning) or on the whole CTA in turn (IMRPhenomD form), then thread 0 replays the
// sequential slice logic over them in order.  Which candidates the sequential move evaluates
// next depends on outcomes only through where it stops:
//   stepping out: the left end is tried at lo, lo - 1, lo - 2, ... while it is inside the slice
//     (budget J) and the right end at hi, hi + 1, ... (budget K); a round holds the next ends of
//     both sides, as if every one were inside, and the replay stops each side at its first end
//     outside the slice (the two sides do not interact, so their order does not matter);
//   shrinkage: with the draws U_j fixed by their Philox counters, the j-th candidate is
//     t_j = lo_j + (hi_j - lo_j) U_j, where (lo_j, hi_j) is the bracket left by rejecting
//     t_1 .. t_{j-1}; a round holds the next candidates as if all were rejected, and the replay
//     takes the first inside the slice.
// A stepping-out round holds up to max(1, spec/4) ends a side and fills the rest of the round
// with the first shrinkage candidates of the bracket as it stands: they are the move's next
// candidates exactly when every side still extending stops at its first end in the round, and
// the replay uses them only then -- a move whose bracket does not grow ends in one round.
// The chain, the moves and the likelihood-call counts are those of the one-candidate kernel (calls
// of candidates after the replay's stopping point are counted in n_spec only); per round at most
// task.spec candidates (1 .. kHrssQ).  Directions do not depend on the walker's position: the
// whole CTA forms those of 32 moves at a time (Box-Muller on the Philox blocks of hrss_kernel,
// d = C z / |z| row by row in the same order).
constexpr int kHrssQ = 16;

template <int NDET, int WF>
__global__ void __launch_bounds__(kThreads, 4) hrss_kernel_ff(const EventDev* __restrict__ evs, WalkTask* tasks,
                                                             const int32_t* __restrict__ blk_task,
                                                             const int32_t* __restrict__ blk_local) {
  constexpr int NV = NVals<NDET, WF>::value;
  __shared__ WalkerParams P[kHrssQ];
  __shared__ ff propf[kHrssQ][kMaxDim];
  __shared__ std::conditional_t<WF == 0, TF2Part, PDPart> parts[kHrssQ];
  __shared__ float part_sums[kHrssQ][2 * kMaxVals];
  __shared__ float wsums[WF == 1 ? kHrssQ : 1][kWarps][2 * kMaxVals];
  __shared__ double s_rbl[kHrssQ];
  __shared__ int s_rbk[kHrssQ];
  __shared__ double x[kMaxDim];
  __shared__ double zn_all[32][kMaxDim + 1];     // normals of the next 32 moves
  __shared__ double dir_all[32][kMaxDim];        // their directions d = C z / |z|
  __shared__ double ct[kHrssQ];              // t of each candidate of the round, in evaluation order
  __shared__ double cpt[kHrssQ][kMaxDim];    // its point
  __shared__ ff cf[kHrssQ][kMaxDim];         // the point as float pairs
  __shared__ double s_u[kHrssQ];             // the round's shrinkage draws
  __shared__ int s_oob[kHrssQ];              // the point lies outside the cube
  __shared__ int ins_c[kHrssQ];              // each slot's ln L exceeds ln L*
  __shared__ int cslot[kHrssQ];              // its likelihood slot, -1 for a point outside the cube
  __shared__ double lnl_c[kHrssQ];           // ln L of each slot
  __shared__ int kend_c[kHrssQ];             // grid bins each slot's evaluation touched
  __shared__ int s_nc, s_nin, s_newmove, s_exit, s_t, s_mode, s_nsh;
  const WalkTask& T = tasks[blk_task[blockIdx.x]];
  const int j = blk_local[blockIdx.x];
  const EventDev& ev = evs[T.event];
  if (T.done) return;
  const int D = ev.n_dim;
  const int n_steps = T.n_steps;
  const double lnl_star = T.lnl_star;
  const uint64_t it = (uint64_t)T.iteration;
  const uint64_t wid = (uint64_t)(T.walker_offset + j);
  const double* chol = T.chol;
  const int Q = T.spec < 1 ? 1 : (T.spec > kHrssQ ? kHrssQ : T.spec);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool split = ev.ff_setup;
  const bool rb = ev.rb_nb > 0;
  const int sw = (int)(blockIdx.x % (unsigned)kWarps);   // the setup warp of the non-split setups
  if ((int)threadIdx.x < D) x[threadIdx.x] = T.u0[(size_t)j * D + threadIdx.x];
  double lnl = T.lnl0[j];
  int moves = 0, calls = 0;
  int64_t n_bins = 0, n_spec = 0;
  const uint64_t t0 = threadIdx.x == 0 ? global_ns() : 0ull;
  // thread 0's move state: t the move, stepping (the bracket's ends still extend: jl, kr left),
  // lo, hi the bracket, nsh shrinkage draws used
  int t = 0, jl = 0, kr = 0, nsh = 0;
  bool left_on = false, right_on = false;
  double lo = 0.0, hi = 0.0;
  if (threadIdx.x == 0) {
    s_exit = n_steps <= 0 ? 1 : 0;
    s_newmove = 1;
    s_t = 0;
  }
  __syncthreads();
  while (!s_exit) {
    // A1. the directions of the next 32 moves, on the whole CTA, when a block of moves begins:
    //     a direction depends on its move's Philox counter only, not on the walker's position
    if (s_newmove && (s_t & 31) == 0) {
      const int base = s_t, nm = min(32, n_steps - base), nb = (D + 3) / 4;
      for (int q = threadIdx.x; q < nm * nb; q += kThreads) {
        const int mv = q / nb, c = q - mv * nb;
        const Philox4 b = philox4x64((uint64_t)(base + mv), wid, it, 32ull + (uint64_t)c, T.key0, T.key1);
        for (int h = 0; h < 2; ++h) {
          const double r = sqrt(-2.0 * log(rand_open_unit(b.v[2 * h])));
          double sn, cs;
          sincospi(2.0 * rand_open_unit(b.v[2 * h + 1]), &sn, &cs);
          const int i0 = 4 * c + 2 * h;
          if (i0 < D) zn_all[mv][i0] = r * cs;
          if (i0 + 1 < D) zn_all[mv][i0 + 1] = r * sn;
        }
      }
      __syncthreads();
      for (int q = threadIdx.x; q < nm * D; q += kThreads) {
        const int mv = q / D, i = q - mv * D;
        double nz = 0.0;
        for (int k = 0; k < D; ++k) nz += zn_all[mv][k] * zn_all[mv][k];
        nz = sqrt(nz);
        double acc = 0.0;
        for (int k = 0; k <= i; ++k) acc += chol[i * D + k] * zn_all[mv][k];
        dir_all[mv][i] = acc / nz;
      }
      __syncthreads();
    }
    // A2. warp 0: a new move's bracket; the round's candidates (shrinkage draws on the lanes) and
    //     their points ((candidate, coordinate) pairs over the lanes)
    if (warp == 0) {
      const int tm = s_t;
      const double* dv = dir_all[tm & 31];
      if (lane == 0) {
        if (s_newmove) {
          const Philox4 b = philox4x64((uint64_t)t, wid, it, 40ull, T.key0, T.key1);
          lo = -rand_open_unit(b.v[0]);
          hi = lo + 1.0;
          jl = (int)floor((double)kHrssMaxOut * rand_open_unit(b.v[1]));
          kr = kHrssMaxOut - 1 - jl;
          nsh = 0;
          left_on = jl > 0;
          right_on = kr > 0;
        }
        int ql = 0, qr = 0, S;
        if (left_on || right_on) {
          // stepping out: up to max(1, Q/4) next ends a side, the rest of the round's candidates
          // the shrinkage draws from the current bracket, which hold if every side still extending
          // stops at its first end in this round
          const int qs = max(1, Q / 4);
          ql = left_on ? min(jl, qs) : 0;
          qr = right_on ? min(kr, qs) : 0;
          if (ql + qr > Q) qr = Q - ql;
          S = min(Q - ql - qr, kHrssMaxShrink - nsh);
        } else {
          S = min(Q, kHrssMaxShrink - nsh);
        }
        s_mode = S;
        s_nsh = nsh;
        s_nc = (ql << 8) | (qr << 16);
      }
      __syncwarp();
      const int S = s_mode;
      if (lane < S) {
        const int jj = s_nsh + lane;
        const Philox4 b = philox4x64((uint64_t)tm, wid, it, 48ull + (uint64_t)(jj >> 2), T.key0, T.key1);
        s_u[lane] = rand_open_unit(b.v[jj & 3]);
      }
      __syncwarp();
      if (lane == 0) {
        int nc = 0;
        if (left_on || right_on) {
          // the next ends of both sides, as if every one were inside the slice, then the
          // shrinkage candidates of the bracket as it stands, as if each were rejected
          const int ql = (s_nc >> 8) & 255, qr = (s_nc >> 16) & 255;
          for (int i = 0; i < ql; ++i) ct[nc++] = lo - (double)i;
          for (int i = 0; i < qr; ++i) ct[nc++] = hi + (double)i;
          double l2 = lo, h2 = hi;
          for (int q = 0; q < S; ++q) {
            const double tc = l2 + (h2 - l2) * s_u[q];
            ct[nc++] = tc;
            if (tc < 0.0) l2 = tc;
            else h2 = tc;
          }
          s_nc = nc | (ql << 8) | (qr << 16);
        } else {
          // the next shrinkage candidates, as if every one were rejected
          double l2 = lo, h2 = hi;
          for (int q = 0; q < S; ++q) {
            const double tc = l2 + (h2 - l2) * s_u[q];
            ct[nc++] = tc;
            if (tc < 0.0) l2 = tc;
            else h2 = tc;
          }
          s_nc = nc;
        }
      }
      __syncwarp();
      const int nc = s_nc & 255;
      if (lane < nc) s_oob[lane] = 0;
      __syncwarp();
      for (int q = lane; q < nc * D; q += 32) {
        const int c = q / D, i = q - c * D;
        double v = x[i] + ct[c] * dv[i];
        if (ev.prior[ev.dim_param[i]].periodic) v -= floor(v);
        cpt[c][i] = v;
        cf[c][i] = ff_from_double(v);
        if (!(v >= 0.0 && v <= 1.0)) atomicOr(&s_oob[c], 1);
      }
      __syncwarp();
      const int inb = (lane < nc && s_oob[lane] == 0) ? 1 : 0;
      const unsigned im = __ballot_sync(0xffffffffu, inb);
      if (lane < nc) cslot[lane] = inb ? __popc(im & ((1u << lane) - 1u)) : -1;
      if (lane == 0) s_nin = __popc(im);
      __syncwarp();
      // the in-cube candidates' coordinates in slot order
      for (int q = lane; q < nc * kMaxDim; q += 32) {
        const int c = q / kMaxDim, d = q - c * kMaxDim;
        const int sl = cslot[c];
        if (sl >= 0) propf[sl][d] = d < D ? cf[c][d] : ff_make(0.0f);
      }
    }
    __syncthreads();
    const int nin = s_nin;
    // B. the candidates' constants
    if (nin > 0) {
      if (split) {
        if (lane < nin) {
          if constexpr (WF == 0) tf2_split_first(warp, ev, propf[lane], parts[lane], P[lane]);
          else pd_split_first(warp, ev, propf[lane], parts[lane], P[lane]);
        }
        __syncthreads();
        if (lane < nin) {
          if constexpr (WF == 0) tf2_split_second(warp, ev, parts[lane], P[lane]);
          else pd_split_second(warp, ev, parts[lane], P[lane]);
        }
      } else if (warp == sw && lane < nin) {
        if (ev.ff_setup) {
          if (WF == 0) taylorf2_setup_ff(ev, propf[lane], P[lane]);
          else phenomd_setup_ff(ev, propf[lane], P[lane]);
        } else {
          double pd[kMaxDim];
#pragma unroll
          for (int d = 0; d < kMaxDim; ++d) pd[d] = d < D ? (double)propf[lane][d].h + (double)propf[lane][d].l : 0.0;
          setup_from_unit<2, WF>(ev, pd, P[lane]);
        }
      }
      __syncthreads();
    }
    // C. likelihoods
    constexpr int V = Pow2Vals<NV>::value;
    constexpr int group = 32 / V;
    if (nin > 0) {
      if (rb) {
        for (int i = warp; i < nin; i += kWarps) {
          int nk;
          const double v = rb_lnl_warp<NDET, WF>(ev, P[i], lane, &nk);
          if (lane == 0) { s_rbl[i] = v; s_rbk[i] = nk; }
        }
      } else if (WF == 1) {
        for (int i = 0; i < nin; ++i) {
          double dv[NV];
          float fv[NV], fc[NV];
          partials<2, NDET, WF>(ev, P[i], threadIdx.x, kThreads, dv, fv, fc);
          float rs, rc;
          int q;
          warp_halving_sums<NV>(fv, fc, lane, rs, rc, q);
          if ((lane & (group - 1)) == 0 && q < NV) { wsums[i][warp][2 * q] = rs; wsums[i][warp][2 * q + 1] = rc; }
        }
      } else {
        for (int i = warp; i < nin; i += kWarps) {
          double dv[NV];
          float fv[NV], fc[NV];
          partials<2, NDET, WF>(ev, P[i], lane, 32, dv, fv, fc);
          float rs, rc;
          int q;
          warp_halving_sums<NV>(fv, fc, lane, rs, rc, q);
          if ((lane & (group - 1)) == 0 && q < NV) { part_sums[i][2 * q] = rs; part_sums[i][2 * q + 1] = rc; }
        }
      }
      __syncthreads();
    }
    // D. ln L of every slot (warp 0), then thread 0 replays the sequential move over the candidates
    if (warp == 0) {
      if (lane < nin) {
        double l;
        int kb;
        if (rb) {
          l = s_rbl[lane];
          kb = s_rbk[lane];
        } else if (WF == 1) {
          float ps[2 * NV];
#pragma unroll
          for (int q = 0; q < NV; ++q) {
            float sh = wsums[lane][0][2 * q], sl = wsums[lane][0][2 * q + 1];
#pragma unroll
            for (int w2 = 1; w2 < kWarps; ++w2) {
              float tt, e;
              two_sum(sh, wsums[lane][w2][2 * q], tt, e);
              sh = tt;
              sl += wsums[lane][w2][2 * q + 1] + e;
            }
            ps[2 * q] = sh;
            ps[2 * q + 1] = sl;
          }
          l = lnl_ff<NDET, WF>(ev, P[lane], ps);
          kb = P[lane].k_end;
        } else {
          l = lnl_ff<NDET, WF>(ev, P[lane], part_sums[lane]);
          kb = P[lane].k_end;
        }
        lnl_c[lane] = l;
        kend_c[lane] = kb;
        ins_c[lane] = l > lnl_star ? 1 : 0;
      }
      __syncwarp();
      if (lane == 0) {
        const int nc = s_nc & 255;
        n_spec += nin;
        bool move_end = false;
        int sh0 = 0;          // first shrinkage candidate of the round
        bool shrink = true;   // the round's shrinkage candidates are the move's next ones
        if (left_on || right_on) {
          const int ql = (s_nc >> 8) & 255, qr = (s_nc >> 16) & 255;
          // the speculative shrinkage holds iff every side extending at the round's start stops
          // at its first end here (the bracket is then the one the candidates were drawn in)
          if ((left_on && ql == 0) || (right_on && qr == 0)) shrink = false;
          for (int i = 0; i < ql && left_on; ++i) {
            const int sl = cslot[i];
            bool ins = false;
            if (sl >= 0) {
              ++calls;
              n_bins += kend_c[sl];
              ins = ins_c[sl] != 0;
            }
            if (ins) {
              shrink = false;
              lo -= 1.0;
              if (--jl == 0) left_on = false;
            } else {
              left_on = false;
            }
          }
          for (int i = ql; i < ql + qr && right_on; ++i) {
            const int sl = cslot[i];
            bool ins = false;
            if (sl >= 0) {
              ++calls;
              n_bins += kend_c[sl];
              ins = ins_c[sl] != 0;
            }
            if (ins) {
              shrink = false;
              hi += 1.0;
              if (--kr == 0) right_on = false;
            } else {
              right_on = false;
            }
          }
          sh0 = ql + qr;
          if (left_on || right_on) shrink = false;
        }
        if (shrink) {
          for (int i = sh0; i < nc; ++i) {
            const int sl = cslot[i];
            if (sl >= 0) {
              ++calls;
              n_bins += kend_c[sl];
              if (ins_c[sl]) {
                for (int d = 0; d < D; ++d) x[d] = cpt[i][d];
                lnl = lnl_c[sl];
                ++moves;
                move_end = true;
                break;
              }
            }
            if (ct[i] < 0.0) lo = ct[i];
            else hi = ct[i];
            if (++nsh == kHrssMaxShrink) {
              move_end = true;
              break;
            }
          }
        }
        if (move_end) ++t;
        s_newmove = move_end ? 1 : 0;
        s_t = t;
        if (t >= n_steps) s_exit = 1;
        if (!s_exit && walk_should_stop(T, t0, walk_abort_flag(T))) {   // watchdog: the walker stays where it is
          s_exit = 1;
          if (T.status) atomicOr(T.status, 1);
        }
      }
    }
    __syncthreads();
  }
  if ((int)threadIdx.x < D) T.u_out[(size_t)j * D + threadIdx.x] = x[threadIdx.x];
  if (threadIdx.x == 0) {
    T.lnl_out[j] = lnl;
    T.n_acc[j] = moves;
    T.n_like[j] = calls;
    if (T.n_bins) T.n_bins[j] = n_bins;
    if (T.n_spec) T.n_spec[j] = n_spec;
  }
}

}  // namespace

// Launchers of one precision P; each kernels_pP.cu instantiates its own.
#define GWNS_DISPATCH_N(K, P, W)                                                  \
  if (n_det == 1) K(P, 1, W); else if (n_det == 2) K(P, 2, W);                    \
  else if (n_det == 3) K(P, 3, W); else K(P, 4, W);
#define GWNS_DISPATCH_W(K, P)                                                     \
  if (waveform == 0) { GWNS_DISPATCH_N(K, P, 0) } else { GWNS_DISPATCH_N(K, P, 1) }

template <int P>
cudaError_t launch_likelihood_p(int waveform, int n_det, const EventDev* d_ev, const double* d_theta, int n,
                                double* d_lnl, int32_t* d_status, cudaStream_t s) {
#define GWNS_LIK(P_, N, W) likelihood_kernel<P_, N, W><<<n, kThreads, 0, s>>>(d_ev, d_theta, n, d_lnl, d_status)
  GWNS_DISPATCH_W(GWNS_LIK, P)
#undef GWNS_LIK
  return cudaGetLastError();
}

template <int P>
cudaError_t launch_unit_likelihood_p(int waveform, int n_det, const EventDev* d_ev, const double* d_u, int n,
                                     double* d_lnl, cudaStream_t s) {
#define GWNS_UL(P_, N, W) unit_likelihood_kernel<P_, N, W><<<n, kThreads, 0, s>>>(d_ev, d_u, n, d_lnl)
  GWNS_DISPATCH_W(GWNS_UL, P)
#undef GWNS_UL
  return cudaGetLastError();
}

// Mode 2 runs the float-float walk; modes 0 and 1 the FP64-recheck walk.  A TaylorF2 launch
// whose tasks use neither flow proposals nor the relative-binning likelihood (extras false)
// runs the float-float walk compiled without those paths (a smaller kernel: its round is
// short and instruction fetch is among its first stalls).  Both properties of an event are
// fixed before its first ns_step (ns_relbin_set is refused after it), so the sampler's
// captured batch graphs keep a valid choice.
template <int P, int N, int W>
void launch_walk_one(int n_blocks, cudaStream_t s, const EventDev* d_evs, WalkTask* d_tasks,
                     const int32_t* d_blk_task, const int32_t* d_blk_local, bool extras) {
  if constexpr (P == 2) {
    if (W == 0 && !extras)
      walk_kernel_ff<N, W, false><<<n_blocks, kThreads, 0, s>>>(d_evs, d_tasks, d_blk_task, d_blk_local);
    else
      walk_kernel_ff<N, W, true><<<n_blocks, kThreads, 0, s>>>(d_evs, d_tasks, d_blk_task, d_blk_local);
  } else {
    walk_kernel<P, N, W><<<n_blocks, kThreads, 0, s>>>(d_evs, d_tasks, d_blk_task, d_blk_local);
  }
}

template <int P>
cudaError_t launch_walk_p(int waveform, int n_det, const EventDev* d_evs, WalkTask* d_tasks,
                          const int32_t* d_blk_task, const int32_t* d_blk_local, int n_blocks, cudaStream_t s,
                          bool extras) {
#define GWNS_WALK(P_, N, W) launch_walk_one<P_, N, W>(n_blocks, s, d_evs, d_tasks, d_blk_task, d_blk_local, extras)
  GWNS_DISPATCH_W(GWNS_WALK, P)
#undef GWNS_WALK
  return cudaGetLastError();
}

// Mode 2 runs the speculative float-float HRSS kernel; modes 0 and 1 one candidate at a time.
template <int P, int N, int W>
void launch_hrss_one(int n_blocks, cudaStream_t s, const EventDev* d_evs, WalkTask* d_tasks,
                     const int32_t* d_blk_task, const int32_t* d_blk_local) {
  if constexpr (P == 2) hrss_kernel_ff<N, W><<<n_blocks, kThreads, 0, s>>>(d_evs, d_tasks, d_blk_task, d_blk_local);
  else hrss_kernel<P, N, W><<<n_blocks, kThreads, 0, s>>>(d_evs, d_tasks, d_blk_task, d_blk_local);
}

template <int P>
cudaError_t launch_hrss_p(int waveform, int n_det, const EventDev* d_evs, WalkTask* d_tasks,
                          const int32_t* d_blk_task, const int32_t* d_blk_local, int n_blocks, cudaStream_t s) {
#define GWNS_HRSS(P_, N, W) launch_hrss_one<P_, N, W>(n_blocks, s, d_evs, d_tasks, d_blk_task, d_blk_local)
  GWNS_DISPATCH_W(GWNS_HRSS, P)
#undef GWNS_HRSS
  return cudaGetLastError();
}

}  // namespace gwns
