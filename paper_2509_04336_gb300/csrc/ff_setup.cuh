// ff_setup.cuh -- the per-proposal constants of the float-float TaylorF2 likelihood, formed in
// float-float arithmetic (ff.cuh) on the FP32 pipe.
//
// It computes what taylorf2_setup_lean followed by make_ff computes -- prior transform, masses,
// the 3.5PN phase coefficients regrouped on the frequency basis, the phase constant, the
// arrival delays and the split time shifts, the antenna patterns and the template power -- from
// the unit-cube coordinates as float pairs, without FP64.  With about 48 significant bits every
// coefficient is accurate far below what the phase needs (~1e-6 cycle).  The amplitude factors
// K P_det are FP32, scaled by 2^70, and <h|h> comes from an FP32 copy of the template-power
// prefix sums scaled by 2^-140; lnl_ff assembles ln L in float-float.
#pragma once

#include "ff.cuh"

namespace gwns {

__device__ __forceinline__ ff ff_of(const float* f) { return ff{f[0], f[1]}; }
__device__ __forceinline__ ff ff_from_double(double x) {
  const float h = __double2float_rn(x);
  return ff{h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ bool ff_le(ff a, ff b) { return a.h < b.h || (a.h == b.h && a.l <= b.l); }

// Frequency of bin k (f_min + k df) as a float-float pair.
__device__ __forceinline__ ff ff_bin_freq(const EventDev& ev, int k) {
  return ff_add(ff_of(ev.fmin_f), ff_mul_f(ff_of(ev.df_f), (float)k));
}

// The sampled parameters, masses and PN coefficients of one proposal in float-float.
struct FFCore {
  ff mc, q, opq, eta, delta, chis, chia, chi1, chi2, phic, tc, ra, sd, cd;
  ff c1, ci1, ci2, ci3, ci5, lpm, pre;
  ff a[8], al5;
  float dl, ci, psi;
};

// Parameter i with a uniform or fixed prior at the float-float unit-cube point x.
__device__ __forceinline__ ff ff_prior_lin(const EventDev& ev, int i, const ff* x) {
  const PriorDev& P = ev.prior[i];
  const int d = ev.param_dim[i];
  if (d < 0) return ff_of(P.v_f);
  return ff_add(ff_of(P.lo_f), ff_mul(x[d], ff_of(P.w_f)));
}
// The distance (uniform, power law or fixed): an amplitude-only parameter, FP32.
__device__ __forceinline__ float ff_prior_dl(const EventDev& ev, const ff* x) {
  const PriorDev& P = ev.prior[4];
  const int d = ev.param_dim[4];
  if (d < 0) return P.v_f[0];
  if (P.kind == kPowerLaw) return powf(P.A_f[0] + x[d].h * P.B_f[0], P.einv_f);
  return ff_add(ff_of(P.lo_f), ff_mul(x[d], ff_of(P.w_f))).h;
}
// cos(theta_jn) (uniform, sine or fixed prior): amplitude only, FP32.
__device__ __forceinline__ float ff_prior_ci(const EventDev& ev, const ff* x) {
  const PriorDev& P = ev.prior[5];
  const int d = ev.param_dim[5];
  if (d < 0) return P.cv_f[0];
  if (P.kind == kSine) return fminf(1.0f, fmaxf(-1.0f, P.A_f[0] - x[d].h * P.B_f[0]));
  return cosf(ff_add(ff_of(P.lo_f), ff_mul(x[d], ff_of(P.w_f))).h);
}
// sin and cos of the declination (uniform, cosine or fixed prior), float-float.
__device__ __forceinline__ void ff_prior_dec(const EventDev& ev, const ff* x, ff& sd, ff& cd) {
  const PriorDev& P = ev.prior[10];
  const int d = ev.param_dim[10];
  if (d < 0) {
    sd = ff_of(P.sv_f);
    cd = ff_of(P.cv_f);
  } else if (P.kind == kCosine) {
    sd = ff_add(ff_of(P.A_f), ff_mul(x[d], ff_of(P.B_f)));
    if (sd.h > 1.0f) sd = ff_make(1.0f);
    if (sd.h < -1.0f) sd = ff_make(-1.0f);
    cd = ff_sqrt(ff_mul(ff_add_f(ff_neg(sd), 1.0f), ff_add_f(sd, 1.0f)));
  } else {
    ff_sincos(ff_add(ff_of(P.lo_f), ff_mul(x[d], ff_of(P.w_f))), sd, cd);
  }
}

// 1 + q, eta = q / (1 + q)^2 and delta = (1 - q) / (1 + q) from c.q.
__device__ __forceinline__ void ff_mass_ratio(FFCore& c) {
  c.opq = ff_add_f(c.q, 1.0f);
  const ff r_opq = ff_div(ff_make(1.0f), c.opq);
  c.eta = ff_mul(c.q, ff_mul(r_opq, r_opq));
  c.delta = ff_mul(ff_add_f(ff_neg(c.q), 1.0f), r_opq);
}
// The powers of (pi M)^(1/3) that the phase needs, from c.mc and c.eta.
__device__ __forceinline__ void ff_mass_scales(FFCore& c) {
  const ff pmc = ff_mul(GWNS_FF(kPi * kMsunS), c.mc);   // pi Mc [s]
  const ff w = ff_rcbrt(pmc);                            // (pi Mc)^(-1/3)
  const ff z = ff_rfifth(c.eta);                         // eta^(-1/5)
  c.c1 = ff_mul(ff_mul(pmc, ff_mul(w, w)), z);           // (pi M)^(1/3)
  const ff z2 = ff_mul(z, z);
  c.ci1 = ff_mul(ff_mul(w, c.eta), ff_mul(z2, z2));      // (pi M)^(-1/3)
  c.ci2 = ff_mul(c.ci1, c.ci1);
  c.ci3 = ff_mul(c.ci2, c.ci1);
  c.ci5 = ff_mul(c.ci3, c.ci2);
}
// ln(pi M) and the Newtonian prefactor 3 / (256 pi eta), from c.c1, c.opq and c.q.
__device__ __forceinline__ void ff_log_and_prefactor(FFCore& c) {
  c.lpm = ff_mul_f(ff_log(c.c1), 3.0f);
  c.pre = ff_div(ff_mul(GWNS_FF(3.0 / (256.0 * kPi)), ff_mul(c.opq, c.opq)), c.q);
}

// 3.5PN aligned-spin coefficients (the same polynomials as taylorf2_pn_coeffs) from c.eta,
// c.delta and the spins.
__device__ inline void ff_pn_coeffs(FFCore& c) {
  c.chis = ff_ldexp(ff_add(c.chi1, c.chi2), -1);
  c.chia = ff_ldexp(ff_sub(c.chi1, c.chi2), -1);
  const ff eta = c.eta, chis = c.chis, chia = c.chia;
  const ff e2 = ff_mul(eta, eta), e3 = ff_mul(e2, eta);
  const ff dchia = ff_mul(c.delta, chia);
  c.a[0] = ff_make(1.0f);
  c.a[1] = ff_make(0.0f);
  c.a[2] = ff_add(GWNS_FF(3715.0 / 756.0), ff_mul(GWNS_FF(55.0 / 9.0), eta));
  c.a[3] = ff_add(ff_add(GWNS_FF(-16.0 * kPi), ff_mul(GWNS_FF(113.0 / 3.0), dchia)),
                  ff_mul(ff_add(GWNS_FF(113.0 / 3.0), ff_mul(GWNS_FF(-76.0 / 3.0), eta)), chis));
  ff a4 = ff_add(ff_add(GWNS_FF(15293365.0 / 508032.0), ff_mul(GWNS_FF(27145.0 / 504.0), eta)),
                 ff_mul(GWNS_FF(3085.0 / 72.0), e2));
  a4 = ff_add(a4, ff_mul(ff_add(GWNS_FF(-405.0 / 8.0), ff_mul(GWNS_FF(200.0), eta)), ff_mul(chia, chia)));
  a4 = ff_add(a4, ff_mul(GWNS_FF(-405.0 / 4.0), ff_mul(dchia, chis)));
  a4 = ff_add(a4, ff_mul(ff_add(GWNS_FF(-405.0 / 8.0), ff_mul(GWNS_FF(5.0 / 2.0), eta)), ff_mul(chis, chis)));
  c.a[4] = a4;
  const ff gso = ff_add(
      ff_mul(ff_add(ff_add(GWNS_FF(732985.0 / 2268.0), ff_mul(GWNS_FF(-24260.0 / 81.0), eta)),
                    ff_mul(GWNS_FF(-340.0 / 9.0), e2)),
             chis),
      ff_mul(ff_add(GWNS_FF(732985.0 / 2268.0), ff_mul(GWNS_FF(140.0 / 9.0), eta)), dchia));
  c.a[5] = ff_sub(ff_add(GWNS_FF(38645.0 * kPi / 756.0), ff_mul(GWNS_FF(-65.0 * kPi / 9.0), eta)), gso);
  ff a6 = GWNS_FF(11583231236531.0 / 4694215680.0 - 6848.0 * kEulerGamma / 21.0 - 640.0 * kPi * kPi / 3.0 -
                  6848.0 / 21.0 * kLn4);
  a6 = ff_add(a6, ff_mul(GWNS_FF(-15737765635.0 / 3048192.0 + 2255.0 * kPi * kPi / 12.0), eta));
  a6 = ff_add(a6, ff_add(ff_mul(GWNS_FF(76055.0 / 1728.0), e2), ff_mul(GWNS_FF(-127825.0 / 1296.0), e3)));
  a6 = ff_add(a6, ff_mul(GWNS_FF(kPi * 2270.0 / 3.0), dchia));
  a6 = ff_add(a6, ff_mul(ff_add(GWNS_FF(kPi * 2270.0 / 3.0), ff_mul(GWNS_FF(-520.0 * kPi), eta)), chis));
  c.a[6] = a6;
  ff a7 = ff_add(ff_add(GWNS_FF(kPi * 77096675.0 / 254016.0), ff_mul(GWNS_FF(kPi * 378515.0 / 1512.0), eta)),
                 ff_mul(GWNS_FF(-kPi * 74045.0 / 756.0), e2));
  {
    ff s = ff_add(ff_add(GWNS_FF(-25150083775.0 / 3048192.0), ff_mul(GWNS_FF(10566655595.0 / 762048.0), eta)),
                  ff_add(ff_mul(GWNS_FF(-1042165.0 / 3024.0), e2), ff_mul(GWNS_FF(5345.0 / 36.0), e3)));
    a7 = ff_add(a7, ff_mul(s, chis));
    ff t = ff_add(ff_add(GWNS_FF(-25150083775.0 / 3048192.0), ff_mul(GWNS_FF(26804935.0 / 6048.0), eta)),
                  ff_mul(GWNS_FF(-1985.0 / 48.0), e2));
    a7 = ff_add(a7, ff_mul(t, dchia));
  }
  c.a[7] = a7;
  c.al5 = ff_mul_f(c.a[5], 3.0f);
}

// The sky and amplitude parameters of the projection.
__device__ __forceinline__ void ff_extrinsic(const EventDev& ev, const ff* x, FFCore& c) {
  c.mc = ff_prior_lin(ev, 0, x);
  c.tc = ff_prior_lin(ev, 8, x);
  c.ra = ff_prior_lin(ev, 9, x);
  c.psi = ff_prior_lin(ev, 6, x).h;
  c.dl = ff_prior_dl(ev, x);
  c.ci = ff_prior_ci(ev, x);
  ff_prior_dec(ev, x, c.sd, c.cd);
}

// Prior transform, masses and the 3.5PN coefficients from the float-float unit-cube point x
// (requires ev.ff_setup).
__device__ inline void ff_core(const EventDev& ev, const ff* x, FFCore& c) {
  ff_extrinsic(ev, x, c);
  c.q = ff_prior_lin(ev, 1, x);
  c.chi1 = ff_prior_lin(ev, 2, x);
  c.chi2 = ff_prior_lin(ev, 3, x);
  c.phic = ff_prior_lin(ev, 7, x);
  ff_mass_ratio(c);
  ff_mass_scales(c);
  ff_pn_coeffs(c);
  ff_log_and_prefactor(c);
}

// The products that make the TaylorF2 basis coefficients (cycles): C_j for j in [j0, j1).
__device__ inline void ff_tf2_coeff_range(const FFCore& c, int j0, int j1, WalkerParams& p) {
  const ff pre = c.pre, c1 = c.c1;
  const ff al6 = GWNS_FF(-6848.0 / 21.0);
  const ff lpm3 = ff_mul(c.lpm, GWNS_FF(1.0 / 3.0));
#pragma unroll
  for (int j = 0; j < kBasis; ++j) {
    if (j < j0 || j >= j1) continue;
    ff C;
    if (j == 0) C = ff_mul(pre, c.ci5);
    else if (j == 1) C = ff_mul(ff_mul(pre, c.ci3), c.a[2]);
    else if (j == 2) C = ff_mul(ff_mul(pre, c.ci2), c.a[3]);
    else if (j == 3) C = ff_mul(ff_mul(pre, c.ci1), c.a[4]);
    else if (j == 4) C = ff_mul(ff_mul(pre, c1), ff_add(c.a[6], ff_mul(al6, lpm3)));
    else if (j == 5) C = ff_mul(ff_mul(pre, ff_mul(c1, c1)), c.a[7]);
    else if (j == 6) C = ff_mul(ff_mul(pre, c.al5), GWNS_FF(1.0 / 3.0));
    else C = ff_mul(ff_mul(ff_mul(pre, c1), al6), GWNS_FF(1.0 / 3.0));
    p.Ch[j] = C.h;
    p.Cl[j] = C.l;
  }
}
// The phase constant (cycles).
__device__ inline void ff_tf2_phase0(const FFCore& c, WalkerParams& p) {
  const ff lpm3 = ff_mul(c.lpm, GWNS_FF(1.0 / 3.0));
  ff ph0 = ff_mul(c.pre, ff_add(c.a[5], ff_mul(c.al5, lpm3)));
  ph0 = ff_sub(ph0, ff_mul(c.phic, GWNS_FF(1.0 / kPi)));
  ph0 = ff_add_f(ph0, -0.125f);
  p.ph0h = ph0.h;
  p.ph0l = ph0.l;
}
// TaylorF2 phase coefficients on the basis and the phase constant, float-float.
__device__ inline void ff_tf2_coeffs(const FFCore& c, WalkerParams& p) {
  ff_tf2_coeff_range(c, 0, kBasis, p);
  ff_tf2_phase0(c, p);
}

// Number of bins with f_k <= f_cut (le) or f_k < f_cut (strict), float-float comparisons.
__device__ inline int ff_bins_below(const EventDev& ev, ff f_cut, bool strict) {
  const float kg = floorf((f_cut.h - ev.fmin_f[0]) / ev.df_f[0]);
  int k = (int)fminf(fmaxf(kg, -1.0f), (float)(ev.n_bins - 1));
  auto in = [&](int kk) {
    const ff f = ff_bin_freq(ev, kk);
    return strict ? !ff_le(f_cut, f) : ff_le(f, f_cut);
  };
  while (k + 1 <= ev.n_bins - 1 && in(k + 1)) ++k;
  while (k >= 0 && !in(k)) --k;
  return k + 1;
}

// Sky direction (float-float: it sets the arrival delays), antenna patterns and amplitude in
// FP32 (K P scaled by 2^70) and the split time shifts.
__device__ inline void ff_projection(const EventDev& ev, const FFCore& c, WalkerParams& p) {
  ff sp, cp;
  ff_sincos(ff_sub(c.ra, ff_of(ev.gmst_f)), sp, cp);
  const ff n0 = ff_mul(c.cd, cp), n1 = ff_mul(c.cd, sp), n2 = c.sd;
  const float spf = sp.h, cpf = cp.h, ctf = c.sd.h, stf = c.cd.h;
  float ssf, csf;
  sincosf(c.psi, &ssf, &csf);
  const float X0 = spf * csf - ssf * cpf * ctf, X1 = -(cpf * csf + ssf * spf * ctf), X2 = ssf * stf;
  const float Y0 = -spf * ssf - csf * cpf * ctf, Y1 = cpf * ssf - csf * spf * ctf, Y2 = stf * csf;
  const float mcs = c.mc.h * (float)kMsunS;
  // K scaled by 2^70: K P ~ 1e-21 and (K P)^2 would leave FP32's normal range
  const float K = ldexpf((float)kAmp0 * sqrtf(mcs) * cbrtf(mcs) * (float)(kC / kMpcM) / c.dl, kKpScaleExp);
  const float ap = 0.5f * (1.0f + c.ci * c.ci);
  for (int det = 0; det < ev.n_det; ++det) {
    const float* xa = ev.xarm32[det];
    const float* ya = ev.yarm32[det];
    float xX = xa[0] * X0 + xa[1] * X1 + xa[2] * X2, xY = xa[0] * Y0 + xa[1] * Y1 + xa[2] * Y2;
    float yX = ya[0] * X0 + ya[1] * X1 + ya[2] * X2, yY = ya[0] * Y0 + ya[1] * Y1 + ya[2] * Y2;
    float fp = 0.5f * (xX * xX - xY * xY - yX * yX + yY * yY);
    float fc = xX * xY - yX * yY;
    p.kpf_re[det] = K * (fp * ap);
    p.kpf_im[det] = K * (-fc * c.ci);
    // tau = t_c - (r . n) / c, and its products with f_min (reduced) and df (split at a 9-bit head)
    const ff dot = ff_add(ff_add(ff_mul(ff_of(ev.vc_f[det][0]), n0), ff_mul(ff_of(ev.vc_f[det][1]), n1)),
                          ff_mul(ff_of(ev.vc_f[det][2]), n2));
    const ff tau = ff_sub(c.tc, dot);
    const ff a = ff_mul(tau, ff_of(ev.fmin_f));
    p.sa[det] = (a.h - rintf(a.h)) + a.l;
    const ff b = ff_mul(tau, ff_of(ev.df_f));
    const float bh = __int_as_float(__float_as_int(b.h) & (int)0xFFFF8000u);
    p.sbh[det] = bh;
    p.sbl[det] = (b.h - bh) + b.l;
  }
}

// TaylorF2 <h|h> = sum_det (K P_det)^2 sum_{k < k_end} 4 df f^-7/3 / S from the prefix sums
// (the two 2^(+-140) scalings cancel in the assembly); needs p.k_end and p.kpf.
__device__ inline void ff_tf2_hh(const EventDev& ev, WalkerParams& p) {
  float hh = 0.0f;
  for (int det = 0; det < ev.n_det; ++det) {
    const float psum = p.k_end > 0 ? ev.hhp32[(size_t)det * ev.n_bins + p.k_end - 1] : 0.0f;
    hh += (p.kpf_re[det] * p.kpf_re[det] + p.kpf_im[det] * p.kpf_im[det]) * psum;
  }
  p.hh_f = hh;
}

// Last bin at or below the test-mass ISCO frequency 1/(6^(3/2) pi M).
__device__ __forceinline__ int ff_tf2_kend(const EventDev& ev, const FFCore& c) {
  return ff_bins_below(ev, ff_mul(GWNS_FF(1.0 / kSix15), c.ci3), false);
}

// Mode-2 TaylorF2 proposal constants straight from the float-float unit-cube point x.
__device__ inline void taylorf2_setup_ff(const EventDev& ev, const ff* x, WalkerParams& p) {
  FFCore c;
  ff_core(ev, x, c);
  p.k_end = ff_tf2_kend(ev, c);
  ff_tf2_coeffs(c, p);
  ff_projection(ev, c, p);
  ff_tf2_hh(ev, p);
}

// The same constants formed by the warps of a CTA at once: each warp runs one part for every
// proposal of a round (lane i: proposal i), the parts exchange through shared memory, then a
// second pass forms the products.  The arithmetic is the one-lane setup's, split at its
// independent chains -- first pass: (0) mass scales, ln(pi M), prefactor; (1) PN coefficients;
// (2) sky, antenna patterns, delays; second pass: (0, 1) the basis coefficients, (2) the phase
// constant, (3) the ISCO bin and <h|h>.  TF2Part carries (0) and (1) to the second pass.
struct TF2Part {
  ff pre, c1, ci1, ci2, ci3, ci5, lpm, phic;
  ff a[8], al5;
};

__device__ inline void tf2_split_first(int part, const EventDev& ev, const ff* x, TF2Part& s, WalkerParams& p) {
  FFCore c;
  if (part == 0) {
    c.mc = ff_prior_lin(ev, 0, x);
    c.q = ff_prior_lin(ev, 1, x);
    ff_mass_ratio(c);
    ff_mass_scales(c);
    ff_log_and_prefactor(c);
    s.pre = c.pre; s.c1 = c.c1; s.ci1 = c.ci1; s.ci2 = c.ci2; s.ci3 = c.ci3; s.ci5 = c.ci5; s.lpm = c.lpm;
    s.phic = ff_prior_lin(ev, 7, x);
  } else if (part == 1) {
    c.q = ff_prior_lin(ev, 1, x);
    c.chi1 = ff_prior_lin(ev, 2, x);
    c.chi2 = ff_prior_lin(ev, 3, x);
    ff_mass_ratio(c);
    ff_pn_coeffs(c);
#pragma unroll
    for (int j = 0; j < 8; ++j) s.a[j] = c.a[j];
    s.al5 = c.al5;
  } else if (part == 2) {
    ff_extrinsic(ev, x, c);
    ff_projection(ev, c, p);
  }
}

__device__ inline void tf2_split_second(int part, const EventDev& ev, const TF2Part& s, WalkerParams& p) {
  FFCore c;
  c.pre = s.pre; c.c1 = s.c1; c.ci1 = s.ci1; c.ci2 = s.ci2; c.ci3 = s.ci3; c.ci5 = s.ci5; c.lpm = s.lpm;
  c.phic = s.phic;
#pragma unroll
  for (int j = 0; j < 8; ++j) c.a[j] = s.a[j];
  c.al5 = s.al5;
  if (part == 0) ff_tf2_coeff_range(c, 0, 4, p);
  else if (part == 1) ff_tf2_coeff_range(c, 4, 8, p);
  else if (part == 2) ff_tf2_phase0(c, p);
  else {
    p.k_end = ff_tf2_kend(ev, c);
    ff_tf2_hh(ev, p);
  }
}

// Mode-2 IMRPhenomD-form proposal constants from the unit-cube point u: the TaylorF2 part as
// above, then the quantities of phenomd_extra<true> -- the ringdown fit, the pseudo-PN and
// continuity constants and the region coefficients in float-float, the bin boundaries by
// float-float comparisons, the ringdown frequency, damping and amplitude shape in FP32 (the
// FP64 path's FAST variant rounds the same quantities to FP32).  Two halves that depend on the
// TaylorF2 core only: pd_chain (continuity constants, region coefficients, phase constants) and
// pd_bins_amp (region boundaries, amplitude shape); the one-lane setup runs both, the split setup
// runs them on different warps.
// Quantities both halves need: mass scales of the ringdown model and the ringdown frequency and
// damping (units of 1/M, FP32).
struct PDPro {
  ff eta, inv2pe, piM, M, M13, lnM;
  float qf32, etaf, at, af, mfin, om, qfac, frd, fd;
};
__device__ inline PDPro pd_prologue(const FFCore& c) {
  PDPro r;
  r.eta = c.eta;
  r.inv2pe = ff_div(ff_make(1.0f), ff_mul(GWNS_FF(2.0 * kPi), r.eta));
  r.piM = ff_mul(ff_mul(c.c1, c.c1), c.c1);
  r.M = ff_mul(r.piM, GWNS_FF(1.0 / kPi));
  r.M13 = ff_mul(c.c1, GWNS_FF(1.0 / 1.4645918875615231));   // M^(1/3)
  r.lnM = ff_sub(c.lpm, GWNS_FF(kLnPi));
  r.qf32 = c.q.h;
  r.etaf = r.eta.h;
  const float qf32 = r.qf32, etaf = r.etaf;
  r.at = (c.chi1.h + c.chi2.h * qf32 * qf32) / (1.0f + qf32 * qf32);
  const float at = r.at;
  r.af = at + at * etaf * (-0.1229f * at + 0.4537f * etaf - 2.8904f) +
         etaf * (2.0f * 1.7320508075688772f + -3.5171f * etaf + 2.5763f * etaf * etaf);
  r.mfin = 1.0f - ((float)kPdE1 * etaf + (float)kPdE2 * etaf * etaf);
  r.om = 1.5251f - 1.1568f * powf(1.0f - r.af, 0.1292f);
  r.qfac = 0.7000f + 1.4187f * powf(1.0f - r.af, -0.4990f);
  r.frd = r.om / (2.0f * (float)kPi * r.mfin);
  r.fd = r.frd / (2.0f * r.qfac);
  return r;
}
__device__ inline void pd_chain(const FFCore& c, WalkerParams& p) {
  PhenomExtra& e = p.pd;
  const PDPro pro = pd_prologue(c);
  const ff eta = pro.eta, inv2pe = pro.inv2pe, M = pro.M, M13 = pro.M13, lnM = pro.lnM;
  const float frd = pro.frd, fd = pro.fd;
  // inspiral at x1: value and slope of the TaylorF2 part from constant powers of v1
  ff s = ff_make(0.0f), ds = ff_make(0.0f);
  // v1^(k - 5), k = 0..7
  const ff vkf[8] = {GWNS_FF(120.0317221056134), GWNS_FF(46.07197497267014), GWNS_FF(17.683882565766147), GWNS_FF(6.78763397456508),
                     GWNS_FF(2.60530880598924), GWNS_FF(1.0), GWNS_FF(0.3838316585355026), GWNS_FF(0.14732674209411467)};
  const ff al6 = GWNS_FF(-6848.0 / 21.0);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const ff alk = k == 5 ? c.al5 : (k == 6 ? al6 : ff_make(0.0f));
    const ff t = ff_add(c.a[k], ff_mul(alk, GWNS_FF(kPdLnV1)));
    s = ff_add(s, ff_mul(t, vkf[k]));
    ds = ff_add(ds, ff_mul(vkf[k], ff_add(ff_mul_f(t, (float)(k - 5)), alk)));
  }
  const double x1 = kPdXIns;
  const ff cc = ff_div(GWNS_FF(3.0 / 128.0), eta);
  const ff ieta = ff_div(ff_make(1.0f), eta);
  const ff p1 = ff_add(ff_mul(cc, s), ff_mul(GWNS_FF(0.75 * kPdS2 * 0.004717334509576015 + 0.6 * kPdS3 *
                                                     0.001236291381957598 + 0.5 * kPdS4 * x1 * x1), ieta));
  const ff dp1 = ff_add(ff_mul(ff_mul(cc, ds), GWNS_FF(1.0 / (3.0 * x1))),
                        ff_mul(GWNS_FF(kPdS2 * 0.2620741394208897 + kPdS3 * 0.06868285455319992 + kPdS4 * x1),
                               ieta));
  const ff b1 = ff_add(ff_mul(eta, dp1), GWNS_FF(-kPdB2 / x1 - kPdB3 / (x1 * x1 * x1 * x1)));
  const ff b0 = ff_add(ff_sub(ff_mul(eta, p1), ff_mul(b1, GWNS_FF(x1))),
                       GWNS_FF(-kPdB2 * (-4.017383521085972) + kPdB3 / (3.0 * x1 * x1 * x1)));
  // intermediate at x2, merger-ringdown continuity (x2, frd, fd exact FP32 numbers)
  const float x2 = 0.5f * frd;
  const ff lnx2 = ff_log(ff_make(x2));
  const ff ix2 = ff_div(ff_make(1.0f), ff_make(x2));
  const ff ix2_2 = ff_mul(ix2, ix2), ix2_3 = ff_mul(ix2_2, ix2), ix2_4 = ff_mul(ix2_2, ix2_2);
  const ff pint2 = ff_mul(ff_add(ff_add(ff_add(b0, ff_mul_f(b1, x2)), ff_mul(GWNS_FF(kPdB2), lnx2)),
                                 ff_mul(GWNS_FF(-kPdB3 / 3.0), ix2_3)),
                          ieta);
  const ff dpint2 = ff_mul(ff_add(ff_add(b1, ff_mul(GWNS_FF(kPdB2), ix2)), ff_mul(GWNS_FF(kPdB3), ix2_4)), ieta);
  const float x2p34 = powf(x2, 0.75f), x2m14 = powf(x2, -0.25f);
  const float l2 = (float)kPdA4 * atanf((x2 - (float)kPdA5 * frd) / fd);
  const ff dd2 = ff_make(x2 - (float)kPdA5 * frd);
  const ff dl2 = ff_div(ff_mul_f(GWNS_FF(kPdA4), fd), ff_add(ff_mul(dd2, dd2), two_prod_ff(fd, fd)));
  const ff a1 = ff_sub(ff_sub(ff_sub(ff_mul(eta, dpint2), ff_mul(GWNS_FF(kPdA2), ix2_2)),
                              ff_mul_f(GWNS_FF(kPdA3), x2m14)),
                       dl2);
  const ff a0 = ff_add_f(ff_sub(ff_add(ff_sub(ff_mul(eta, pint2), ff_mul_f(a1, x2)), ff_mul(GWNS_FF(kPdA2), ix2)),
                                ff_mul_f(GWNS_FF(4.0 / 3.0 * kPdA3), x2p34)),
                         -l2);
  // region coefficients in f (cycles)
  const ff M2 = ff_mul(M, M);
  ff Cx[9];
  Cx[0] = ff_mul(ff_mul(GWNS_FF(0.75 * kPdS2), ff_mul(M, M13)), inv2pe);
  Cx[1] = ff_mul(ff_mul(GWNS_FF(0.6 * kPdS3), ff_mul(M, ff_mul(M13, M13))), inv2pe);
  Cx[2] = ff_mul(ff_mul(GWNS_FF(0.5 * kPdS4), M2), inv2pe);
  Cx[3] = ff_mul(GWNS_FF(kPdB2), inv2pe);
  Cx[4] = ff_mul(ff_div(GWNS_FF(-kPdB3 / 3.0), ff_mul(M2, M)), inv2pe);
  Cx[5] = ff_mul(ff_mul(b1, M), inv2pe);
  Cx[6] = ff_mul(ff_div(GWNS_FF(-kPdA2), M), inv2pe);
  Cx[7] = ff_mul(ff_mul_f(GWNS_FF(4.0 / 3.0 * kPdA3), powf(M.h, 0.75f)), inv2pe);
  Cx[8] = ff_mul(ff_mul(a1, M), inv2pe);
#pragma unroll
  for (int j = 0; j < 9; ++j) { e.Cxh[j] = Cx[j].h; e.Cxl[j] = Cx[j].l; }
  const ff tail = ff_add_f(ff_mul(c.phic, GWNS_FF(-1.0 / kPi)), -0.125f);
  const ff ph0_int = ff_add(ff_mul(ff_add(b0, ff_mul(GWNS_FF(kPdB2), lnM)), inv2pe), tail);
  const ff ph0_mr = ff_add(ff_mul(a0, inv2pe), tail);
  e.ph0_int_h = ph0_int.h; e.ph0_int_l = ph0_int.l;
  e.ph0_mr_h = ph0_mr.h; e.ph0_mr_l = ph0_mr.l;
}

__device__ inline void pd_bins_amp(const EventDev& ev, const FFCore& c, WalkerParams& p) {
  PhenomExtra& e = p.pd;
  const PDPro pro = pd_prologue(c);
  const ff inv2pe = pro.inv2pe, M = pro.M;
  const float etaf = pro.etaf, frd = pro.frd, fd = pro.fd;
  const double x1 = kPdXIns;
  const float x2 = 0.5f * frd;
  // region boundaries as bin indices
  const ff iM = ff_div(ff_make(1.0f), M);
  e.k1 = ff_bins_below(ev, ff_mul(GWNS_FF(x1), iM), true);
  e.k2 = ff_bins_below(ev, ff_mul_f(iM, x2), true);
  p.k_end = ff_bins_below(ev, ff_mul(GWNS_FF(kPdXCut), iM), false);
  // amplitude shape, FP32
  const float deltaf = c.delta.h, chiaf = c.chia.h, chisf = c.chis.h;
  const float A2 = -323.0f / 224.0f + 451.0f * etaf / 168.0f;
  const float A3 = 27.0f * deltaf * chiaf / 8.0f + (27.0f / 8.0f - 11.0f * etaf / 6.0f) * chisf;
  const float gd = (float)kPdG3 * fd;
  const float xa = (float)kPdXAmpIns;
  const float xp = fabsf(frd + gd * (sqrtf(1.0f - (float)(kPdG2 * kPdG2)) - 1.0f) / (float)kPdG2);
  const float va = cbrtf((float)kPi * xa);       // (pi x_amp_ins)^(1/3), as the FP64 path's FAST variant
  const float y0 = 1.0f + A2 * va * va + A3 * va * va * va;
  const float d0 = (2.0f * A2 * va + 3.0f * A3 * va * va) * va / (3.0f * xa);
  const float dp = xp - frd;
  const float ex = expf(-(float)kPdG2 * dp / gd);
  const float den = dp * dp + gd * gd;
  const float y1 = (float)kPdG1 * gd / den * ex;
  const float d1 = y1 * (-2.0f * dp / den - (float)kPdG2 / gd);
  const float span = xp - xa;
  e.ka = ff_bins_below(ev, ff_mul_f(iM, xa), true);
  e.kp = ff_bins_below(ev, ff_mul_f(iM, xp), true);
  e.A2f = A2; e.A3f = A3; e.c13f = c.c1.h; e.Mf = M.h; e.xaf = xa; e.inv_spanf = 1.0f / span;
  e.hy0f = y0; e.hd0f = span * d0;
  e.hc2f = 3.0f * (y1 - y0) - 2.0f * span * d0 - span * d1;
  e.hc3f = 2.0f * (y0 - y1) + span * d0 + span * d1;
  e.frdf = frd; e.gdf = gd; e.g1gdf = (float)kPdG1 * gd; e.g2_gdf = (float)kPdG2 / gd;
  e.at_scalef = (float)kPdA4 * (inv2pe.h + inv2pe.l); e.at_cf = (float)kPdA5 * frd; e.at_invf = 1.0f / fd;
  p.hh_f = 0.0f;   // the IMRPhenomD form sums its template power per bin
}

__device__ inline void phenomd_setup_ff(const EventDev& ev, const ff* x, WalkerParams& p) {
  FFCore c;
  ff_core(ev, x, c);
  ff_tf2_coeffs(c, p);
  pd_chain(c, p);
  pd_bins_amp(ev, c, p);
  ff_projection(ev, c, p);
}

// The IMRPhenomD-form constants formed by the warps of a CTA at once, as tf2_split_first /
// tf2_split_second: first pass (0) mass scales, ln(pi M), prefactor, mass ratio; (1) PN
// coefficients and spin combinations; (2) sky, antenna patterns, delays; second pass (0, 1) the
// TaylorF2 basis coefficients, (2) the phase constant and pd_chain, (3) pd_bins_amp.  The
// arithmetic of every quantity is the one-lane setup's.
struct PDPart {
  TF2Part t;
  ff q, eta, delta, chis, chia, chi1, chi2;
};

__device__ inline void pd_split_first(int part, const EventDev& ev, const ff* x, PDPart& s, WalkerParams& p) {
  tf2_split_first(part, ev, x, s.t, p);
  if (part == 0) {
    FFCore c;
    c.q = ff_prior_lin(ev, 1, x);
    ff_mass_ratio(c);
    s.q = c.q;
    s.eta = c.eta;
    s.delta = c.delta;
  } else if (part == 1) {
    s.chi1 = ff_prior_lin(ev, 2, x);
    s.chi2 = ff_prior_lin(ev, 3, x);
    s.chis = ff_ldexp(ff_add(s.chi1, s.chi2), -1);
    s.chia = ff_ldexp(ff_sub(s.chi1, s.chi2), -1);
  }
}

__device__ inline void pd_split_second(int part, const EventDev& ev, const PDPart& s, WalkerParams& p) {
  FFCore c;
  const TF2Part& t = s.t;
  c.pre = t.pre; c.c1 = t.c1; c.ci1 = t.ci1; c.ci2 = t.ci2; c.ci3 = t.ci3; c.ci5 = t.ci5; c.lpm = t.lpm;
  c.phic = t.phic;
#pragma unroll
  for (int j = 0; j < 8; ++j) c.a[j] = t.a[j];
  c.al5 = t.al5;
  c.q = s.q; c.eta = s.eta; c.delta = s.delta; c.chis = s.chis; c.chia = s.chia; c.chi1 = s.chi1; c.chi2 = s.chi2;
  if (part == 0) ff_tf2_coeff_range(c, 0, 4, p);
  else if (part == 1) ff_tf2_coeff_range(c, 4, 8, p);
  else if (part == 2) {
    ff_tf2_phase0(c, p);
    pd_chain(c, p);
  } else {
    pd_bins_amp(ev, c, p);
  }
}

}  // namespace gwns
