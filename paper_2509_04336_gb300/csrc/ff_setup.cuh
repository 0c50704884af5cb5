// ff_setup.cuh -- the per-proposal constants of the float-float TaylorF2 likelihood, formed in
// float-float arithmetic (ff.cuh) on the FP32 pipe.
//
// It computes what taylorf2_setup_lean followed by make_ff computes -- prior transform, masses,
// the 3.5PN phase coefficients regrouped on the frequency basis, the phase constant, the
// arrival delays and the split time shifts, the antenna patterns and the template power -- but
// keeps FP64 only for splitting the unit-cube coordinates (FP64 inputs) into float pairs.  With about 48
// significant bits every coefficient is accurate far below what the phase needs (~1e-6 cycle).
// The amplitude factors K P_det are FP32, scaled by 2^70, and <h|h> comes from an FP32 copy of
// the template-power prefix sums scaled by 2^-140; lnl_ff assembles ln L in float-float.
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

// Mode-2 TaylorF2 proposal constants straight from the unit-cube point u (requires
// ev.ff_setup; see taylorf2_setup_lean for the same quantities in FP64).
__device__ inline void taylorf2_setup_ff(const EventDev& ev, const double* u, WalkerParams& p) {
  ff x[kParams];
  float dl = 1.0f, ci = 1.0f;
  ff sd = ff_make(0.0f), cd = ff_make(1.0f);
  int d = 0;
#pragma unroll 1
  for (int i = 0; i < kParams; ++i) {
    const PriorDev& P = ev.prior[i];
    x[i] = ff_of(P.v_f);
    if (P.kind == kFixed) {
      if (i == 4) dl = P.v_f[0];
      if (i == 5) ci = P.cv_f[0];
      if (i == 10) { sd = ff_of(P.sv_f); cd = ff_of(P.cv_f); }
      continue;
    }
    const double v = u[d++];
    if (P.kind == kUniform) {
      x[i] = ff_add(ff_of(P.lo_f), ff_mul(ff_from_double(v), ff_of(P.w_f)));
      if (i == 4) dl = x[i].h;
      if (i == 5) ci = cosf(x[i].h);
    } else if (P.kind == kPowerLaw) {   // the distance: an amplitude-only parameter
      dl = powf(P.A_f[0] + (float)v * P.B_f[0], P.einv_f);
    } else if (P.kind == kSine) {       // cos(theta_jn), amplitude only
      ci = fminf(1.0f, fmaxf(-1.0f, P.A_f[0] - (float)v * P.B_f[0]));
    } else {                            // sin(declination)
      sd = ff_add(ff_of(P.A_f), ff_mul(ff_from_double(v), ff_of(P.B_f)));
      if (sd.h > 1.0f) sd = ff_make(1.0f);
      if (sd.h < -1.0f) sd = ff_make(-1.0f);
      cd = ff_sqrt(ff_mul(ff_add_f(ff_neg(sd), 1.0f), ff_add_f(sd, 1.0f)));
    }
  }
  if (ev.prior[10].kind == kUniform) ff_sincos(x[10], sd, cd);
  const ff mc = x[0], q = x[1], chi1 = x[2], chi2 = x[3], phic = x[7], tc = x[8], ra = x[9];
  const float psi = x[6].h;

  // masses and spins
  const ff opq = ff_add_f(q, 1.0f);
  const ff r_opq = ff_div(ff_make(1.0f), opq);
  const ff eta = ff_mul(q, ff_mul(r_opq, r_opq));
  const ff delta = ff_mul(ff_add_f(ff_neg(q), 1.0f), r_opq);
  const ff chis = ff_ldexp(ff_add(chi1, chi2), -1), chia = ff_ldexp(ff_sub(chi1, chi2), -1);
  const ff pmc = ff_mul(GWNS_FF(kPi * kMsunS), mc);     // pi Mc [s]
  const ff w = ff_rcbrt(pmc);                            // (pi Mc)^(-1/3)
  const ff z = ff_rfifth(eta);                           // eta^(-1/5)
  const ff c1 = ff_mul(ff_mul(pmc, ff_mul(w, w)), z);    // (pi M)^(1/3)
  const ff z2 = ff_mul(z, z);
  const ff ci1 = ff_mul(ff_mul(w, eta), ff_mul(z2, z2)); // (pi M)^(-1/3)
  const ff ci2 = ff_mul(ci1, ci1), ci3 = ff_mul(ci2, ci1), ci5 = ff_mul(ci3, ci2);

  // last bin at or below the test-mass ISCO frequency 1/(6^(3/2) pi M)
  {
    const ff f_cut = ff_mul(GWNS_FF(1.0 / kSix15), ci3);
    float kg = floorf((f_cut.h - ev.fmin_f[0]) / ev.df_f[0]);
    int k = (int)fminf(fmaxf(kg, -1.0f), (float)(ev.n_bins - 1));
    while (k + 1 <= ev.n_bins - 1 && ff_le(ff_bin_freq(ev, k + 1), f_cut)) ++k;
    while (k >= 0 && !ff_le(ff_bin_freq(ev, k), f_cut)) --k;
    p.k_end = k + 1;
  }

  // 3.5PN aligned-spin coefficients (the same polynomials as taylorf2_pn_coeffs)
  const ff e2 = ff_mul(eta, eta), e3 = ff_mul(e2, eta);
  const ff dchia = ff_mul(delta, chia);
  const ff a2 = ff_add(GWNS_FF(3715.0 / 756.0), ff_mul(GWNS_FF(55.0 / 9.0), eta));
  const ff a3 = ff_add(ff_add(GWNS_FF(-16.0 * kPi), ff_mul(GWNS_FF(113.0 / 3.0), dchia)),
                       ff_mul(ff_add(GWNS_FF(113.0 / 3.0), ff_mul(GWNS_FF(-76.0 / 3.0), eta)), chis));
  ff a4 = ff_add(ff_add(GWNS_FF(15293365.0 / 508032.0), ff_mul(GWNS_FF(27145.0 / 504.0), eta)),
                 ff_mul(GWNS_FF(3085.0 / 72.0), e2));
  a4 = ff_add(a4, ff_mul(ff_add(GWNS_FF(-405.0 / 8.0), ff_mul(GWNS_FF(200.0), eta)), ff_mul(chia, chia)));
  a4 = ff_add(a4, ff_mul(GWNS_FF(-405.0 / 4.0), ff_mul(dchia, chis)));
  a4 = ff_add(a4, ff_mul(ff_add(GWNS_FF(-405.0 / 8.0), ff_mul(GWNS_FF(5.0 / 2.0), eta)), ff_mul(chis, chis)));
  const ff gso = ff_add(
      ff_mul(ff_add(ff_add(GWNS_FF(732985.0 / 2268.0), ff_mul(GWNS_FF(-24260.0 / 81.0), eta)),
                    ff_mul(GWNS_FF(-340.0 / 9.0), e2)),
             chis),
      ff_mul(ff_add(GWNS_FF(732985.0 / 2268.0), ff_mul(GWNS_FF(140.0 / 9.0), eta)), dchia));
  const ff a5 = ff_sub(ff_add(GWNS_FF(38645.0 * kPi / 756.0), ff_mul(GWNS_FF(-65.0 * kPi / 9.0), eta)), gso);
  ff a6 = GWNS_FF(11583231236531.0 / 4694215680.0 - 6848.0 * kEulerGamma / 21.0 - 640.0 * kPi * kPi / 3.0 -
                  6848.0 / 21.0 * kLn4);
  a6 = ff_add(a6, ff_mul(GWNS_FF(-15737765635.0 / 3048192.0 + 2255.0 * kPi * kPi / 12.0), eta));
  a6 = ff_add(a6, ff_add(ff_mul(GWNS_FF(76055.0 / 1728.0), e2), ff_mul(GWNS_FF(-127825.0 / 1296.0), e3)));
  a6 = ff_add(a6, ff_mul(GWNS_FF(kPi * 2270.0 / 3.0), dchia));
  a6 = ff_add(a6, ff_mul(ff_add(GWNS_FF(kPi * 2270.0 / 3.0), ff_mul(GWNS_FF(-520.0 * kPi), eta)), chis));
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
  const ff al5 = ff_mul_f(a5, 3.0f);
  const ff al6 = GWNS_FF(-6848.0 / 21.0);
  const ff lpm = ff_mul_f(ff_log(c1), 3.0f);            // ln(pi M)
  const ff pre = ff_div(ff_mul(GWNS_FF(3.0 / (256.0 * kPi)), ff_mul(opq, opq)), q);   // 3/(256 pi eta)

  ff C[kBasis];
  C[0] = ff_mul(pre, ci5);
  C[1] = ff_mul(ff_mul(pre, ci3), a2);
  C[2] = ff_mul(ff_mul(pre, ci2), a3);
  C[3] = ff_mul(ff_mul(pre, ci1), a4);
  const ff lpm3 = ff_div(lpm, ff_make(3.0f));
  C[4] = ff_mul(ff_mul(pre, c1), ff_add(a6, ff_mul(al6, lpm3)));
  C[5] = ff_mul(ff_mul(pre, ff_mul(c1, c1)), a7);
  C[6] = ff_div(ff_mul(pre, al5), ff_make(3.0f));
  C[7] = ff_div(ff_mul(ff_mul(pre, c1), al6), ff_make(3.0f));
#pragma unroll
  for (int j = 0; j < kBasis; ++j) { p.Ch[j] = C[j].h; p.Cl[j] = C[j].l; }
  ff ph0 = ff_mul(pre, ff_add(a5, ff_mul(al5, lpm3)));
  ph0 = ff_sub(ph0, ff_mul(phic, GWNS_FF(1.0 / kPi)));
  ph0 = ff_add_f(ph0, -0.125f);
  p.ph0h = ph0.h;
  p.ph0l = ph0.l;

  // sky direction (float-float: it sets the arrival delays), antenna patterns in FP32
  ff sp, cp;
  ff_sincos(ff_sub(ra, ff_of(ev.gmst_f)), sp, cp);
  const ff n0 = ff_mul(cd, cp), n1 = ff_mul(cd, sp), n2 = sd;
  const float spf = sp.h, cpf = cp.h, ctf = sd.h, stf = cd.h;
  float ssf, csf;
  sincosf(psi, &ssf, &csf);
  const float X0 = spf * csf - ssf * cpf * ctf, X1 = -(cpf * csf + ssf * spf * ctf), X2 = ssf * stf;
  const float Y0 = -spf * ssf - csf * cpf * ctf, Y1 = cpf * ssf - csf * spf * ctf, Y2 = stf * csf;
  const float mcs = mc.h * (float)kMsunS;
  // K scaled by 2^70: K P ~ 1e-21 and (K P)^2 would leave FP32's normal range
  const float K = ldexpf((float)kAmp0 * sqrtf(mcs) * cbrtf(mcs) * (float)(kC / kMpcM) / dl, kKpScaleExp);
  const float ap = 0.5f * (1.0f + ci * ci);
  float hh = 0.0f;
  for (int det = 0; det < ev.n_det; ++det) {
    const float* xa = ev.xarm32[det];
    const float* ya = ev.yarm32[det];
    float xX = xa[0] * X0 + xa[1] * X1 + xa[2] * X2, xY = xa[0] * Y0 + xa[1] * Y1 + xa[2] * Y2;
    float yX = ya[0] * X0 + ya[1] * X1 + ya[2] * X2, yY = ya[0] * Y0 + ya[1] * Y1 + ya[2] * Y2;
    float fp = 0.5f * (xX * xX - xY * xY - yX * yX + yY * yY);
    float fc = xX * xY - yX * yY;
    p.kpf_re[det] = K * (fp * ap);
    p.kpf_im[det] = K * (-fc * ci);
    // tau = t_c - (r . n) / c, and its products with f_min (reduced) and df (split at a 9-bit head)
    const ff dot = ff_add(ff_add(ff_mul(ff_of(ev.vc_f[det][0]), n0), ff_mul(ff_of(ev.vc_f[det][1]), n1)),
                          ff_mul(ff_of(ev.vc_f[det][2]), n2));
    const ff tau = ff_sub(tc, dot);
    const ff a = ff_mul(tau, ff_of(ev.fmin_f));
    p.sa[det] = (a.h - rintf(a.h)) + a.l;
    const ff b = ff_mul(tau, ff_of(ev.df_f));
    const float bh = __int_as_float(__float_as_int(b.h) & (int)0xFFFF8000u);
    p.sbh[det] = bh;
    p.sbl[det] = (b.h - bh) + b.l;
    // <h|h>_det = (K P)^2 sum_{k < k_end} 4 df f^-7/3 / S, with the two 2^(+-140) scalings
    const float psum = p.k_end > 0 ? ev.hhp32[(size_t)det * ev.n_bins + p.k_end - 1] : 0.0f;
    hh += (p.kpf_re[det] * p.kpf_re[det] + p.kpf_im[det] * p.kpf_im[det]) * psum;
  }
  p.hh_f = hh;
}

}  // namespace gwns
