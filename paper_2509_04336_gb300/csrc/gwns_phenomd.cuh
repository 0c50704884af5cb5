// gwns_phenomd.cuh -- IMRPhenomD-form waveform on the device (the paper's analyses use
// IMRPhenomD, Sec. 3.3).  Functional form of IMRPhenomD with a stated form-only coefficient
// table (the same table as the oracle's; the published calibration is not used).
//
// With x = M f (M the total mass in seconds) the phase, without 2 pi f t_c - 2 phi_c - pi/4, is
//   inspiral (x < 0.018):  TaylorF2 + (3/4 s2 x^(4/3) + 3/5 s3 x^(5/3) + 1/2 s4 x^2) / eta
//   intermediate (x < fRD/2): (b0 + b1 x + b2 ln x - b3/(3 x^3)) / eta
//   merger-ringdown: (a0 + a1 x - a2/x + 4/3 a3 x^(3/4) + a4 atan((x - a5 fRD)/fd)) / eta
// with (b0, b1) and (a0, a1) fixed by continuity of the phase and its slope at the boundaries.
// Each region is regrouped over per-bin basis functions of f, so only coefficients depend on
// theta.  Basis layout (14 functions per bin):
//   0..7 the TaylorF2 basis (f^-5/3, f^-1, f^-2/3, f^-1/3, f^1/3, f^2/3, ln f, f^1/3 ln f),
//   8 f^4/3, 9 f^5/3, 10 f^2, 11 f^-3, 12 f^3/4, 13 f.
// The amplitude is K f^-7/6 a(x): a = 1 + A2 v^2 + A3 v^3 (x < 0.014, v = (pi x)^(1/3)),
// a cubic Hermite interpolant up to the ringdown peak x_p, then
// g1 g3 fd / ((x - fRD)^2 + (g3 fd)^2) exp(-g2 (x - fRD)/(g3 fd)); a = 0 above x = 0.2.
// fRD and fd come from the Kerr (2,2,0) quasi-normal-mode fit of Berti, Cardoso & Will 2006 at
// the remnant spin of Rezzolla et al. 2008 and a remnant mass 1 - (e1 eta + e2 eta^2).
#pragma once

#include "gwns_model.cuh"

namespace gwns {

constexpr int kBasisPD = 14;

// form-only table
constexpr double kPdXIns = 0.018, kPdXAmpIns = 0.014, kPdXCut = 0.2;
constexpr double kPdS2 = 50.0, kPdS3 = -100.0, kPdS4 = 40.0;
constexpr double kPdB2 = 1.0, kPdB3 = 1.0e-5;
constexpr double kPdA2 = 0.01, kPdA3 = 0.5, kPdA4 = 0.05, kPdA5 = 1.0;
constexpr double kPdG1 = 0.006, kPdG2 = 0.9, kPdG3 = 1.3;
constexpr double kPdE1 = 0.0572, kPdE2 = 0.498;
// v1 = (pi x_ins)^(1/3) and its logarithm (x_ins = 0.018)
constexpr double kPdV1 = 0.3838316585355026, kPdLnV1 = -0.957551211745524;
constexpr double kLnPi = 1.1447298858494002;

// Number of bins with f_k < f_b.
__device__ inline int bins_strictly_below(double f_min, double df, int n_bins, double f_b) {
  if (!(f_b > f_min)) return 0;
  double x = floor((f_b - f_min) * (1.0 / df));
  long k = (long)fmin(x, (double)n_bins);
  while (k + 1 <= n_bins - 1 && f_min + df * (double)(k + 1) < f_b) ++k;
  while (k >= 0 && (k > n_bins - 1 || f_min + df * (double)k >= f_b)) --k;
  return (int)(k + 1);
}

// Region coefficients, continuity constants and amplitude parameters.  Inputs: the TaylorF2
// part already in p (C[0..7], phase0 with the -phi_c/pi - 1/8 terms, k_end of TaylorF2 to be
// replaced), eta, delta, chi_s, chi_a, the PN coefficients a[], al[], c1 = (pi M)^(1/3),
// lpm = ln(pi M), q, chi1, chi2, phic.  FAST selects FP32 for what only scales the amplitude
// or enters the phase at the 1e-8 level (ringdown fit powers, x2^(3/4), atan at x2).
template <bool FAST>
__device__ void phenomd_extra(const EventDev& ev, WalkerParams& p, PhenomExtra& e, double eta,
                                     double delta, double chis, double chia, const double* a, const double* al,
                                     double c1, double lpm, double q, double chi1, double chi2, double phic) {
  const double inv2pe = 1.0 / (2.0 * kPi * eta);
  const double piM = c1 * c1 * c1;
  const double M = piM * (1.0 / kPi);
  const double M13 = c1 * (1.0 / 1.4645918875615231);   // M^(1/3) = (pi M)^(1/3) / pi^(1/3)
  const double lnM = lpm - kLnPi;
  // ringdown frequency and damping (units of 1/M)
  const double at = (chi1 + chi2 * q * q) / (1.0 + q * q);
  const double af = at + at * eta * (-0.1229 * at + 0.4537 * eta - 2.8904) +
                    eta * (2.0 * 1.7320508075688772 + -3.5171 * eta + 2.5763 * eta * eta);
  const double mfin = 1.0 - (kPdE1 * eta + kPdE2 * eta * eta);
  double om, qf;
  if (FAST) {
    om = 1.5251 - 1.1568 * (double)powf((float)(1.0 - af), 0.1292f);
    qf = 0.7000 + 1.4187 * (double)powf((float)(1.0 - af), -0.4990f);
  } else {
    om = 1.5251 - 1.1568 * pow(1.0 - af, 0.1292);
    qf = 0.7000 + 1.4187 * pow(1.0 - af, -0.4990);
  }
  const double frd = om / (2.0 * kPi * mfin);
  const double fd = frd / (2.0 * qf);
  // inspiral at x1 (value and slope): TaylorF2 part from constant powers of v1
  double vk[8];
  const double vinv5 = 1.0 / (kPdV1 * kPdV1 * kPdV1 * kPdV1 * kPdV1);
  for (int k = 0; k < 8; ++k) vk[k] = (k == 0) ? vinv5 : vk[k - 1] * kPdV1;
  double s = 0.0, ds = 0.0;
  for (int k = 0; k < 8; ++k) {
    double t = a[k] + al[k] * kPdLnV1;
    s += t * vk[k];
    ds += vk[k] * ((k - 5) * t + al[k]);
  }
  const double x1 = kPdXIns;
  const double c = 3.0 / (128.0 * eta);
  double p1 = c * s + (0.75 * kPdS2 * 0.004717334509576015 + 0.6 * kPdS3 * 0.001236291381957598 +
                       0.5 * kPdS4 * x1 * x1) / eta;
  double dp1 = c * ds / (3.0 * x1) +
               (kPdS2 * 0.2620741394208897 + kPdS3 * 0.06868285455319992 + kPdS4 * x1) / eta;
  const double b1 = eta * dp1 - kPdB2 / x1 - kPdB3 / (x1 * x1 * x1 * x1);
  const double b0 = eta * p1 - b1 * x1 - kPdB2 * (-4.017383521085972) + kPdB3 / (3.0 * x1 * x1 * x1);
  // intermediate at x2, merger-ringdown continuity
  const double x2 = 0.5 * frd;
  const double lnx2 = log(x2);
  const double ix2 = 1.0 / x2;
  const double pint2 = (b0 + b1 * x2 + kPdB2 * lnx2 - kPdB3 / 3.0 * ix2 * ix2 * ix2) / eta;
  const double dpint2 = (b1 + kPdB2 * ix2 + kPdB3 * ix2 * ix2 * ix2 * ix2) / eta;
  double x2p34, x2m14, l2;
  if (FAST) {
    x2p34 = (double)powf((float)x2, 0.75f);
    x2m14 = (double)powf((float)x2, -0.25f);
    l2 = kPdA4 * (double)atanf((float)((x2 - kPdA5 * frd) / fd));
  } else {
    x2p34 = pow(x2, 0.75);
    x2m14 = pow(x2, -0.25);
    l2 = kPdA4 * atan((x2 - kPdA5 * frd) / fd);
  }
  const double dl2 = kPdA4 * fd / ((x2 - kPdA5 * frd) * (x2 - kPdA5 * frd) + fd * fd);
  const double a1 = eta * dpint2 - kPdA2 * ix2 * ix2 - kPdA3 * x2m14 - dl2;
  const double a0 = eta * pint2 - a1 * x2 + kPdA2 * ix2 - (4.0 / 3.0) * kPdA3 * x2p34 - l2;
  // region coefficients in f, in cycles
  const double M2 = M * M;
  e.Cx[0] = 0.75 * kPdS2 * M * M13 * inv2pe;             // f^4/3
  e.Cx[1] = 0.6 * kPdS3 * M * M13 * M13 * inv2pe;        // f^5/3
  e.Cx[2] = 0.5 * kPdS4 * M2 * inv2pe;                   // f^2
  e.Cx[3] = kPdB2 * inv2pe;                              // ln f
  e.Cx[4] = -kPdB3 / (3.0 * M2 * M) * inv2pe;            // f^-3
  e.Cx[5] = b1 * M * inv2pe;                             // f
  e.Cx[6] = -kPdA2 / M * inv2pe;                         // f^-1
  double M34;
  if (FAST) M34 = (double)powf((float)M, 0.75f); else M34 = pow(M, 0.75);
  e.Cx[7] = (4.0 / 3.0) * kPdA3 * M34 * inv2pe;          // f^3/4
  e.Cx[8] = a1 * M * inv2pe;                             // f
  const double tail = -phic / kPi - 0.125;
  e.ph0_int = (b0 + kPdB2 * lnM) * inv2pe + tail;
  e.ph0_mr = a0 * inv2pe + tail;
  // region boundaries as bin indices
  e.k1 = bins_strictly_below(ev.f_min, ev.df, ev.n_bins, x1 / M);
  e.k2 = bins_strictly_below(ev.f_min, ev.df, ev.n_bins, x2 / M);
  p.k_end = bins_below(ev.f_min, ev.df, ev.n_bins, kPdXCut / M);
  // amplitude shape
  const double A2 = -323.0 / 224.0 + 451.0 * eta / 168.0;
  const double A3 = 27.0 * delta * chia / 8.0 + (27.0 / 8.0 - 11.0 * eta / 6.0) * chis;
  const double gd = kPdG3 * fd;
  const double xa = kPdXAmpIns;
  const double xp = fabs(frd + gd * (sqrt(1.0 - kPdG2 * kPdG2) - 1.0) / kPdG2);
  const double va = (FAST ? (double)cbrtf((float)(kPi * xa)) : cbrt(kPi * xa));
  const double y0 = 1.0 + A2 * va * va + A3 * va * va * va;
  const double d0 = (2.0 * A2 * va + 3.0 * A3 * va * va) * va / (3.0 * xa);
  const double dp = xp - frd;
  const double ex = FAST ? (double)expf((float)(-kPdG2 * dp / gd)) : exp(-kPdG2 * dp / gd);
  const double den = dp * dp + gd * gd;
  const double y1 = kPdG1 * gd / den * ex;
  const double d1 = y1 * (-2.0 * dp / den - kPdG2 / gd);
  const double span = xp - xa;
  e.ka = bins_strictly_below(ev.f_min, ev.df, ev.n_bins, xa / M);
  e.kp = bins_strictly_below(ev.f_min, ev.df, ev.n_bins, xp / M);
  e.A2 = A2; e.A3 = A3; e.c13 = c1; e.M = M; e.xa = xa; e.inv_span = 1.0 / span;
  e.hy0 = y0; e.hd0 = span * d0;
  e.hc2 = 3.0 * (y1 - y0) - 2.0 * span * d0 - span * d1;
  e.hc3 = 2.0 * (y0 - y1) + span * d0 + span * d1;
  e.frd = frd; e.gd = gd; e.g1gd = kPdG1 * gd; e.g2_gd = kPdG2 / gd;
  e.at_scale = kPdA4 * inv2pe; e.at_c = kPdA5 * frd; e.at_inv = 1.0 / fd;
  e.A2f = (float)e.A2; e.A3f = (float)e.A3; e.c13f = (float)e.c13; e.Mf = (float)e.M; e.xaf = (float)e.xa;
  e.inv_spanf = (float)e.inv_span; e.hy0f = (float)e.hy0; e.hd0f = (float)e.hd0; e.hc2f = (float)e.hc2;
  e.hc3f = (float)e.hc3; e.frdf = (float)e.frd; e.gdf = (float)e.gd; e.g1gdf = (float)e.g1gd;
  e.g2_gdf = (float)e.g2_gd; e.at_scalef = (float)e.at_scale; e.at_cf = (float)e.at_c;
  e.at_invf = (float)e.at_inv;
}

// amplitude shape a(x) at bin k (x = M f_k)
__device__ __forceinline__ double pd_amp_f64(const PhenomExtra& e, int k, double f, double f13) {
  if (k < e.ka) {
    double v = e.c13 * f13;
    return 1.0 + e.A2 * v * v + e.A3 * v * v * v;
  }
  double x = e.M * f;
  if (k < e.kp) {
    double s = (x - e.xa) * e.inv_span;
    return e.hy0 + s * (e.hd0 + s * (e.hc2 + s * e.hc3));
  }
  double d = x - e.frd;
  return e.g1gd / (d * d + e.gd * e.gd) * exp(-e.g2_gd * d);
}

__device__ __forceinline__ float pd_amp_f32(const PhenomExtra& e, int k, float f, float f13) {
  if (k < e.ka) {
    float v = e.c13f * f13;
    return 1.0f + e.A2f * v * v + e.A3f * v * v * v;
  }
  float x = e.Mf * f;
  if (k < e.kp) {
    float s = (x - e.xaf) * e.inv_spanf;
    return e.hy0f + s * (e.hd0f + s * (e.hc2f + s * e.hc3f));
  }
  float d = x - e.frdf;
  return __fdividef(e.g1gdf, d * d + e.gdf * e.gdf) * __expf(-e.g2_gdf * d);
}

struct AccPD64 {
  double re[kMaxDet], im[kMaxDet], hh[kMaxDet];
  __device__ void zero() { for (int i = 0; i < kMaxDet; ++i) { re[i] = 0.0; im[i] = 0.0; hh[i] = 0.0; } }
};
struct AccPD32 {
  float re[kMaxDet], im[kMaxDet], hh[kMaxDet], cre[kMaxDet], cim[kMaxDet], chh[kMaxDet];
  __device__ void zero() {
    for (int i = 0; i < kMaxDet; ++i) { re[i] = im[i] = hh[i] = cre[i] = cim[i] = chh[i] = 0.f; }
  }
};

// FP64 path.
template <int NDET>
__device__ __forceinline__ void pd_accumulate_f64(const EventDev& ev, const WalkerParams& p, const PhenomExtra& e,
                                                  int k, AccPD64& acc) {
  const double* g = ev.basis64 + (size_t)k * kBasisPD;
  const double f = ev.f_min + ev.df * (double)k;
  double phi;
  if (k < e.k1) {
    phi = p.phase0;
#pragma unroll
    for (int j = 0; j < 8; ++j) phi = fma(p.C[j], g[j], phi);
    phi = fma(e.Cx[0], g[8], phi);
    phi = fma(e.Cx[1], g[9], phi);
    phi = fma(e.Cx[2], g[10], phi);
  } else if (k < e.k2) {
    phi = fma(e.Cx[3], g[6], e.ph0_int);
    phi = fma(e.Cx[4], g[11], phi);
    phi = fma(e.Cx[5], g[13], phi);
  } else {
    phi = fma(e.Cx[6], g[1], e.ph0_mr);
    phi = fma(e.Cx[7], g[12], phi);
    phi = fma(e.Cx[8], g[13], phi);
    phi += e.at_scale * atan((e.M * f - e.at_c) * e.at_inv);
  }
  const double amp = pd_amp_f64(e, k, f, g[4]);
  const double amp2 = amp * amp;
#pragma unroll
  for (int det = 0; det < NDET; ++det) {
    double ph = fma(p.tau[det], f, phi);
    double s, c;
    sincos_phase_f64(ph, &s, &c);
    const double2 z = ev.z64[(size_t)det * ev.n_bins + k];
    const double ax = amp * z.x, ay = amp * z.y;
    // amp z exp(-2 pi i ph), accumulated by two FMAs a component
    acc.re[det] = fma(ax, c, fma(ay, s, acc.re[det]));
    acc.im[det] = fma(ay, c, fma(-ax, s, acc.im[det]));
    acc.hh[det] = fma(amp2, ev.gw64[(size_t)det * ev.n_bins + k], acc.hh[det]);
  }
}

// Mixed path with the FP64 phase.
template <int NDET>
__device__ __forceinline__ void pd_accumulate_mixed(const EventDev& ev, const WalkerParams& p, const PhenomExtra& e,
                                                    int k, AccPD32& acc) {
  const double* g = ev.basis64 + (size_t)k * kBasisPD;
  const double f = ev.f_min + ev.df * (double)k;
  double phi;
  float extra = 0.f;
  if (k < e.k1) {
    phi = p.phase0;
#pragma unroll
    for (int j = 0; j < 8; ++j) phi = fma(p.C[j], g[j], phi);
    phi = fma(e.Cx[0], g[8], phi);
    phi = fma(e.Cx[1], g[9], phi);
    phi = fma(e.Cx[2], g[10], phi);
  } else if (k < e.k2) {
    phi = fma(e.Cx[3], g[6], e.ph0_int);
    phi = fma(e.Cx[4], g[11], phi);
    phi = fma(e.Cx[5], g[13], phi);
  } else {
    phi = fma(e.Cx[6], g[1], e.ph0_mr);
    phi = fma(e.Cx[7], g[12], phi);
    phi = fma(e.Cx[8], g[13], phi);
    extra = e.at_scalef * atanf((e.Mf * (float)f - e.at_cf) * e.at_invf);
  }
  const float ff = (float)f;
  const float amp = pd_amp_f32(e, k, ff, ev.basis_ff[(size_t)4 * ev.n_bins + k].x);
#pragma unroll
  for (int det = 0; det < NDET; ++det) {
    double ph = fma(p.tau[det], f, phi);
    float r = (float)(ph - rint(ph)) + extra;
    float s, c;
    sincospif(2.0f * r, &s, &c);
    float2 z = ev.z32[(size_t)det * ev.n_bins + k];
    kahan_add(acc.re[det], acc.cre[det], amp * fmaf(z.x, c, z.y * s));
    kahan_add(acc.im[det], acc.cim[det], amp * fmaf(z.y, c, -z.x * s));
    kahan_add(acc.hh[det], acc.chh[det], amp * amp * ev.gw32[(size_t)det * ev.n_bins + k]);
  }
}

// Mixed path with the float-float phase.
__device__ __forceinline__ void ff_term(float& sh, float& sl, float ch, float cl, float2 g) {
  float q = ch * g.x;
  float e = fmaf(ch, g.x, -q);
  e = fmaf(ch, g.y, e);
  e = fmaf(cl, g.x, e);
  float t = sh + q;
  float bb = t - sh;
  float err = (sh - (t - bb)) + (q - bb);
  sh = t;
  sl += err + e;
}

template <int NDET>
__device__ __forceinline__ void pd_accumulate_ff(const EventDev& ev, const WalkerParams& p, const PhenomExtra& e, int k,
                                                 AccPD32& acc) {
  const float2* g = ev.basis_ff + k;
  const size_t gs = (size_t)ev.n_bins;
  const float ff = g[13 * gs].x;   // f (exact on the grids used: f_min + k df in FP32)
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
  const float r0 = (sh - rintf(sh)) + sl + extra;
  const float amp = pd_amp_f32(e, k, ff, g[4 * gs].x);
  const float amp2 = amp * amp;
  const float kf = (float)k;
#pragma unroll
  for (int det = 0; det < NDET; ++det) {
    float kb = kf * p.sbh[det];
    float x = kb - rintf(kb);
    float ph = (r0 + p.sa[det]) + x + kf * p.sbl[det];
    ph = ph - rintf(ph);
    float s, c;
    sincos_turn_sfu(ph, &s, &c);
    float2 z = ev.z32[(size_t)det * ev.n_bins + k];
    kahan_add(acc.re[det], acc.cre[det], amp * fmaf(z.x, c, z.y * s));
    kahan_add(acc.im[det], acc.cim[det], amp * fmaf(z.y, c, -z.x * s));
    // template power: positive terms, no cancellation -- a plain FP32 sum per lane (the lanes'
    // sums are combined with error-free additions)
    acc.hh[det] = fmaf(amp2, ev.gw32[(size_t)det * ev.n_bins + k], acc.hh[det]);
  }
}

}  // namespace gwns
