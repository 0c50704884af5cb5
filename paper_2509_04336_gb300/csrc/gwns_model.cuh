// gwns_model.cuh -- device-side model of the frequency-domain GW likelihood (Sec. 3.3)
// and of the unit-cube prior transforms (Sec. 3.4, Table 1) used by every kernel.
//
// Factorisation used on the GPU (algebraically identical to the plain definition):
//   h_det(f_k) = K f_k^(-7/6) P_det exp(-2 pi i Phi_det(f_k)),   P_det = F+ (1+ci^2)/2 - i Fx ci
//   Phi_det(f) = sum_j C_j g_j(f) + phase0 + (t_c + dt_det) f        [cycles]
//   g = (f^-5/3, f^-1, f^-2/3, f^-1/3, f^1/3, f^2/3, ln f, f^1/3 ln f): the TaylorF2 PN
//   series  3/(128 eta v^5) sum_k (a_k + a^l_k ln v) v^k  with v^k = (pi M)^(k/3) f^(k/3)
//   and ln v = (ln(pi M) + ln f)/3, regrouped by powers of f.  The g_j are per-bin
//   constants shared by every walker; only the C_j depend on theta.
//   <d|h_det> = Re[K P_det S_det],   S_det = sum_k z_k exp(-2 pi i Phi_det(f_k)),
//   z_k = 4 df conj(d_k) f_k^(-7/6) / S_n(f_k)      (per-bin constant)
//   <h|h>_det = K^2 |P_det|^2 sum_{k < k_end} 4 df f_k^(-7/3) / S_n(f_k)   (prefix sums)
//   ln L = -1/2 (sum <d|d> - 2 sum <d|h> + sum <h|h>);  use_ratio: sum <d|h> - 1/2 sum <h|h>.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <math.h>

namespace gwns {

constexpr int kParams = 11;
constexpr int kMaxDet = 4;
constexpr int kMaxDim = 11;
constexpr int kBasis = 8;        // TaylorF2 phase basis

// SI constants: exact c, IAU 2015 nominal solar mass parameter, IAU parsec.
constexpr double kC = 299792458.0;
constexpr double kGMsun = 1.32712440018e20;
constexpr double kMsunS = kGMsun / (kC * kC * kC);
constexpr double kMpcM = 3.085677581491367e22;
constexpr double kPi = 3.141592653589793;
constexpr double kEulerGamma = 0.5772156649015329;
constexpr double kLn4 = 1.3862943611198906;
constexpr double kSix15 = 14.696938456699069;   // 6^(3/2)
constexpr double kAmp0 = 0.21278751013966343;   // sqrt(5/24) pi^(-2/3)

struct EventDev;
struct WalkerParams;
struct PhenomExtra;
// IMRPhenomD-form constants of a proposal (gwns_phenomd.cuh), called by the setups below.
template <bool FAST>
__device__ void phenomd_extra(const EventDev& ev, WalkerParams& p, PhenomExtra& e, double eta, double delta,
                              double chis, double chia, const double* a, const double* al, double c1, double lpm,
                              double q, double chi1, double chi2, double phic);

enum PriorKind { kUniform = 0, kPowerLaw = 1, kSine = 2, kCosine = 3, kFixed = 4 };

// One prior entry with its inverse-CDF constants precomputed on the host.
//   uniform:  x = lo + u*w                     (w = hi - lo)
//   powerlaw: x = (A + u*B)^(1/(alpha+1))      (A = lo^(alpha+1), B = hi^(alpha+1) - A, e = alpha+1)
//   sine:     cos x = A - u*B                  (A = cos lo, B = cos lo - cos hi)
//   cosine:   sin x = A + u*B                  (A = sin lo, B = sin hi - sin lo)
//   fixed:    x = value (cosv = cos value, sinv = sin value)
struct PriorDev {
  int kind;
  int periodic;
  double lo, hi, w, A, B, e, value, cosv, sinv;
  // float-float copies (h, l) of lo, w, A, B, value, cos value, sin value
  float lo_f[2], w_f[2], A_f[2], B_f[2], v_f[2], cv_f[2], sv_f[2];
  float einv_f;   // 1 / (alpha + 1) of a power law
};

// Device copy of one event and its sampler configuration.
struct EventDev {
  int n_det, n_bins, n_dim, use_ratio;
  int waveform, n_basis;               // 0 TaylorF2 (8 basis functions), 1 IMRPhenomD form (14)
  double f_min, df, gmst;
  double dd_total;                     // sum_det <d|d>
  double vertex[kMaxDet][3], xarm[kMaxDet][3], yarm[kMaxDet][3];
  float xarm32[kMaxDet][3], yarm32[kMaxDet][3];
  PriorDev prior[kParams];
  int dim_param[kMaxDim];              // physical index of each sampled dimension
  int param_dim[kParams];              // sampled dimension of each parameter (-1: fixed)
  const double* basis64;               // [n_bins][kBasis]
  const float2* basis_ff;              // [n_basis][n_bins] (hi, lo) float-float copy of basis64,
                                       // term-major: a warp's loads of one term are contiguous
  const double2* z64;                  // [n_det][n_bins]
  const float2* z32;                   // [n_det][n_bins]
  const double* hh_prefix;             // [n_det][n_bins] inclusive prefix sums of 4 df f^-7/3 / S
  const double* gw64;                  // [n_det][n_bins] 4 df f^-7/3 / S (per-bin template power)
  const float* gw32;                   // [n_det][n_bins] FP32 copy scaled by 1/gw32_unscale (a power
                                       //   of two: the weights reach ~1e43, beyond FP32's range)
  double gw32_unscale;
  // float-float copies of the geometry for the float-float proposal setup
  int ff_setup;                        // 1 when every sampled prior has a float-float transform
  float dd_f[2];                       // sum_det <d|d> as a float pair
  float hh_unscale_f;                  // gw32_unscale * 2^-140 (IMRPhenomD template power, FP32)
  const float* hhp32;                  // [n_det][n_bins] hh_prefix * 2^-140 (FP32 range)
  float vc_f[kMaxDet][3][2];           // detector vertex / c [s]
  float fmin_f[2], df_f[2], gmst_f[2];
  // relative binning (ns_relbin_set; rb_nb = 0: the full likelihood)
  int rb_nb;                           // coarse bins
  const int32_t* rb_edges;             // [rb_nb + 1] grid-bin edges, rb_edges[rb_nb] = n_bins
  const float2* rb_q0;                 // [n_det][rb_nb] f^(-7/6) / (h0 2^70) at the edges
  const float2* rb_a;                  // [n_det][rb_nb][2] summary data A0, A1
  const float4* rb_b;                  // [n_det][rb_nb] summary data (B0, B1, B2, 0)
};

// The IMRPhenomD-form part of the per-walker constants (in cycles).
struct PhenomExtra {
  double Cx[9];         // ins: f^4/3 f^5/3 f^2 | int: ln f, f^-3, f | mr: f^-1, f^3/4, f
  double ph0_int, ph0_mr;
  float Cxh[9], Cxl[9];
  float ph0_int_h, ph0_int_l, ph0_mr_h, ph0_mr_l;
  int k1, k2, ka, kp;   // first bins of: intermediate phase, MR phase, intermediate amp, MR amp
  // amplitude shape and the ringdown atan term, FP64 (FP64 path) and FP32 (mixed paths)
  double A2, A3, c13, M, xa, inv_span, hy0, hd0, hc2, hc3, frd, gd, g1gd, g2_gd, at_scale, at_c, at_inv;
  float A2f, A3f, c13f, Mf, xaf, inv_spanf, hy0f, hd0f, hc2f, hc3f, frdf, gdf, g1gdf, g2_gdf, at_scalef, at_cf,
      at_invf;
};

// Per-walker constants of one likelihood evaluation.  The float fields are the
// float-float split used by the FP32-pipe phase path (make_ff).
struct WalkerParams {
  double C[kBasis];
  double phase0;
  double tau[kMaxDet];
  double kp_re[kMaxDet], kp_im[kMaxDet];
  double hh;
  int k_end;
  int pad;
  float Ch[kBasis], Cl[kBasis];        // C_j = Ch + Cl
  float ph0h, ph0l;                    // phase0 = ph0h + ph0l
  float sa[kMaxDet];                   // frac(tau f_min)                       [cycles]
  float sbh[kMaxDet], sbl[kMaxDet];    // tau df = sbh + sbl, sbh with 9 significant bits
  float kpf_re[kMaxDet], kpf_im[kMaxDet];   // K P_det * 2^70 (FP32 range), float-float assembly
  float hh_f;                          // <h|h> (TaylorF2), float-float assembly
  PhenomExtra pd;                      // IMRPhenomD-form regions (unused for TaylorF2)
};

constexpr int kKpScaleExp = 70;        // K P ~ 1e-21: scaled by 2^70 into FP32's comfortable range

// ---------------------------------------------------------------- Philox4x64-10
// Salmon, Moraes, Dror & Shaw 2011: 10 rounds of multiply-xor with a Weyl key schedule.
struct Philox4 { uint64_t v[4]; };

__device__ __forceinline__ Philox4 philox4x64(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                              uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
    uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
    uint64_t n0 = hi1 ^ c1 ^ k0;
    uint64_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += W0; k1 += W1;
  }
  Philox4 r; r.v[0] = c0; r.v[1] = c1; r.v[2] = c2; r.v[3] = c3;
  return r;
}

// floor(x * n / 2^64)
__device__ __forceinline__ uint64_t rand_index(uint64_t x, uint64_t n) { return __umul64hi(x, n); }
// uniform on (0, 1): ((x >> 12) + 1/2) / 2^52
__device__ __forceinline__ double rand_open_unit(uint64_t x) {
  return __dmul_rn(__dadd_rn((double)(x >> 12), 0.5), 2.220446049250313e-16);
}

// ---------------------------------------------------------------- prior transform
// Physical theta [11] from unit-cube u [D], plus cos(theta_jn), sin(dec), cos(dec), which
// the sine / cosine priors give without inverse trigonometry.
__device__ inline void unit_to_theta(const EventDev& ev, const double* u, double* th,
                                     double* cos_iota, double* sin_dec, double* cos_dec) {
  int d = 0;
  double ci = 0.0, sd = 0.0, cd = 1.0;
  bool have_ci = false, have_dec = false;
  for (int i = 0; i < kParams; ++i) {
    const PriorDev& p = ev.prior[i];
    double x;
    if (p.kind == kFixed) {
      x = p.value;
      if (i == 5) { ci = p.cosv; have_ci = true; }
      if (i == 10) { sd = p.sinv; cd = p.cosv; have_dec = true; }
    } else {
      double v = u[d++];
      if (p.kind == kUniform) {
        x = __dadd_rn(p.lo, __dmul_rn(v, p.w));
      } else if (p.kind == kPowerLaw) {
        double y = __dadd_rn(p.A, __dmul_rn(v, p.B));
        x = (p.e == 3.0) ? cbrt(y) : pow(y, 1.0 / p.e);
      } else if (p.kind == kSine) {
        double c = __dsub_rn(p.A, __dmul_rn(v, p.B));
        c = fmin(1.0, fmax(-1.0, c));
        x = acos(c);
        if (i == 5) { ci = c; have_ci = true; }
      } else {  // cosine
        double s = __dadd_rn(p.A, __dmul_rn(v, p.B));
        s = fmin(1.0, fmax(-1.0, s));
        x = asin(s);
        if (i == 10) { sd = s; cd = sqrt(fmax(0.0, (1.0 - s) * (1.0 + s))); have_dec = true; }
      }
    }
    th[i] = x;
  }
  if (!have_ci) ci = cos(th[5]);
  if (!have_dec) { sincos(th[10], &sd, &cd); }
  *cos_iota = ci; *sin_dec = sd; *cos_dec = cd;
}

// ---------------------------------------------------------------- TaylorF2 setup
// 3.5PN aligned-spin TaylorF2 phase coefficients a_k, a^l_k (non-spinning terms of
// Buonanno et al. 2009; spin terms in the chi_s, chi_a, delta form of Khan et al. 2016).
__device__ inline void taylorf2_pn_coeffs(double eta, double delta, double chis, double chia,
                                          double a[8], double al[8]) {
  const double pi = kPi;
  double e2 = eta * eta, e3 = e2 * eta;
  a[0] = 1.0; a[1] = 0.0;
  a[2] = 3715.0 / 756.0 + 55.0 * eta / 9.0;
  a[3] = -16.0 * pi + 113.0 / 3.0 * delta * chia + (113.0 / 3.0 - 76.0 * eta / 3.0) * chis;
  a[4] = 15293365.0 / 508032.0 + 27145.0 * eta / 504.0 + 3085.0 * e2 / 72.0
       + (-405.0 / 8.0 + 200.0 * eta) * chia * chia - 405.0 / 4.0 * delta * chia * chis
       + (-405.0 / 8.0 + 5.0 * eta / 2.0) * chis * chis;
  double gso = (732985.0 / 2268.0 - 24260.0 * eta / 81.0 - 340.0 * e2 / 9.0) * chis
             + (732985.0 / 2268.0 + 140.0 * eta / 9.0) * delta * chia;
  a[5] = 38645.0 * pi / 756.0 - 65.0 * pi * eta / 9.0 - gso;
  a[6] = 11583231236531.0 / 4694215680.0 - 6848.0 * kEulerGamma / 21.0 - 640.0 * pi * pi / 3.0
       + (-15737765635.0 / 3048192.0 + 2255.0 * pi * pi / 12.0) * eta
       + 76055.0 * e2 / 1728.0 - 127825.0 * e3 / 1296.0 - 6848.0 / 21.0 * kLn4
       + pi * 2270.0 / 3.0 * delta * chia + pi * (2270.0 / 3.0 - 520.0 * eta) * chis;
  a[7] = pi * (77096675.0 / 254016.0 + 378515.0 * eta / 1512.0 - 74045.0 * e2 / 756.0)
       + (-25150083775.0 / 3048192.0 + 10566655595.0 * eta / 762048.0 - 1042165.0 * e2 / 3024.0
          + 5345.0 * e3 / 36.0) * chis
       + (-25150083775.0 / 3048192.0 + 26804935.0 * eta / 6048.0 - 1985.0 * e2 / 48.0) * delta * chia;
  for (int k = 0; k < 8; ++k) al[k] = 0.0;
  al[5] = 3.0 * a[5];
  al[6] = -6848.0 / 21.0;
}

// Number of bins with f_k <= f_cut (f_k = f_min + k df, exactly as the grid is defined).
__device__ inline int bins_below(double f_min, double df, int n_bins, double f_cut) {
  if (!(f_cut >= f_min)) return 0;
  // a first guess from the reciprocal; the two loops make the count exact
  double x = floor((f_cut - f_min) * (1.0 / df));
  long k = (long)fmin(x, (double)n_bins);
  while (k + 1 <= n_bins - 1 && f_min + df * (double)(k + 1) <= f_cut) ++k;
  while (k >= 0 && (k > n_bins - 1 || f_min + df * (double)k > f_cut)) --k;
  return (int)(k + 1);
}

// Antenna pattern (F+, Fx) and arrival delay of one detector.  F+ = D:e+, Fx = D:ex with
// D = (x x^T - y y^T)/2 reduce to projections of the arms on the wave axes X, Y.
__device__ inline void detector_response(const EventDev& ev, int det, double sp, double cp,
                                         double sdec, double cdec, double ss, double cs,
                                         double* fp, double* fc, double* dt) {
  // theta = pi/2 - dec: cos theta = sin dec, sin theta = cos dec
  double ct = sdec, st = cdec;
  double X0 = sp * cs - ss * cp * ct, X1 = -(cp * cs + ss * sp * ct), X2 = ss * st;
  double Y0 = -sp * ss - cs * cp * ct, Y1 = cp * ss - cs * sp * ct, Y2 = st * cs;
  const double* x = ev.xarm[det];
  const double* y = ev.yarm[det];
  double xX = x[0] * X0 + x[1] * X1 + x[2] * X2, xY = x[0] * Y0 + x[1] * Y1 + x[2] * Y2;
  double yX = y[0] * X0 + y[1] * X1 + y[2] * X2, yY = y[0] * Y0 + y[1] * Y1 + y[2] * Y2;
  *fp = 0.5 * (xX * xX - xY * xY - yX * yX + yY * yY);
  *fc = xX * xY - yX * yY;
  const double* r = ev.vertex[det];
  double n0 = cdec * cp, n1 = cdec * sp, n2 = sdec;
  *dt = -(r[0] * n0 + r[1] * n1 + r[2] * n2) / kC;
}

// Per-walker constants for theta (with cos iota, sin dec, cos dec supplied); WF 1 adds the
// IMRPhenomD-form regions.
template <int WF>
__device__ inline void taylorf2_setup(const EventDev& ev, const double* th, double ci, double sdec,
                                      double cdec, WalkerParams& p) {
  double mc = th[0], q = th[1], chi1 = th[2], chi2 = th[3], dl = th[4];
  double psi = th[6], phic = th[7], tc = th[8], ra = th[9];
  double eta = q / ((1.0 + q) * (1.0 + q));
  double mtot = mc * pow(eta, -0.6);
  double delta = (1.0 - q) / (1.0 + q);
  double chis = 0.5 * (chi1 + chi2), chia = 0.5 * (chi1 - chi2);
  double piM = kPi * (mtot * kMsunS);
  double f_cut = 1.0 / (kSix15 * piM);
  p.k_end = bins_below(ev.f_min, ev.df, ev.n_bins, f_cut);

  double a[8], al[8];
  taylorf2_pn_coeffs(eta, delta, chis, chia, a, al);
  double lpm = log(piM);
  double c1 = cbrt(piM);
  double ci1 = 1.0 / c1;
  double ci2 = ci1 * ci1, ci3 = ci2 * ci1, ci5 = ci3 * ci2;
  double pre = 3.0 / (256.0 * kPi * eta);      // 3/(128 eta) / (2 pi): cycles
  p.C[0] = pre * ci5 * a[0];
  p.C[1] = pre * ci3 * a[2];
  p.C[2] = pre * ci2 * a[3];
  p.C[3] = pre * ci1 * a[4];
  p.C[4] = pre * c1 * (a[6] + al[6] * lpm / 3.0);
  p.C[5] = pre * c1 * c1 * a[7];
  p.C[6] = pre * al[5] / 3.0;
  p.C[7] = pre * c1 * al[6] / 3.0;
  p.phase0 = pre * (a[5] + al[5] * lpm / 3.0) - phic / kPi - 0.125;
  if (WF == 1) phenomd_extra<false>(ev, p, p.pd, eta, delta, chis, chia, a, al, c1, lpm, q, chi1, chi2, phic);

  // restricted amplitude K = sqrt(5/24) pi^(-2/3) (G Mc/c^3)^(5/6) / (d_L/c)
  double mcs = mc * kMsunS;
  double K = kAmp0 * sqrt(mcs) * cbrt(mcs) * kC / (dl * kMpcM);

  double sp, cp, ss, cs;
  sincos(ra - ev.gmst, &sp, &cp);
  sincos(psi, &ss, &cs);
  double ap = 0.5 * (1.0 + ci * ci);
  double hh = 0.0;
  for (int det = 0; det < ev.n_det; ++det) {
    double fp, fc, dt;
    detector_response(ev, det, sp, cp, sdec, cdec, ss, cs, &fp, &fc, &dt);
    double pre_re = fp * ap, pre_im = -fc * ci;
    p.kp_re[det] = K * pre_re;
    p.kp_im[det] = K * pre_im;
    p.tau[det] = tc + dt;
    double psum = (WF == 0 && p.k_end > 0) ? ev.hh_prefix[(size_t)det * ev.n_bins + p.k_end - 1] : 0.0;
    hh += K * K * (pre_re * pre_re + pre_im * pre_im) * psum;
  }
  p.hh = hh;
}

// Float-float split of the per-walker constants.  k * sbh is exact in FP32 for k < 2^15
// because sbh keeps 9 significant bits, so the time-shift phase k tau df is reduced exactly.
template <int WF>
__device__ inline void make_ff(const EventDev& ev, WalkerParams& p) {
  for (int j = 0; j < kBasis; ++j) {
    float h = (float)p.C[j];
    p.Ch[j] = h;
    p.Cl[j] = (float)(p.C[j] - (double)h);
  }
  float h0 = (float)p.phase0;
  p.ph0h = h0;
  p.ph0l = (float)(p.phase0 - (double)h0);
  if (WF == 1) {
    PhenomExtra& e = p.pd;
    for (int j = 0; j < 9; ++j) {
      float h = (float)e.Cx[j];
      e.Cxh[j] = h;
      e.Cxl[j] = (float)(e.Cx[j] - (double)h);
    }
    float h = (float)e.ph0_int;
    e.ph0_int_h = h;
    e.ph0_int_l = (float)(e.ph0_int - (double)h);
    h = (float)e.ph0_mr;
    e.ph0_mr_h = h;
    e.ph0_mr_l = (float)(e.ph0_mr - (double)h);
  }
  p.hh_f = (float)p.hh;
  for (int det = 0; det < ev.n_det; ++det) {
    p.kpf_re[det] = (float)ldexp(p.kp_re[det], kKpScaleExp);
    p.kpf_im[det] = (float)ldexp(p.kp_im[det], kKpScaleExp);
    double a = p.tau[det] * ev.f_min;
    p.sa[det] = (float)(a - rint(a));
    double b = p.tau[det] * ev.df;
    float bh = __int_as_float(__float_as_int((float)b) & (int)0xFFFF8000u);
    p.sbh[det] = bh;
    p.sbl[det] = (float)(b - (double)bh);
  }
}

// ---------------------------------------------------------------- lean setup (mixed paths)
// The mixed paths need FP64 only for what moves the phase: chirp mass, mass ratio, spins,
// coalescence phase and time, and the arrival delays.  Amplitude, inclination, polarisation
// and the antenna patterns only scale h and are computed in FP32.  Roots are FP32 seeds with
// two FP64 Newton steps each (quadratic convergence from ~1e-7 to below 1 ulp), which keeps
// the FP64 instruction count and latency of a proposal low.

// a^(-1/3) for a > 0: w <- w (4 - a w^3) / 3.
__device__ __forceinline__ double rcbrt_newton(double a) {
  double w = (double)rcbrtf((float)a);
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    double w3 = w * w * w;
    w = w * (4.0 - a * w3) * (1.0 / 3.0);
  }
  return w;
}

// a^(-1/5) for a > 0: z <- z (6 - a z^5) / 5.
__device__ __forceinline__ double rfifth_newton(double a) {
  double z = (double)__powf((float)a, -0.2f);
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    double z2 = z * z;
    double z5 = z2 * z2 * z;
    z = z * (6.0 - a * z5) * 0.2;
  }
  return z;
}

// The sampled physical quantities a mixed-precision likelihood needs, from unit-cube u.
struct LeanTheta {
  double mc, q, chi1, chi2, phic, tc, ra, sdec, cdec;
  float dl, ci, psi;
};

__device__ inline void unit_to_lean(const EventDev& ev, const double* u, LeanTheta& t) {
  int d = 0;
  double x[kParams];
  double ci = 0.0, sd = 0.0, cd = 1.0;
  bool have_ci = false, have_dec = false;
  for (int i = 0; i < kParams; ++i) {
    const PriorDev& p = ev.prior[i];
    if (p.kind == kFixed) {
      x[i] = p.value;
      if (i == 5) { ci = p.cosv; have_ci = true; }
      if (i == 10) { sd = p.sinv; cd = p.cosv; have_dec = true; }
      continue;
    }
    double v = u[d++];
    if (p.kind == kUniform) {
      x[i] = __dadd_rn(p.lo, __dmul_rn(v, p.w));
    } else if (p.kind == kPowerLaw) {
      double y = __dadd_rn(p.A, __dmul_rn(v, p.B));
      x[i] = (double)powf((float)y, (float)(1.0 / p.e));   // amplitude-only parameter (distance)
    } else if (p.kind == kSine) {
      double c = fmin(1.0, fmax(-1.0, __dsub_rn(p.A, __dmul_rn(v, p.B))));
      x[i] = 0.0;
      if (i == 5) { ci = c; have_ci = true; } else x[i] = acos(c);
    } else {
      double sv = fmin(1.0, fmax(-1.0, __dadd_rn(p.A, __dmul_rn(v, p.B))));
      x[i] = 0.0;
      if (i == 10) { sd = sv; cd = sqrt(fmax(0.0, (1.0 - sv) * (1.0 + sv))); have_dec = true; }
      else x[i] = asin(sv);
    }
  }
  if (!have_ci) ci = cos(x[5]);
  if (!have_dec) sincos(x[10], &sd, &cd);
  t.mc = x[0]; t.q = x[1]; t.chi1 = x[2]; t.chi2 = x[3];
  t.dl = (float)x[4]; t.ci = (float)ci; t.psi = (float)x[6];
  t.phic = x[7]; t.tc = x[8]; t.ra = x[9]; t.sdec = sd; t.cdec = cd;
}

template <int WF>
__device__ inline void taylorf2_setup_lean(const EventDev& ev, const LeanTheta& t, WalkerParams& p) {
  const double q = t.q;
  const double opq = 1.0 + q;
  const double r_opq = 1.0 / opq;
  const double eta = q * r_opq * r_opq;
  const double delta = (1.0 - q) * r_opq;
  const double chis = 0.5 * (t.chi1 + t.chi2), chia = 0.5 * (t.chi1 - t.chi2);
  const double pmc = kPi * kMsunS * t.mc;           // pi Mc [s]
  const double w = rcbrt_newton(pmc);                // (pi Mc)^(-1/3)
  const double z = rfifth_newton(eta);               // eta^(-1/5)
  const double c1 = pmc * w * w * z;                 // (pi M)^(1/3) = (pi Mc)^(1/3) eta^(-1/5)
  const double z2 = z * z;
  const double ci1 = w * eta * z2 * z2;              // (pi M)^(-1/3)
  const double ci1_3 = ci1 * ci1 * ci1;                 // 1/(pi M)
  p.k_end = bins_below(ev.f_min, ev.df, ev.n_bins, (1.0 / kSix15) * ci1_3);
  double a[8], al[8];
  taylorf2_pn_coeffs(eta, delta, chis, chia, a, al);
  const double lpm = 3.0 * log(c1);
  const double ci2 = ci1 * ci1, ci3 = ci1_3, ci5 = ci3 * ci2;
  const double pre = (3.0 / (256.0 * kPi)) * opq * opq / q;   // 3/(256 pi eta)
  p.C[0] = pre * ci5 * a[0];
  p.C[1] = pre * ci3 * a[2];
  p.C[2] = pre * ci2 * a[3];
  p.C[3] = pre * ci1 * a[4];
  p.C[4] = pre * c1 * (a[6] + al[6] * lpm / 3.0);
  p.C[5] = pre * c1 * c1 * a[7];
  p.C[6] = pre * al[5] / 3.0;
  p.C[7] = pre * c1 * al[6] / 3.0;
  p.phase0 = pre * (a[5] + al[5] * lpm / 3.0) - t.phic / kPi - 0.125;
  if (WF == 1)
    phenomd_extra<true>(ev, p, p.pd, eta, delta, chis, chia, a, al, c1, lpm, q, t.chi1, t.chi2, t.phic);
  // sky direction in FP64 (it sets the arrival delays), the rest in FP32
  double sp, cp;
  sincos(t.ra - ev.gmst, &sp, &cp);
  const double n0 = t.cdec * cp, n1 = t.cdec * sp, n2 = t.sdec;
  const float spf = (float)sp, cpf = (float)cp, ctf = (float)t.sdec, stf = (float)t.cdec;
  float ssf, csf;
  sincosf(t.psi, &ssf, &csf);
  const float X0 = spf * csf - ssf * cpf * ctf, X1 = -(cpf * csf + ssf * spf * ctf), X2 = ssf * stf;
  const float Y0 = -spf * ssf - csf * cpf * ctf, Y1 = cpf * ssf - csf * spf * ctf, Y2 = stf * csf;
  const float mcs = (float)(t.mc * kMsunS);
  const float K = (float)kAmp0 * sqrtf(mcs) * cbrtf(mcs) * (float)(kC / kMpcM) / t.dl;
  const float ap = 0.5f * (1.0f + t.ci * t.ci);
  double hh = 0.0;
  for (int det = 0; det < ev.n_det; ++det) {
    const float* xa = ev.xarm32[det];
    const float* ya = ev.yarm32[det];
    float xX = xa[0] * X0 + xa[1] * X1 + xa[2] * X2, xY = xa[0] * Y0 + xa[1] * Y1 + xa[2] * Y2;
    float yX = ya[0] * X0 + ya[1] * X1 + ya[2] * X2, yY = ya[0] * Y0 + ya[1] * Y1 + ya[2] * Y2;
    float fp = 0.5f * (xX * xX - xY * xY - yX * yX + yY * yY);
    float fc = xX * xY - yX * yY;
    float pr = fp * ap, pi_ = -fc * t.ci;
    p.kp_re[det] = (double)(K * pr);
    p.kp_im[det] = (double)(K * pi_);
    const double* r = ev.vertex[det];
    p.tau[det] = t.tc - (r[0] * n0 + r[1] * n1 + r[2] * n2) * (1.0 / kC);
    double psum = (WF == 0 && p.k_end > 0) ? ev.hh_prefix[(size_t)det * ev.n_bins + p.k_end - 1] : 0.0;
    // K ~ 1e-21: its square underflows FP32, so |K P|^2 is formed in FP64
    hh += (p.kp_re[det] * p.kp_re[det] + p.kp_im[det] * p.kp_im[det]) * psum;
  }
  p.hh = hh;
}

// Lean constants from a physical theta (ns_likelihood_batch in the mixed paths).
__device__ inline void theta_to_lean(const double* th, LeanTheta& t) {
  t.mc = th[0]; t.q = th[1]; t.chi1 = th[2]; t.chi2 = th[3];
  t.dl = (float)th[4]; t.ci = (float)cos(th[5]); t.psi = (float)th[6];
  t.phic = th[7]; t.tc = th[8]; t.ra = th[9];
  sincos(th[10], &t.sdec, &t.cdec);
}

// ---------------------------------------------------------------- per-bin accumulation
struct AccF64 {
  double re[kMaxDet], im[kMaxDet];
  __device__ void zero() { for (int i = 0; i < kMaxDet; ++i) { re[i] = 0.0; im[i] = 0.0; } }
};

// Kahan-compensated FP32 accumulator.
struct AccF32 {
  float re[kMaxDet], im[kMaxDet], cre[kMaxDet], cim[kMaxDet];
  __device__ void zero() {
    for (int i = 0; i < kMaxDet; ++i) { re[i] = 0.f; im[i] = 0.f; cre[i] = 0.f; cim[i] = 0.f; }
  }
};

// sin and cos of 2 pi x for a reduced phase |x| <= 1/2 on the special-function unit (mode 2):
// __sincosf's absolute error is below 2^-21.41 on [-pi, pi], and the rounding of 2 pi x adds
// at most pi 2^-24; over n bins the sums' error stays below ~5.5e-7 sum |d h| / S.
__device__ __forceinline__ void sincos_turn_sfu(float x, float* s, float* c) {
  __sincosf(6.2831853071795865f * x, s, c);
}

__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
  float y = x - c;
  float t = s + y;
  c = (t - s) - y;
  s = t;
}

// (sin, cos)(2 pi k / 256), k = 0 .. 255: the table of sincos_phase_f64, filled by ns_init from
// extended-precision host values (turn_table_upload).
__device__ double2 g_turn_tab[256];

// sin and cos of 2 pi ph for a phase ph in cycles (|256 ph| < 2^31), FP64, by angle addition:
// ph = j / 256 + d with j the integer nearest 256 ph (rounded by adding 1.5 * 2^52, whose low
// word then holds j) and d = ph - j / 256 exact (|d| <= 1/512); sin and cos of 2 pi j / 256
// (j mod 256) come from g_turn_tab, those of x = 2 pi d (|x| <= pi / 256) from their Taylor
// series to x^7 and x^6, whose first omitted terms are below 1e-20 of the result.  The
// whole-cycle part of ph drops out with j mod 256, so no separate reduction of ph is needed.
__device__ __forceinline__ void sincos_phase_f64(double ph, double* s, double* c) {
  const double big = fma(256.0, ph, 6755399441055744.0);
  const int j = __double2loint(big) & 255;
  const double jd = big - 6755399441055744.0;
  const double d = fma(jd, -0.00390625, ph);
  const double x = d * 6.283185307179586;
  const double x2 = x * x;
  const double sp = fma(x * x2, fma(x2, fma(x2, -1.0 / 5040.0, 1.0 / 120.0), -1.0 / 6.0), x);
  const double cp = fma(x2, fma(x2, fma(x2, -1.0 / 720.0, 1.0 / 24.0), -0.5), 1.0);
  const double2 t = g_turn_tab[j];
  *s = fma(t.x, cp, t.y * sp);
  *c = fma(t.y, cp, -(t.x * sp));
}

// FP64 path: every operation in double precision.
template <int NDET>
__device__ __forceinline__ void bin_accumulate_f64(const EventDev& ev, const WalkerParams& p, int k,
                                                   AccF64& acc) {
  const double* g = ev.basis64 + (size_t)k * ev.n_basis;
  double phi = p.phase0;
#pragma unroll
  for (int j = 0; j < kBasis; ++j) phi = fma(p.C[j], g[j], phi);
  double f = ev.f_min + ev.df * (double)k;
#pragma unroll
  for (int det = 0; det < NDET; ++det) {
    double ph = fma(p.tau[det], f, phi);
    double s, c;
    sincos_phase_f64(ph, &s, &c);
    double2 z = ev.z64[(size_t)det * ev.n_bins + k];
    // z * exp(-2 pi i ph) = (zr c + zi s) + i (zi c - zr s), accumulated by two FMAs each
    acc.re[det] = fma(z.x, c, fma(z.y, s, acc.re[det]));
    acc.im[det] = fma(z.y, c, fma(-z.x, s, acc.im[det]));
  }
}

// Mixed path: FP64 phase and its reduction, FP32 sincos and compensated FP32 sums.
template <int NDET>
__device__ __forceinline__ void bin_accumulate_mixed(const EventDev& ev, const WalkerParams& p, int k,
                                                     AccF32& acc) {
  const double* g = ev.basis64 + (size_t)k * ev.n_basis;
  double phi = p.phase0;
#pragma unroll
  for (int j = 0; j < kBasis; ++j) phi = fma(p.C[j], g[j], phi);
  double f = ev.f_min + ev.df * (double)k;
#pragma unroll
  for (int det = 0; det < NDET; ++det) {
    double ph = fma(p.tau[det], f, phi);
    float r = (float)(ph - rint(ph));
    float s, c;
    sincospif(2.0f * r, &s, &c);
    float2 z = ev.z32[(size_t)det * ev.n_bins + k];
    kahan_add(acc.re[det], acc.cre[det], fmaf(z.x, c, z.y * s));
    kahan_add(acc.im[det], acc.cim[det], fmaf(z.y, c, -z.x * s));
  }
}

// Float-float path: the phase sum_j C_j g_j is accumulated as an unevaluated (hi, lo) pair
// with error-free products (FMA) and two-sums, reduced modulo one cycle exactly, and the
// time shift k tau df is added through its 9-bit head; FP32 sincos and compensated sums.
template <int NDET>
__device__ __forceinline__ void bin_accumulate_ff(const EventDev& ev, const WalkerParams& p, int k,
                                                  AccF32& acc) {
  const float2* g = ev.basis_ff + k;
  const size_t gs = (size_t)ev.n_bins;
  // products C_j g_j as q_j + e_j (q_j = fl(Ch g.x); e_j its rounding error plus the Ch g.y and
  // Cl g.x cross terms), then an error-free pairwise sum of the q_j (depth 3 instead of a chain
  // of 8) whose errors join the low part
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
  float sh;
  {
    const float t = p.ph0h + q[0];
    const float bb = t - p.ph0h;
    sl += (p.ph0h - (t - bb)) + (q[0] - bb);
    sh = t;
  }
  const float r0 = (sh - rintf(sh)) + sl;
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
    kahan_add(acc.re[det], acc.cre[det], fmaf(z.x, c, z.y * s));
    kahan_add(acc.im[det], acc.cim[det], fmaf(z.y, c, -z.x * s));
  }
}

// ln L from the reduced sums S_det (FP64 assembly).
// s_hh: per-detector accumulated template power (IMRPhenomD form; ignored for TaylorF2, whose
// <h|h> comes from the prefix sums).
__device__ inline double assemble_lnl(const EventDev& ev, const WalkerParams& p, const double* s_re,
                                      const double* s_im, const double* s_hh = nullptr) {
  double dh = 0.0, hh = p.hh;
  for (int det = 0; det < ev.n_det; ++det) dh += p.kp_re[det] * s_re[det] - p.kp_im[det] * s_im[det];
  if (ev.waveform == 1 && s_hh) {
    hh = 0.0;
    for (int det = 0; det < ev.n_det; ++det)
      hh += (p.kp_re[det] * p.kp_re[det] + p.kp_im[det] * p.kp_im[det]) * s_hh[det];
  }
  if (ev.use_ratio) return dh - 0.5 * hh;
  return -0.5 * (ev.dd_total - 2.0 * dh + hh);
}

}  // namespace gwns

#include "gwns_phenomd.cuh"
#include "ff_setup.cuh"
