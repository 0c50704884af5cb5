// api.cu -- C ABI of libgwns: handle lifetime, input checks, event preprocessing and the
// entry points that evaluate the model (ns_waveform, ns_likelihood_batch, ns_walk_batch).
// The nested-sampling driver entry points live in nested.cu.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/gwns.h"
#include "api_internal.h"

using namespace gwns;

static thread_local std::string g_init_error;

int set_error(ns_handle* h, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (h) h->err = buf; else g_init_error = buf;
  return code;
}

int cuda_fail(ns_handle* h, cudaError_t e, const char* what) {
  return set_error(h, NS_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Grow-only device scratch owned by the handle (never shrinks until ns_free).
int ensure_scratch(ns_handle* h, Scratch& s, size_t bytes) {
  if (s.bytes >= bytes) return NS_OK;
  if (s.ptr) cudaFree(s.ptr);
  s.ptr = nullptr;
  s.bytes = 0;
  cudaError_t e = cudaMalloc(&s.ptr, bytes);
  if (e != cudaSuccess) return set_error(h, NS_ENOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
  s.bytes = bytes;
  return NS_OK;
}

static bool finite_array(const double* p, int n) {
  for (int i = 0; i < n; ++i) if (!std::isfinite(p[i])) return false;
  return true;
}

static int check_config(const ns_config& c, int e) {
  int D = 0;
  for (int i = 0; i < GWNS_N_PARAMS; ++i) {
    const ns_prior& p = c.prior[i];
    if (p.kind < NS_PRIOR_UNIFORM || p.kind > NS_PRIOR_FIXED)
      return set_error(nullptr, NS_EINVAL, "event %d: prior %d has unknown kind %d", e, i, p.kind);
    if (p.kind == NS_PRIOR_FIXED) {
      if (!std::isfinite(p.value)) return set_error(nullptr, NS_EINVAL, "event %d: fixed value %d not finite", e, i);
      continue;
    }
    ++D;
    if (!(std::isfinite(p.lo) && std::isfinite(p.hi) && p.hi > p.lo))
      return set_error(nullptr, NS_EINVAL, "event %d: prior %d needs finite lo < hi", e, i);
    if (p.kind == NS_PRIOR_POWERLAW && (!(p.alpha != -1.0) || !(p.lo > 0.0)))
      return set_error(nullptr, NS_EINVAL, "event %d: power-law prior %d needs alpha != -1 and lo > 0", e, i);
    if (p.kind == NS_PRIOR_SINE && (p.lo < 0.0 || p.hi > M_PI + 1e-12))
      return set_error(nullptr, NS_EINVAL, "event %d: sine prior %d must lie in [0, pi]", e, i);
    if (p.kind == NS_PRIOR_COSINE && (p.lo < -M_PI_2 - 1e-12 || p.hi > M_PI_2 + 1e-12))
      return set_error(nullptr, NS_EINVAL, "event %d: cosine prior %d must lie in [-pi/2, pi/2]", e, i);
  }
  if (D < 1) return set_error(nullptr, NS_EINVAL, "event %d: no sampled parameter", e);
  if (c.n_live < 3) return set_error(nullptr, NS_EINVAL, "event %d: n_live must be >= 3", e);
  if (c.n_live > kMaxLive) return set_error(nullptr, NS_EINVAL, "event %d: n_live > %d", e, kMaxLive);
  if (c.num_delete < 1 || c.n_live - c.num_delete < 2)
    return set_error(nullptr, NS_EINVAL, "event %d: need 1 <= num_delete <= n_live - 2", e);
  if (c.naccept < 1 || c.maxmcmc < 1) return set_error(nullptr, NS_EINVAL, "event %d: naccept, maxmcmc >= 1", e);
  if (c.spec_depth < 0 || c.spec_depth > kSpecMax)
    return set_error(nullptr, NS_EINVAL, "event %d: spec_depth must be in 0..%d", e, kSpecMax);
  if (c.proposal == NS_PROPOSAL_HRSS) {
    if (c.hrss_moves < 0 || c.hrss_moves > 1000000)
      return set_error(nullptr, NS_EINVAL, "event %d: hrss_moves must be in 0..1000000", e);
    if (c.n_live - c.num_delete <= D)
      return set_error(nullptr, NS_EINVAL, "event %d: HRSS needs n_live - num_delete > D = %d", e, D);
  } else if (c.hrss_moves != 0) {
    return set_error(nullptr, NS_EINVAL, "event %d: hrss_moves is for NS_PROPOSAL_HRSS (0 otherwise)", e);
  }
  if (c.precision != NS_PREC_FP64 && c.precision != NS_PREC_MIXED && c.precision != NS_PREC_MIXED_FF)
    return set_error(nullptr, NS_EINVAL, "event %d: unknown precision %d", e, c.precision);
  if (c.waveform != NS_WAVEFORM_TAYLORF2 && c.waveform != NS_WAVEFORM_PHENOMD_FORM)
    return set_error(nullptr, NS_EINVAL, "event %d: unknown waveform %d", e, c.waveform);
  if (c.term_kind != NS_TERM_DLOGZ && c.term_kind != NS_TERM_FRAC_REMAINING)
    return set_error(nullptr, NS_EINVAL, "event %d: unknown termination %d", e, c.term_kind);
  if (!(c.term_value > 0.0)) return set_error(nullptr, NS_EINVAL, "event %d: term_value must be > 0", e);
  return flow_check_config(c, e);
}

static int check_event(const ns_event& ev, int e) {
  if (ev.n_det < 1 || ev.n_det > GWNS_MAX_DET) return set_error(nullptr, NS_EINVAL, "event %d: n_det out of range", e);
  if (ev.n_bins < 1) return set_error(nullptr, NS_EINVAL, "event %d: n_bins must be >= 1", e);
  if (!(ev.f_min > 0.0 && ev.df > 0.0 && std::isfinite(ev.gmst)))
    return set_error(nullptr, NS_EINVAL, "event %d: need f_min > 0, df > 0, finite gmst", e);
  for (int d = 0; d < ev.n_det; ++d) {
    const ns_detector& det = ev.det[d];
    if (!det.d_re || !det.d_im || !det.psd) return set_error(nullptr, NS_EINVAL, "event %d det %d: null data", e, d);
    if (!finite_array(det.vertex, 3) || !finite_array(det.x_arm, 3) || !finite_array(det.y_arm, 3))
      return set_error(nullptr, NS_ENONFINITE, "event %d det %d: geometry not finite", e, d);
    if (!finite_array(det.d_re, ev.n_bins) || !finite_array(det.d_im, ev.n_bins))
      return set_error(nullptr, NS_ENONFINITE, "event %d det %d: data not finite", e, d);
    for (int k = 0; k < ev.n_bins; ++k)
      if (!(det.psd[k] > 0.0) || !std::isfinite(det.psd[k]))
        return set_error(nullptr, NS_ENONFINITE, "event %d det %d: psd[%d] not finite and positive", e, d, k);
  }
  return NS_OK;
}

// Host-side preprocessing of one event (FP64): per-bin phase basis, whitened data products
// and inclusive prefix sums of the template power.  Kahan summation keeps the running sums
// accurate to a few ulp.
static int prepare_event(ns_handle* h, int e, const ns_config& c, const ns_event& in) {
  EventHost& E = h->events[e];
  E.cfg = c;
  E.n_det = in.n_det;
  E.n_bins = in.n_bins;
  const int nb = in.n_bins, nd = in.n_det;
  const int nbas = c.waveform == NS_WAVEFORM_PHENOMD_FORM ? kBasisPD : kBasis;
  std::vector<double> basis((size_t)nb * nbas);
  std::vector<float2> basis_ff((size_t)nb * nbas);
  std::vector<double> gw64((size_t)nd * nb);
  std::vector<float> gw32((size_t)nd * nb);
  std::vector<double2> z64((size_t)nd * nb);
  std::vector<float2> z32((size_t)nd * nb);
  std::vector<double> pref((size_t)nd * nb);
  double dd = 0.0, ddc = 0.0;
  for (int k = 0; k < nb; ++k) {
    double f = in.f_min + in.df * (double)k;
    double c3 = std::cbrt(f), lf = std::log(f);
    double* g = &basis[(size_t)k * nbas];
    g[0] = 1.0 / (f * c3 * c3);   // f^-5/3
    g[1] = 1.0 / f;               // f^-1
    g[2] = 1.0 / (c3 * c3);       // f^-2/3
    g[3] = 1.0 / c3;              // f^-1/3
    g[4] = c3;                    // f^1/3
    g[5] = c3 * c3;               // f^2/3
    g[6] = lf;                    // ln f
    g[7] = c3 * lf;               // f^1/3 ln f
    if (nbas == kBasisPD) {
      g[8] = f * c3;              // f^4/3
      g[9] = f * c3 * c3;         // f^5/3
      g[10] = f * f;              // f^2
      g[11] = 1.0 / (f * f * f);  // f^-3
      g[12] = std::pow(f, 0.75);  // f^3/4
      g[13] = f;                  // f
    }
    for (int j = 0; j < nbas; ++j) {
      float hi = (float)g[j];
      basis_ff[(size_t)j * nb + k] = make_float2(hi, (float)(g[j] - (double)hi));
    }
  }
  for (int d = 0; d < nd; ++d) {
    const ns_detector& det = in.det[d];
    double run = 0.0, runc = 0.0;
    for (int k = 0; k < nb; ++k) {
      double f = in.f_min + in.df * (double)k;
      double w = 4.0 * in.df / det.psd[k];
      double a = std::pow(f, -7.0 / 6.0);
      double zr = w * det.d_re[k] * a, zi = -w * det.d_im[k] * a;   // 4 df conj(d) f^-7/6 / S
      z64[(size_t)d * nb + k] = make_double2(zr, zi);
      z32[(size_t)d * nb + k] = make_float2((float)zr, (float)zi);
      double term = w * a * a;                                      // 4 df f^-7/3 / S
      gw64[(size_t)d * nb + k] = term;
      double y = term - runc, t = run + y;
      runc = (t - run) - y;
      run = t;
      pref[(size_t)d * nb + k] = run;
      double dterm = w * (det.d_re[k] * det.d_re[k] + det.d_im[k] * det.d_im[k]);
      double y2 = dterm - ddc, t2 = dd + y2;
      ddc = (t2 - dd) - y2;
      dd = t2;
    }
  }
  // FP32 template-power weights scaled by a power of two so that the largest is ~1
  double gmax = 0.0;
  for (double v : gw64) gmax = std::fmax(gmax, v);
  const double gscale = gmax > 0.0 ? std::ldexp(1.0, -std::ilogb(gmax)) : 1.0;
  for (size_t i = 0; i < gw64.size(); ++i) gw32[i] = (float)(gw64[i] * gscale);
  // FP32 copy of the template-power prefix sums scaled by 2^-140 (the float-float path pairs
  // it with amplitude factors scaled by 2^70)
  std::vector<float> pref32(pref.size());
  for (size_t i = 0; i < pref.size(); ++i) pref32[i] = (float)std::ldexp(pref[i], -2 * kKpScaleExp);
  // device copies
  cudaError_t err;
  if ((err = cudaMalloc(&E.d_basis64, basis.size() * sizeof(double))) != cudaSuccess ||
      (err = cudaMalloc(&E.d_basis_ff, basis_ff.size() * sizeof(float2))) != cudaSuccess ||
      (err = cudaMalloc(&E.d_z64, z64.size() * sizeof(double2))) != cudaSuccess ||
      (err = cudaMalloc(&E.d_z32, z32.size() * sizeof(float2))) != cudaSuccess ||
      (err = cudaMalloc(&E.d_hh_prefix, pref.size() * sizeof(double))) != cudaSuccess ||
      (err = cudaMalloc(&E.d_gw64, gw64.size() * sizeof(double))) != cudaSuccess ||
      (err = cudaMalloc(&E.d_gw32, gw32.size() * sizeof(float))) != cudaSuccess ||
      (err = cudaMalloc(&E.d_hhp32, pref32.size() * sizeof(float))) != cudaSuccess)
    return set_error(nullptr, NS_ENOMEM, "event %d: device allocation failed: %s", e, cudaGetErrorString(err));
  if ((err = copy_on(h, E.d_basis64, basis.data(), basis.size() * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (err = copy_on(h, E.d_basis_ff, basis_ff.data(), basis_ff.size() * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (err = copy_on(h, E.d_z64, z64.data(), z64.size() * sizeof(double2), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (err = copy_on(h, E.d_z32, z32.data(), z32.size() * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (err = copy_on(h, E.d_hh_prefix, pref.data(), pref.size() * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (err = copy_on(h, E.d_gw64, gw64.data(), gw64.size() * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (err = copy_on(h, E.d_gw32, gw32.data(), gw32.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (err = copy_on(h, E.d_hhp32, pref32.data(), pref32.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess)
    return set_error(nullptr, NS_ECUDA, "event %d: upload failed: %s", e, cudaGetErrorString(err));

  EventDev& D = E.dev;
  std::memset(&D, 0, sizeof(D));
  D.n_det = nd;
  D.n_bins = nb;
  D.waveform = c.waveform;
  D.n_basis = nbas;
  D.use_ratio = c.use_ratio ? 1 : 0;
  D.f_min = in.f_min;
  D.df = in.df;
  D.gmst = in.gmst;
  D.dd_total = dd;
  auto split = [](double x, float* f) { f[0] = (float)x; f[1] = (float)(x - (double)f[0]); };
  split(in.f_min, D.fmin_f);
  split(in.df, D.df_f);
  split(in.gmst, D.gmst_f);
  for (int d = 0; d < nd; ++d)
    for (int i = 0; i < 3; ++i) {
      split(in.det[d].vertex[i] / 299792458.0, D.vc_f[d][i]);
      D.vertex[d][i] = in.det[d].vertex[i];
      D.xarm[d][i] = in.det[d].x_arm[i];
      D.yarm[d][i] = in.det[d].y_arm[i];
      D.xarm32[d][i] = (float)in.det[d].x_arm[i];
      D.yarm32[d][i] = (float)in.det[d].y_arm[i];
    }
  int nd_dim = 0;
  for (int i = 0; i < kParams; ++i) {
    const ns_prior& p = c.prior[i];
    PriorDev& q = D.prior[i];
    q.kind = p.kind;
    q.periodic = p.periodic ? 1 : 0;
    q.lo = p.lo;
    q.hi = p.hi;
    q.w = p.hi - p.lo;
    q.value = p.value;
    q.cosv = std::cos(p.value);
    q.sinv = std::sin(p.value);
    if (p.kind == NS_PRIOR_POWERLAW) {
      q.e = p.alpha + 1.0;
      q.A = std::pow(p.lo, q.e);
      q.B = std::pow(p.hi, q.e) - q.A;
    } else if (p.kind == NS_PRIOR_SINE) {
      q.A = std::cos(p.lo);
      q.B = std::cos(p.lo) - std::cos(p.hi);
    } else if (p.kind == NS_PRIOR_COSINE) {
      q.A = std::sin(p.lo);
      q.B = std::sin(p.hi) - std::sin(p.lo);
    }
    split(q.lo, q.lo_f);
    split(q.w, q.w_f);
    split(q.A, q.A_f);
    split(q.B, q.B_f);
    split(q.value, q.v_f);
    split(q.cosv, q.cv_f);
    split(q.sinv, q.sv_f);
    q.einv_f = q.e != 0.0 ? (float)(1.0 / q.e) : 0.0f;
    D.param_dim[i] = p.kind != NS_PRIOR_FIXED ? nd_dim : -1;
    if (p.kind != NS_PRIOR_FIXED) D.dim_param[nd_dim++] = i;
  }
  // the float-float setup transforms uniform priors, the power law of the distance, the sine
  // prior of the inclination and the cosine prior of the declination
  D.ff_setup = 1;
  for (int i = 0; i < kParams; ++i) {
    const int k = c.prior[i].kind;
    if ((k == NS_PRIOR_POWERLAW && i != 4) || (k == NS_PRIOR_SINE && i != 5) || (k == NS_PRIOR_COSINE && i != 10))
      D.ff_setup = 0;
  }
  D.n_dim = nd_dim;
  D.basis64 = E.d_basis64;
  D.basis_ff = E.d_basis_ff;
  D.z64 = E.d_z64;
  D.z32 = E.d_z32;
  D.hh_prefix = E.d_hh_prefix;
  D.hhp32 = E.d_hhp32;
  D.dd_f[0] = (float)dd;
  D.dd_f[1] = (float)(dd - (double)D.dd_f[0]);
  D.gw64 = E.d_gw64;
  D.gw32 = E.d_gw32;
  D.gw32_unscale = 1.0 / gscale;
  D.hh_unscale_f = (float)std::ldexp(D.gw32_unscale, -2 * kKpScaleExp);
  E.n_dim = nd_dim;
  return NS_OK;
}

void free_event(EventHost& E) {
  relbin_free(E);
  cudaFree(E.d_basis64);
  cudaFree(E.d_basis_ff);
  cudaFree(E.d_z64);
  cudaFree(E.d_z32);
  cudaFree(E.d_hh_prefix);
  cudaFree(E.d_hhp32);
  E.d_hhp32 = nullptr;
  cudaFree(E.d_gw64);
  cudaFree(E.d_gw32);
  E.d_gw64 = nullptr;
  E.d_gw32 = nullptr;
  E.d_basis64 = nullptr;
  E.d_basis_ff = nullptr;
  E.d_z64 = nullptr;
  E.d_z32 = nullptr;
  E.d_hh_prefix = nullptr;
}

extern "C" int ns_init(const ns_config* cfg, const ns_event* ev, int n_events, int device, ns_handle** out) {
  if (!out) return set_error(nullptr, NS_EINVAL, "out is NULL");
  *out = nullptr;
  if (!cfg || !ev) return set_error(nullptr, NS_EINVAL, "cfg or ev is NULL");
  if (n_events < 1 || n_events > GWNS_MAX_EVENTS) return set_error(nullptr, NS_EINVAL, "n_events out of range");
  for (int e = 0; e < n_events; ++e) {
    int r = check_config(cfg[e], e);
    if (r) return r;
    r = check_event(ev[e], e);
    if (r) return r;
    if (cfg[e].precision != cfg[0].precision || cfg[e].waveform != cfg[0].waveform)
      return set_error(nullptr, NS_EINVAL, "every event of a handle needs the same precision and waveform");
    if ((cfg[e].proposal == NS_PROPOSAL_HRSS) != (cfg[0].proposal == NS_PROPOSAL_HRSS))
      return set_error(nullptr, NS_EINVAL, "every event of a handle uses HRSS (NS_PROPOSAL_HRSS) or none does");
    if (ev[e].n_det != ev[0].n_det)
      return set_error(nullptr, NS_EINVAL, "every event of a handle needs the same number of detectors");
  }
  cudaError_t e0 = cudaSetDevice(device);
  if (e0 != cudaSuccess) return set_error(nullptr, NS_ECUDA, "cudaSetDevice(%d): %s", device, cudaGetErrorString(e0));
  cudaGetLastError();   // a stale error of an earlier call must not be reported here
  ns_handle* h = new ns_handle();
  h->device = device;
  h->precision = cfg[0].precision;
  h->waveform = cfg[0].waveform;
  h->hrss = cfg[0].proposal == NS_PROPOSAL_HRSS;
  h->events.resize(n_events);
  int max_det = 0;
  for (int e = 0; e < n_events; ++e) {
    int r = prepare_event(h, e, cfg[e], ev[e]);
    if (r) { ns_free(h); return r; }
    max_det = ev[e].n_det > max_det ? ev[e].n_det : max_det;
  }
  h->max_det = max_det;
  if ((e0 = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking)) != cudaSuccess ||
      (e0 = cudaStreamCreateWithFlags(&h->aux_stream, cudaStreamNonBlocking)) != cudaSuccess) {
    ns_free(h);
    return set_error(nullptr, NS_ECUDA, "stream: %s", cudaGetErrorString(e0));
  }
  if ((e0 = turn_table_upload(h->stream)) != cudaSuccess) {
    ns_free(h);
    return set_error(nullptr, NS_ECUDA, "angle table: %s", cudaGetErrorString(e0));
  }
  if ((e0 = cudaMalloc(&h->d_events, sizeof(EventDev) * n_events)) != cudaSuccess) {
    ns_free(h);
    return set_error(nullptr, NS_ENOMEM, "event table: %s", cudaGetErrorString(e0));
  }
  std::vector<EventDev> tab(n_events);
  for (int e = 0; e < n_events; ++e) tab[e] = h->events[e].dev;
  if ((e0 = copy_on(h, h->d_events, tab.data(), sizeof(EventDev) * n_events, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e0 = cudaMalloc(&h->d_status, sizeof(int32_t) * 4)) != cudaSuccess ||
      (e0 = fill_on(h, h->d_status, 0, sizeof(int32_t) * 4)) != cudaSuccess) {
    ns_free(h);
    return set_error(nullptr, NS_ECUDA, "event table upload: %s", cudaGetErrorString(e0));
  }
  for (int e = 0; e < n_events; ++e) {
    int r = flow_setup(h, e);
    if (r) {
      std::string msg = h->err;
      ns_free(h);
      return set_error(nullptr, r, "%s", msg.c_str());
    }
  }
  int r = nested_init(h);
  if (r) {
    std::string msg = h->err;
    ns_free(h);
    return set_error(nullptr, r, "%s", msg.c_str());
  }
  *out = h;
  return NS_OK;
}

// Speculation depth of a stand-alone walk when the configuration leaves it automatic.
int default_spec(int precision) { return precision == NS_PREC_FP64 ? 4 : 16; }

// Candidates per round of the float-float HRSS kernel when the configuration leaves it automatic:
// TaylorF2 evaluates a warp per candidate (8: two rounds of the four warps cost about one), the
// IMRPhenomD form runs each candidate on the whole CTA (2).
int hrss_default_spec(int waveform) { return waveform == NS_WAVEFORM_TAYLORF2 ? 8 : 2; }

static cudaStream_t pick_stream(ns_handle* h, void* stream) {
  return stream ? (cudaStream_t)stream : h->stream;
}

extern "C" int ns_waveform(ns_handle* h, int event, const double* theta, int n, double* h_re, double* h_im,
                           int ptr_kind, void* stream) {
  if (!h) return set_error(nullptr, NS_EINVAL, "handle is NULL");
  if (event < 0 || event >= (int)h->events.size()) return set_error(h, NS_EINVAL, "event out of range");
  if (n < 0 || (n > 0 && (!theta || !h_re || !h_im))) return set_error(h, NS_EINVAL, "bad arrays");
  if (ptr_kind != NS_PTR_HOST && ptr_kind != NS_PTR_DEVICE) return set_error(h, NS_EINVAL, "bad ptr_kind");
  if (n == 0) return NS_OK;
  cudaSetDevice(h->device);
  cudaGetLastError();
  EventHost& E = h->events[event];
  const EventDev* d_ev = h->d_events + event;
  cudaStream_t s = pick_stream(h, stream);
  size_t nh = (size_t)n * E.n_det * E.n_bins;
  if (ptr_kind == NS_PTR_HOST) {
    if (!finite_array(theta, n * kParams)) return set_error(h, NS_ENONFINITE, "theta not finite");
    size_t tb = sizeof(double) * (size_t)n * kParams;
    int r = ensure_scratch(h, h->scratch_in, tb);
    if (r) return r;
    r = ensure_scratch(h, h->scratch_out, 2 * sizeof(double) * nh);
    if (r) return r;
    double* d_th = (double*)h->scratch_in.ptr;
    double* d_re = (double*)h->scratch_out.ptr;
    double* d_im = d_re + nh;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(d_th, theta, tb, cudaMemcpyHostToDevice, s)) != cudaSuccess) return cuda_fail(h, e, "H2D theta");
    if ((e = launch_waveform(h->waveform, E.n_det, d_ev, d_th, n, E.n_bins, d_re, d_im, s)) != cudaSuccess) return cuda_fail(h, e, "waveform launch");
    if ((e = cudaMemcpyAsync(h_re, d_re, sizeof(double) * nh, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return cuda_fail(h, e, "D2H h_re");
    if ((e = cudaMemcpyAsync(h_im, d_im, sizeof(double) * nh, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return cuda_fail(h, e, "D2H h_im");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(h, e, "waveform");
    return NS_OK;
  }
  cudaError_t e = launch_waveform(h->waveform, E.n_det, d_ev, theta, n, E.n_bins, h_re, h_im, s);
  return e == cudaSuccess ? NS_OK : cuda_fail(h, e, "waveform launch");
}

extern "C" int ns_likelihood_batch(ns_handle* h, int event, const double* theta, int n, double* lnl, int ptr_kind,
                                   void* stream) {
  if (!h) return set_error(nullptr, NS_EINVAL, "handle is NULL");
  if (event < 0 || event >= (int)h->events.size()) return set_error(h, NS_EINVAL, "event out of range");
  if (n < 0 || (n > 0 && (!theta || !lnl))) return set_error(h, NS_EINVAL, "bad arrays");
  if (ptr_kind != NS_PTR_HOST && ptr_kind != NS_PTR_DEVICE) return set_error(h, NS_EINVAL, "bad ptr_kind");
  if (n == 0) return NS_OK;
  cudaSetDevice(h->device);
  cudaGetLastError();
  EventHost& E = h->events[event];
  const EventDev* d_ev = h->d_events + event;
  cudaStream_t s = pick_stream(h, stream);
  cudaError_t e;
  if ((e = cudaMemsetAsync(h->d_status, 0, sizeof(int32_t), s)) != cudaSuccess) return cuda_fail(h, e, "status reset");
  if (ptr_kind == NS_PTR_HOST) {
    if (!finite_array(theta, n * kParams)) return set_error(h, NS_ENONFINITE, "theta not finite");
    size_t tb = sizeof(double) * (size_t)n * kParams;
    int r = ensure_scratch(h, h->scratch_in, tb);
    if (r) return r;
    r = ensure_scratch(h, h->scratch_out, sizeof(double) * (size_t)n);
    if (r) return r;
    double* d_th = (double*)h->scratch_in.ptr;
    double* d_l = (double*)h->scratch_out.ptr;
    if ((e = cudaMemcpyAsync(d_th, theta, tb, cudaMemcpyHostToDevice, s)) != cudaSuccess) return cuda_fail(h, e, "H2D theta");
    if ((e = launch_likelihood(h->precision, h->waveform, E.n_det, d_ev, d_th, n, d_l, h->d_status, s)) != cudaSuccess)
      return cuda_fail(h, e, "likelihood launch");
    if ((e = cudaMemcpyAsync(lnl, d_l, sizeof(double) * n, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return cuda_fail(h, e, "D2H lnl");
    int32_t st = 0;
    if ((e = cudaMemcpyAsync(&st, h->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return cuda_fail(h, e, "D2H status");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(h, e, "likelihood");
    if (st) return set_error(h, NS_ENONFINITE, "a theta was not finite or out of the physical domain");
    return NS_OK;
  }
  e = launch_likelihood(h->precision, h->waveform, E.n_det, d_ev, theta, n, lnl, h->d_status, s);
  return e == cudaSuccess ? NS_OK : cuda_fail(h, e, "likelihood launch");
}

extern "C" int ns_walk_batch(ns_handle* h, int event, const double* live_u, int n_live_pts, const double* u0,
                             const double* lnl0, double lnl_star, int n, int n_steps, int64_t iteration,
                             int64_t walker_offset, double* u_out, double* lnl_out, int32_t* n_accept,
                             int32_t* n_like, int ptr_kind, void* stream) {
  if (!h) return set_error(nullptr, NS_EINVAL, "handle is NULL");
  if (event < 0 || event >= (int)h->events.size()) return set_error(h, NS_EINVAL, "event out of range");
  if (n < 0 || n_steps < 0 || n_live_pts < 2 || iteration < 0 || walker_offset < 0)
    return set_error(h, NS_EINVAL, "need n >= 0, n_steps >= 0, n_live_pts >= 2, iteration >= 0, walker_offset >= 0");
  if (n > 0 && (!live_u || !u0 || !lnl0 || !u_out || !lnl_out || !n_accept || !n_like))
    return set_error(h, NS_EINVAL, "null array");
  if (ptr_kind != NS_PTR_HOST && ptr_kind != NS_PTR_DEVICE) return set_error(h, NS_EINVAL, "bad ptr_kind");
  if (std::isnan(lnl_star)) return set_error(h, NS_ENONFINITE, "lnl_star is NaN");
  if (n == 0) return NS_OK;
  cudaSetDevice(h->device);
  cudaGetLastError();
  EventHost& E = h->events[event];
  const int D = E.n_dim;
  cudaStream_t s = pick_stream(h, stream);
  WalkTask T;
  std::memset(&T, 0, sizeof(T));
  T.lnl_star = lnl_star;
  T.iteration = iteration;
  T.walker_offset = walker_offset;
  T.key0 = E.cfg.seed;
  T.key1 = (uint64_t)event;
  T.n_s = n_live_pts;
  T.n = n;
  T.n_steps = n_steps;
  T.done = 0;
  T.event = event;
  T.spec = E.cfg.spec_depth > 0 ? E.cfg.spec_depth : default_spec(h->precision);
  watchdog_fields(h, T);
  cudaError_t e;
  if ((e = cudaMemsetAsync(h->d_status + 1, 0, sizeof(int32_t) * 2, s)) != cudaSuccess) return cuda_fail(h, e, "status reset");
  int fr = flow_attach(h, event, T, n, n_steps, &h->scratch_flow, s);
  if (fr) return fr;
  // block -> (event, walker) maps, one task slot of the handle
  int r = ensure_scratch(h, h->scratch_map, sizeof(int32_t) * 2 * (size_t)n + sizeof(WalkTask));
  if (r) return r;
  WalkTask* d_task = (WalkTask*)h->scratch_map.ptr;
  int32_t* d_be = (int32_t*)((char*)h->scratch_map.ptr + sizeof(WalkTask));
  int32_t* d_bl = d_be + n;
  std::vector<int32_t> maps(2 * (size_t)n);
  for (int j = 0; j < n; ++j) { maps[j] = 0; maps[n + j] = j; }
  size_t nu = (size_t)n * D, ns_ = (size_t)n_live_pts * D;
  if (ptr_kind == NS_PTR_HOST) {
    if (!finite_array(live_u, (int)ns_) || !finite_array(u0, (int)nu)) return set_error(h, NS_ENONFINITE, "u not finite");
    size_t in_b = sizeof(double) * (ns_ + nu + n);
    size_t out_b = sizeof(double) * (nu + n) + 2 * sizeof(int32_t) * n;
    if ((r = ensure_scratch(h, h->scratch_in, in_b))) return r;
    if ((r = ensure_scratch(h, h->scratch_out, out_b))) return r;
    double* d_surv = (double*)h->scratch_in.ptr;
    double* d_u0 = d_surv + ns_;
    double* d_l0 = d_u0 + nu;
    double* d_uo = (double*)h->scratch_out.ptr;
    double* d_lo = d_uo + nu;
    int32_t* d_na = (int32_t*)(d_lo + n);
    int32_t* d_nl = d_na + n;
    T.surv = d_surv; T.u0 = d_u0; T.lnl0 = d_l0; T.u_out = d_uo; T.lnl_out = d_lo; T.n_acc = d_na; T.n_like = d_nl;
    if ((e = cudaMemcpyAsync(d_surv, live_u, sizeof(double) * ns_, cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(d_u0, u0, sizeof(double) * nu, cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(d_l0, lnl0, sizeof(double) * n, cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(d_task, &T, sizeof(T), cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(d_be, maps.data(), sizeof(int32_t) * 2 * n, cudaMemcpyHostToDevice, s)))
      return cuda_fail(h, e, "H2D walk inputs");
    if ((e = launch_walk(h->precision, h->waveform, E.n_det, h->d_events, d_task, d_be, d_bl, n, s, walk_extras(h, event))) != cudaSuccess)
      return cuda_fail(h, e, "walk launch");
    if ((e = cudaMemcpyAsync(u_out, d_uo, sizeof(double) * nu, cudaMemcpyDeviceToHost, s)) ||
        (e = cudaMemcpyAsync(lnl_out, d_lo, sizeof(double) * n, cudaMemcpyDeviceToHost, s)) ||
        (e = cudaMemcpyAsync(n_accept, d_na, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s)) ||
        (e = cudaMemcpyAsync(n_like, d_nl, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s)))
      return cuda_fail(h, e, "D2H walk outputs");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(h, e, "walk");
    if ((r = watchdog_report(h))) return r;
    for (int j = 0; j < n; ++j) if (n_accept[j] == 0) return NS_WMAXMCMC;
    return NS_OK;
  }
  T.surv = live_u; T.u0 = u0; T.lnl0 = lnl0; T.u_out = u_out; T.lnl_out = lnl_out; T.n_acc = n_accept; T.n_like = n_like;
  // The task and the block maps go through the handle's scratch, ordered on the stream
  // before the launch (a pageable-memory copy has consumed its source when it returns).
  std::vector<char> stage((char*)&T, (char*)&T + sizeof(T));
  stage.insert(stage.end(), (char*)maps.data(), (char*)maps.data() + sizeof(int32_t) * 2 * n);
  if ((e = cudaMemcpyAsync(d_task, stage.data(), stage.size(), cudaMemcpyHostToDevice, s)))
    return cuda_fail(h, e, "H2D walk task");
  e = launch_walk(h->precision, h->waveform, E.n_det, h->d_events, d_task, d_be, d_bl, n, s, walk_extras(h, event));
  return e == cudaSuccess ? NS_OK : cuda_fail(h, e, "walk launch");
}

// The watchdog fields of a walk task: the handle's abort flag (d_status[3]), its timeout bit
// (d_status[2]) and its time budget.
void watchdog_fields(ns_handle* h, WalkTask& T) {
  T.abort = h->d_status + 3;
  T.status = h->d_status + 2;
  T.budget_ns = h->budget_ns;
}

bool walk_extras(const ns_handle* h, int e) {
  const EventHost& E = h->events[e];
  return E.dev.rb_nb > 0 || (E.flow.enabled && E.flow.p_flow > 0.0);
}

bool walk_extras(const ns_handle* h) {
  for (int e = 0; e < (int)h->events.size(); ++e)
    if (walk_extras(h, e)) return true;
  return false;
}

cudaError_t copy_on(ns_handle* h, void* dst, const void* src, size_t bytes, cudaMemcpyKind kind) {
  if (bytes == 0) return cudaSuccess;
  const cudaError_t e = cudaMemcpyAsync(dst, src, bytes, kind, h->stream);
  return e != cudaSuccess ? e : cudaStreamSynchronize(h->stream);
}

cudaError_t fill_on(ns_handle* h, void* dst, int value, size_t bytes) {
  if (bytes == 0) return cudaSuccess;
  const cudaError_t e = cudaMemsetAsync(dst, value, bytes, h->stream);
  return e != cudaSuccess ? e : cudaStreamSynchronize(h->stream);
}

// NS_ETIMEOUT when a walk of the handle stopped on its watchdog since the bit was last cleared.
int watchdog_report(ns_handle* h) {
  int32_t st = 0;
  cudaError_t e = copy_on(h, &st, h->d_status + 2, sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "watchdog status");
  if (st) return set_error(h, NS_ETIMEOUT, "a walk stopped on the watchdog (time budget or abort flag)");
  return NS_OK;
}

extern "C" int ns_set_watchdog(ns_handle* h, double budget_seconds) {
  if (!h) return set_error(nullptr, NS_EINVAL, "handle is NULL");
  if (!(budget_seconds >= 0.0) || !(budget_seconds < 1e9)) return set_error(h, NS_EINVAL, "budget must be in [0, 1e9) s");
  cudaSetDevice(h->device);
  cudaGetLastError();
  h->budget_ns = (uint64_t)(budget_seconds * 1e9);
  if (budget_seconds > 0.0 && h->budget_ns == 0) h->budget_ns = 1;
  // the sampler's tasks read it at every batch
  cudaError_t e = cudaSuccess;
  for (size_t ev = 0; ev < h->events.size() && e == cudaSuccess && h->d_tasks; ++ev)
    e = copy_on(h, &h->d_tasks[ev].budget_ns, &h->budget_ns, sizeof(uint64_t), cudaMemcpyHostToDevice);
  return e == cudaSuccess ? NS_OK : cuda_fail(h, e, "watchdog budget");
}

extern "C" int ns_set_abort(ns_handle* h, int flag) {
  if (!h) return set_error(nullptr, NS_EINVAL, "handle is NULL");
  cudaSetDevice(h->device);
  const int32_t v = flag ? 1 : 0;
  cudaError_t e = cudaMemcpyAsync(h->d_status + 3, &v, sizeof(int32_t), cudaMemcpyHostToDevice, h->aux_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->aux_stream);
  return e == cudaSuccess ? NS_OK : set_error(h, NS_ECUDA, "abort flag: %s", cudaGetErrorString(e));
}

extern "C" void ns_free(ns_handle* h) {
  if (!h) return;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  nested_free(h);
  for (auto& E : h->events) {
    free_event(E);
    flow_free(E);
  }
  cudaFree(h->d_events);
  cudaFree(h->d_status);
  cudaFree(h->scratch_in.ptr);
  cudaFree(h->scratch_out.ptr);
  cudaFree(h->scratch_map.ptr);
  cudaFree(h->scratch_flow.ptr);
  cudaFree(h->scratch_shard.ptr);
  if (h->stream) cudaStreamDestroy(h->stream);
  if (h->aux_stream) cudaStreamDestroy(h->aux_stream);
  delete h;
}

extern "C" const char* ns_last_error(ns_handle* h) {
  return h ? h->err.c_str() : g_init_error.c_str();
}
