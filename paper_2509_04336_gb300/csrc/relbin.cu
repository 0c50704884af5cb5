// relbin.cu -- relative-binning summary data of one event (ns_relbin_set).
//
// Around a fiducial template h0 (the template at theta0, continued above its cutoff), the
// ratio r = h / h0 of a proposal's strain is taken as linear in f across each coarse bin
// [e_b, e_{b+1}) of the grid; with the summary data of the bin and detector (w = 4 df / S,
// x = f - f_{e_b})
//   A0 = sum conj(d) h0 w,  A1 = sum conj(d) h0 w x,  B0 = sum |h0|^2 w,  B1 = sum |h0|^2 w x,
//   B2 = sum |h0|^2 w x^2
// the bin's inner products are <d|h> = Re(A0 r_b + A1 r1_b) and
// <h|h> = B0 |r_b|^2 + 2 B1 Re(conj(r_b) r1_b) + B2 |r1_b|^2, r1_b the slope between the edges
// (the likelihood compression named in Sec. 3.3 and Sec. 5; Zackay, Dai & Venumadhav 2018).
// The summary data are computed here once, in FP64 on the host, from the event's weighted data
// and the fiducial evaluated by the FP64 waveform kernel; the mode-2 kernels evaluate r at the
// edges (rb_lnl_warp).
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/gwns.h"
#include "api_internal.h"

using namespace gwns;

void relbin_free(EventHost& E) {
  cudaFree(E.d_rb_edges);
  cudaFree(E.d_rb_q0);
  cudaFree(E.d_rb_a);
  cudaFree(E.d_rb_b);
  E.d_rb_edges = nullptr;
  E.d_rb_q0 = nullptr;
  E.d_rb_a = nullptr;
  E.d_rb_b = nullptr;
  E.dev.rb_nb = 0;
  E.dev.rb_edges = nullptr;
  E.dev.rb_q0 = nullptr;
  E.dev.rb_a = nullptr;
  E.dev.rb_b = nullptr;
}

// Makes `nd` the event's descriptor: uploads it to the device copy first (a synchronous copy;
// until it succeeds the old descriptor and its arrays stay in place and valid), then adopts
// the new relative-binning arrays, frees the old ones (cudaFree waits for kernels still
// reading them) and re-evaluates the initial live points with the likelihood now in effect.
// On an upload failure the caller still owns the new arrays.
static int relbin_adopt(ns_handle* h, int event, const EventDev& nd, int32_t* ed, float2* q0, float2* a, float4* b) {
  EventHost& E = h->events[event];
  cudaError_t e;
  if ((e = copy_on(h, h->d_events + event, &nd, sizeof(EventDev), cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(h, e, "event upload");
  relbin_free(E);
  E.dev = nd;
  E.d_rb_edges = ed;
  E.d_rb_q0 = q0;
  E.d_rb_a = a;
  E.d_rb_b = b;
  NsState& S = E.ns;
  if (S.live_u && S.live_lnl && S.n_live > 0) {
    if ((e = launch_unit_likelihood(h->precision, h->waveform, E.n_det, h->d_events + event, S.live_u, S.n_live,
                                    S.live_lnl, h->stream)) != cudaSuccess)
      return cuda_fail(h, e, "initial likelihoods");
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return cuda_fail(h, e, "initial likelihoods");
  }
  return NS_OK;
}

// The coarse-bin edge rule (Zackay, Dai & Venumadhav 2018): a coarse bin ends where the largest
// phase difference a template can have from the fiducial could have changed by eps radians.
// That difference is bounded by a sum of the phase's power laws f^g (g = -5/3, -2/3, 1, 5/3,
// 7/3), each normalised at the end of the band where it is largest:
// dpsi(f) = 2 pi sum_g sign(g) (f / f_g)^g, f_g = f_min for g < 0 and the band's top for g > 0.
// Each edge is the first grid bin whose dpsi differs from the previous edge's by more than eps
// (a coarse bin holds at least one grid bin).
extern "C" int ns_relbin_edges(double f_min, double df, int n_bins, double eps, int32_t* edges, int cap,
                               int32_t* n_edges) {
  if (!(f_min > 0.0) || !(df > 0.0) || n_bins < 1 || !(eps > 0.0) || !std::isfinite(f_min + df + eps) || !n_edges ||
      cap < 0 || (cap > 0 && !edges))
    return NS_EINVAL;
  static const double g[5] = {-5.0 / 3.0, -2.0 / 3.0, 1.0, 5.0 / 3.0, 7.0 / 3.0};
  const double f_top = f_min + df * (double)(n_bins - 1);
  std::vector<double> dpsi(n_bins);
  for (int k = 0; k < n_bins; ++k) {
    const double f = f_min + df * (double)k;
    double s = 0.0;
    for (int i = 0; i < 5; ++i) {
      const double ref = g[i] < 0.0 ? f_min : f_top;
      s += (g[i] < 0.0 ? -1.0 : 1.0) * 2.0 * M_PI * std::pow(f / ref, g[i]);
    }
    dpsi[k] = s;
  }
  int32_t count = 0;
  auto put = [&](int32_t v) {
    if (count < cap) edges[count] = v;
    ++count;
  };
  int last = 0;
  put(0);
  for (int k = 1; k < n_bins; ++k) {
    if (std::fabs(dpsi[k] - dpsi[last]) > eps) {
      put(k);
      last = k;
    }
  }
  put(n_bins);
  *n_edges = count;
  return count <= cap ? NS_OK : NS_EINVAL;
}

extern "C" int ns_relbin_set(ns_handle* h, int event, const int32_t* edges, int n_edges, const double* theta0) {
  if (!h) return set_error(nullptr, NS_EINVAL, "handle is NULL");
  if (event < 0 || event >= (int)h->events.size()) return set_error(h, NS_EINVAL, "event out of range");
  if (h->precision != NS_PREC_MIXED_FF)
    return set_error(h, NS_EINVAL, "relative binning runs on the float-float precision (NS_PREC_MIXED_FF)");
  EventHost& E = h->events[event];
  const bool stepped = (size_t)event < h->host_ns.size() &&
                       (h->host_ns[event].iteration != 0 || h->host_ns[event].n_dead != 0);
  if (stepped)
    return set_error(h, NS_EINVAL, "relative binning is set before the first ns_step of the event");
  const int nbins = E.n_bins, nd = E.n_det;
  if (n_edges != 0) {
    if (n_edges < 2 || !edges || !theta0) return set_error(h, NS_EINVAL, "need at least 2 edges and theta0");
    if (edges[0] != 0 || edges[n_edges - 1] != nbins)
      return set_error(h, NS_EINVAL, "edges must run from 0 to n_bins = %d", nbins);
    for (int i = 1; i < n_edges; ++i)
      if (edges[i] <= edges[i - 1]) return set_error(h, NS_EINVAL, "edges must increase strictly (at %d)", i);
    for (int i = 0; i < kParams; ++i)
      if (!std::isfinite(theta0[i])) return set_error(h, NS_ENONFINITE, "theta0 not finite");
  }
  cudaSetDevice(h->device);
  cudaGetLastError();
  if (n_edges == 0) {
    EventDev nd = E.dev;
    nd.rb_nb = 0;
    nd.rb_edges = nullptr;
    nd.rb_q0 = nullptr;
    nd.rb_a = nullptr;
    nd.rb_b = nullptr;
    return relbin_adopt(h, event, nd, nullptr, nullptr, nullptr, nullptr);
  }
  const int nb = n_edges - 1;
  // the fiducial, continued above its cutoff, and the event's weighted data
  const size_t nh = (size_t)nd * nbins;
  int r;
  if ((r = ensure_scratch(h, h->scratch_in, sizeof(double) * kParams))) return r;
  if ((r = ensure_scratch(h, h->scratch_out, 2 * sizeof(double) * nh))) return r;
  double* d_th = (double*)h->scratch_in.ptr;
  double* d_re = (double*)h->scratch_out.ptr;
  double* d_im = d_re + nh;
  std::vector<double> h0re(nh), h0im(nh), gw(nh);
  std::vector<double2> z(nh);
  cudaStream_t s = h->stream;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(d_th, theta0, sizeof(double) * kParams, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = launch_waveform(h->waveform, nd, h->d_events + event, d_th, 1, nbins, d_re, d_im, s, 1)) != cudaSuccess ||
      (e = cudaMemcpyAsync(h0re.data(), d_re, sizeof(double) * nh, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(h0im.data(), d_im, sizeof(double) * nh, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(z.data(), E.d_z64, sizeof(double2) * nh, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(gw.data(), E.d_gw64, sizeof(double) * nh, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return cuda_fail(h, e, "fiducial waveform");
  // summary data (FP64), then their FP32 copies
  const double f_min = E.dev.f_min, df = E.dev.df;
  std::vector<float2> q0((size_t)nd * nb), a((size_t)nd * nb * 2);
  std::vector<float4> b((size_t)nd * nb);
  for (int d = 0; d < nd; ++d) {
    for (int c = 0; c < nb; ++c) {
      double a0r = 0, a0i = 0, a1r = 0, a1i = 0, b0 = 0, b1 = 0, b2 = 0;
      for (int k = edges[c]; k < edges[c + 1]; ++k) {
        const size_t o = (size_t)d * nbins + k;
        const double f = f_min + df * (double)k;
        const double x = df * (double)(k - edges[c]);
        // h0 f^(7/6): z = 4 df conj(d) f^(-7/6) / S and gw = 4 df f^(-7/3) / S carry the rest
        const double a76 = std::pow(f, 7.0 / 6.0);
        const double hr = h0re[o] * a76, hi = h0im[o] * a76;
        const double cr = z[o].x * hr - z[o].y * hi, ci = z[o].x * hi + z[o].y * hr;   // conj(d) h0 w
        const double p0 = gw[o] * (hr * hr + hi * hi);                                  // |h0|^2 w
        a0r += cr;
        a0i += ci;
        a1r += cr * x;
        a1i += ci * x;
        b0 += p0;
        b1 += p0 * x;
        b2 += p0 * x * x;
      }
      const size_t o = (size_t)d * nb + c;
      a[2 * o] = make_float2((float)a0r, (float)a0i);
      a[2 * o + 1] = make_float2((float)a1r, (float)a1i);
      b[o] = make_float4((float)b0, (float)b1, (float)b2, 0.0f);
      // q0 = f^(-7/6) / (h0 2^70) at the edge: the kernels form h f^(7/6) 2^70 and multiply
      const size_t oe = (size_t)d * nbins + edges[c];
      const double fe = f_min + df * (double)edges[c];
      const double a76 = std::ldexp(std::pow(fe, 7.0 / 6.0), kKpScaleExp);
      const double hr = h0re[oe] * a76, hi = h0im[oe] * a76;
      const double m2 = hr * hr + hi * hi;
      const double qr = hr / m2, qi = -hi / m2;
      if (!(m2 > 0.0) || !std::isfinite(qr) || !std::isfinite(qi) || std::fabs(qr) > 1e37 || std::fabs(qi) > 1e37)
        return set_error(h, NS_EINVAL, "the fiducial vanishes (beyond FP32 range) at edge %d of detector %d", c, d);
      q0[o] = make_float2((float)qr, (float)qi);
      if (!std::isfinite(a0r + a0i + a1r + a1i + b0 + b1 + b2))
        return set_error(h, NS_ENONFINITE, "summary data not finite (coarse bin %d, detector %d)", c, d);
    }
  }
  // new arrays first; the event keeps its current ones until the new descriptor is on the device
  int32_t* ned = nullptr;
  float2 *nq0 = nullptr, *na = nullptr;
  float4* nbb = nullptr;
  auto drop = [&]() {
    cudaFree(ned);
    cudaFree(nq0);
    cudaFree(na);
    cudaFree(nbb);
  };
  if ((e = cudaMalloc(&ned, sizeof(int32_t) * (nb + 1))) != cudaSuccess ||
      (e = cudaMalloc(&nq0, sizeof(float2) * q0.size())) != cudaSuccess ||
      (e = cudaMalloc(&na, sizeof(float2) * a.size())) != cudaSuccess ||
      (e = cudaMalloc(&nbb, sizeof(float4) * b.size())) != cudaSuccess) {
    drop();
    return set_error(h, NS_ENOMEM, "relative-binning allocation failed: %s", cudaGetErrorString(e));
  }
  if ((e = copy_on(h, ned, edges, sizeof(int32_t) * (nb + 1), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = copy_on(h, nq0, q0.data(), sizeof(float2) * q0.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = copy_on(h, na, a.data(), sizeof(float2) * a.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = copy_on(h, nbb, b.data(), sizeof(float4) * b.size(), cudaMemcpyHostToDevice)) != cudaSuccess) {
    drop();
    return cuda_fail(h, e, "relative-binning upload");
  }
  EventDev ndev = E.dev;
  ndev.rb_nb = nb;
  ndev.rb_edges = ned;
  ndev.rb_q0 = nq0;
  ndev.rb_a = na;
  ndev.rb_b = nbb;
  r = relbin_adopt(h, event, ndev, ned, nq0, na, nbb);
  if (r && E.d_rb_edges != ned) drop();   // the descriptor upload failed: the old state stands
  return r;
}
