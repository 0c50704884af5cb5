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

// Publishes E.dev to the device copy and re-evaluates the initial live points with the
// likelihood now in effect.
static int relbin_publish(ns_handle* h, int event) {
  EventHost& E = h->events[event];
  cudaError_t e;
  if ((e = cudaMemcpy(h->d_events + event, &E.dev, sizeof(EventDev), cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(h, e, "event upload");
  NsState& S = E.ns;
  if (S.live_u && S.live_lnl && S.n_live > 0) {
    if ((e = launch_unit_likelihood(h->precision, h->waveform, E.n_det, h->d_events + event, S.live_u, S.n_live,
                                    S.live_lnl, h->stream)) != cudaSuccess)
      return cuda_fail(h, e, "initial likelihoods");
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return cuda_fail(h, e, "initial likelihoods");
  }
  return NS_OK;
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
    relbin_free(E);
    return relbin_publish(h, event);
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
  relbin_free(E);
  if ((e = cudaMalloc(&E.d_rb_edges, sizeof(int32_t) * (nb + 1))) != cudaSuccess ||
      (e = cudaMalloc(&E.d_rb_q0, sizeof(float2) * q0.size())) != cudaSuccess ||
      (e = cudaMalloc(&E.d_rb_a, sizeof(float2) * a.size())) != cudaSuccess ||
      (e = cudaMalloc(&E.d_rb_b, sizeof(float4) * b.size())) != cudaSuccess) {
    relbin_free(E);
    return set_error(h, NS_ENOMEM, "relative-binning allocation failed: %s", cudaGetErrorString(e));
  }
  if ((e = cudaMemcpy(E.d_rb_edges, edges, sizeof(int32_t) * (nb + 1), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(E.d_rb_q0, q0.data(), sizeof(float2) * q0.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(E.d_rb_a, a.data(), sizeof(float2) * a.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(E.d_rb_b, b.data(), sizeof(float4) * b.size(), cudaMemcpyHostToDevice)) != cudaSuccess) {
    relbin_free(E);
    return cuda_fail(h, e, "relative-binning upload");
  }
  E.dev.rb_nb = nb;
  E.dev.rb_edges = E.d_rb_edges;
  E.dev.rb_q0 = E.d_rb_q0;
  E.dev.rb_a = E.d_rb_a;
  E.dev.rb_b = E.d_rb_b;
  return relbin_publish(h, event);
}
