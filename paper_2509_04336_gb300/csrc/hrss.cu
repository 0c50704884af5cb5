// hrss.cu -- ns_hrss_batch: one batch of hit-and-run slice-sampling moves (the inner kernel
// the paper names as the vectorised framework's original choice, Sec. 2.2, and as the way
// forward for GPU-native inner kernels, Sec. 5).  The host forms the Cholesky factor of the
// survivors' covariance (D <= 11, FP64) and hrss_kernel (the handle's precision) runs the moves;
// inside ns_step the same kernel runs after chol_kernel forms the factor on the device.
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/gwns.h"
#include "api_internal.h"

using namespace gwns;

extern "C" int ns_hrss_batch(ns_handle* h, int event, const double* live_u, int n_live_pts, const double* u0,
                             const double* lnl0, double lnl_star, int n, int n_steps, int64_t iteration,
                             int64_t walker_offset, double* u_out, double* lnl_out, int32_t* n_move,
                             int32_t* n_like) {
  if (!h) return set_error(nullptr, NS_EINVAL, "handle is NULL");
  if (event < 0 || event >= (int)h->events.size()) return set_error(h, NS_EINVAL, "event out of range");
  if (n < 0 || n_steps < 0 || n_live_pts < 2 || iteration < 0 || walker_offset < 0)
    return set_error(h, NS_EINVAL, "need n >= 0, n_steps >= 0, n_live_pts >= 2, iteration >= 0, walker_offset >= 0");
  if (n > 0 && (!live_u || !u0 || !lnl0 || !u_out || !lnl_out || !n_move || !n_like))
    return set_error(h, NS_EINVAL, "null array");
  if (std::isnan(lnl_star)) return set_error(h, NS_ENONFINITE, "lnl_star is NaN");
  if (n == 0) return NS_OK;
  EventHost& E = h->events[event];
  const int D = E.n_dim;
  const size_t ns_ = (size_t)n_live_pts * D, nu = (size_t)n * D;
  for (size_t i = 0; i < ns_; ++i)
    if (!std::isfinite(live_u[i])) return set_error(h, NS_ENONFINITE, "live_u not finite");
  for (size_t i = 0; i < nu; ++i)
    if (!std::isfinite(u0[i])) return set_error(h, NS_ENONFINITE, "u0 not finite");
  // survivors' sample covariance (divisor n - 1) and its lower Cholesky factor
  std::vector<double> mean(D, 0.0), cov((size_t)D * D, 0.0), L((size_t)D * D, 0.0);
  for (int p = 0; p < n_live_pts; ++p)
    for (int i = 0; i < D; ++i) mean[i] += live_u[(size_t)p * D + i];
  for (int i = 0; i < D; ++i) mean[i] /= (double)n_live_pts;
  for (int p = 0; p < n_live_pts; ++p)
    for (int i = 0; i < D; ++i)
      for (int k = 0; k <= i; ++k)
        cov[(size_t)i * D + k] += (live_u[(size_t)p * D + i] - mean[i]) * (live_u[(size_t)p * D + k] - mean[k]);
  for (int i = 0; i < D; ++i)
    for (int k = 0; k <= i; ++k) cov[(size_t)i * D + k] /= (double)(n_live_pts - 1);
  for (int i = 0; i < D; ++i)
    for (int k = 0; k <= i; ++k) {
      double s = cov[(size_t)i * D + k];
      for (int m = 0; m < k; ++m) s -= L[(size_t)i * D + m] * L[(size_t)k * D + m];
      if (i == k) {
        // a pivot at rounding level of the variance: the survivors span fewer than D directions
        if (!(s > 1e-12 * cov[(size_t)i * D + i]) || !(s > 0.0))
          return set_error(h, NS_EINVAL, "survivor covariance is not positive definite");
        L[(size_t)i * D + i] = std::sqrt(s);
      } else {
        L[(size_t)i * D + k] = s / L[(size_t)k * D + k];
      }
    }
  cudaSetDevice(h->device);
  cudaGetLastError();
  cudaStream_t s = h->stream;
  // task, block maps, factor and starts in one upload; outputs in the output scratch
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
  T.event = event;
  T.spec = E.cfg.spec_depth > 0 ? E.cfg.spec_depth : hrss_default_spec(h->waveform);
  watchdog_fields(h, T);
  const size_t task_b = (sizeof(WalkTask) + 255) / 256 * 256;
  const size_t maps_b = (2 * sizeof(int32_t) * (size_t)n + 255) / 256 * 256;
  const size_t in_b = task_b + maps_b + sizeof(double) * ((size_t)D * D + nu + n);
  const size_t out_b = sizeof(double) * (nu + n) + 2 * sizeof(int32_t) * n;
  int r;
  if ((r = ensure_scratch(h, h->scratch_in, in_b))) return r;
  if ((r = ensure_scratch(h, h->scratch_out, out_b))) return r;
  char* base = (char*)h->scratch_in.ptr;
  WalkTask* d_task = (WalkTask*)base;
  int32_t* d_bt = (int32_t*)(base + task_b);
  int32_t* d_bl = d_bt + n;
  double* d_chol = (double*)(base + task_b + maps_b);
  double* d_u0 = d_chol + (size_t)D * D;
  double* d_l0 = d_u0 + nu;
  double* d_uo = (double*)h->scratch_out.ptr;
  double* d_lo = d_uo + nu;
  int32_t* d_nm = (int32_t*)(d_lo + n);
  int32_t* d_nl = d_nm + n;
  T.chol = d_chol; T.u0 = d_u0; T.lnl0 = d_l0; T.u_out = d_uo; T.lnl_out = d_lo; T.n_acc = d_nm; T.n_like = d_nl;
  std::vector<char> stage(task_b + maps_b, 0);
  std::memcpy(stage.data(), &T, sizeof(T));
  int32_t* bt = (int32_t*)(stage.data() + task_b);
  for (int j = 0; j < n; ++j) { bt[j] = 0; bt[n + j] = j; }
  cudaError_t e;
  if ((e = cudaMemsetAsync(h->d_status + 2, 0, sizeof(int32_t), s)) ||
      (e = cudaMemcpyAsync(base, stage.data(), stage.size(), cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(d_chol, L.data(), sizeof(double) * L.size(), cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(d_u0, u0, sizeof(double) * nu, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(d_l0, lnl0, sizeof(double) * n, cudaMemcpyHostToDevice, s)))
    return cuda_fail(h, e, "H2D hrss inputs");
  if ((e = launch_hrss(h->precision, h->waveform, E.n_det, h->d_events, d_task, d_bt, d_bl, n, s)) != cudaSuccess)
    return cuda_fail(h, e, "hrss launch");
  if ((e = cudaMemcpyAsync(u_out, d_uo, sizeof(double) * nu, cudaMemcpyDeviceToHost, s)) ||
      (e = cudaMemcpyAsync(lnl_out, d_lo, sizeof(double) * n, cudaMemcpyDeviceToHost, s)) ||
      (e = cudaMemcpyAsync(n_move, d_nm, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s)) ||
      (e = cudaMemcpyAsync(n_like, d_nl, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s)))
    return cuda_fail(h, e, "D2H hrss outputs");
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(h, e, "hrss");
  return watchdog_report(h);
}
