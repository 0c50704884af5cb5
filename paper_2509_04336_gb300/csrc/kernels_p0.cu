// kernels_p0.cu -- kernels of precision 0 (FP64).
#include <cmath>

#include "kernels_impl.cuh"

namespace gwns {

template cudaError_t launch_likelihood_p<0>(int, int, const EventDev*, const double*, int, double*, int32_t*,
                                             cudaStream_t);
template cudaError_t launch_unit_likelihood_p<0>(int, int, const EventDev*, const double*, int, double*,
                                                  cudaStream_t);
template cudaError_t launch_walk_p<0>(int, int, const EventDev*, WalkTask*, const int32_t*, const int32_t*, int,
                                       cudaStream_t, bool);
template cudaError_t launch_hrss_p<0>(int, int, const EventDev*, WalkTask*, const int32_t*, const int32_t*, int,
                                       cudaStream_t);

cudaError_t launch_unit_to_theta(const EventDev* d_ev, const double* d_u, int64_t n, double* d_theta,
                                 cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  unit_to_theta_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(d_ev, d_u, n, d_theta);
  return cudaGetLastError();
}

cudaError_t launch_waveform(int waveform, int n_det, const EventDev* d_ev, const double* d_theta, int n, int n_bins,
                            double* d_hre, double* d_him, cudaStream_t s, int no_cutoff) {
  if (n <= 0) return cudaSuccess;
  dim3 grid((n_bins + 255) / 256, n);
#define GWNS_WF(P_, N, W) waveform_kernel<N, W><<<grid, 256, 0, s>>>(d_ev, d_theta, n_bins, d_hre, d_him, no_cutoff)
  GWNS_DISPATCH_W(GWNS_WF, 0)
#undef GWNS_WF
  return cudaGetLastError();
}

// The FP64 path's angle table (sincos_phase_f64): (sin, cos)(2 pi k / 256) from long-double host
// values, into this translation unit's copy of g_turn_tab, which its kernels read.
cudaError_t turn_table_upload(cudaStream_t s) {
  double2 t[256];
  const long double two_pi = 6.283185307179586476925286766559005768L;
  for (int k = 0; k < 256; ++k) {
    const long double a = two_pi * (long double)k / 256.0L;
    t[k] = make_double2((double)sinl(a), (double)cosl(a));
  }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_turn_tab);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p, t, sizeof(t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

}  // namespace gwns
