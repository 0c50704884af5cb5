// kernels.cu -- precision dispatch of the kernel launchers (kernels_p{0,1,2}.cu).
#include "gwns_internal.h"

namespace gwns {

template <int P>
cudaError_t launch_likelihood_p(int waveform, int n_det, const EventDev* d_ev, const double* d_theta, int n,
                                double* d_lnl, int32_t* d_status, cudaStream_t s);
template <int P>
cudaError_t launch_unit_likelihood_p(int waveform, int n_det, const EventDev* d_ev, const double* d_u, int n,
                                     double* d_lnl, cudaStream_t s);
template <int P>
cudaError_t launch_walk_p(int waveform, int n_det, const EventDev* d_evs, WalkTask* d_tasks,
                          const int32_t* d_blk_task, const int32_t* d_blk_local, int n_blocks, cudaStream_t s,
                          bool extras);
template <int P>
cudaError_t launch_hrss_p(int waveform, int n_det, const EventDev* d_evs, WalkTask* d_tasks,
                          const int32_t* d_blk_task, const int32_t* d_blk_local, int n_blocks, cudaStream_t s);

cudaError_t launch_likelihood(int precision, int waveform, int n_det, const EventDev* d_ev, const double* d_theta,
                              int n, double* d_lnl, int32_t* d_status, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (precision == 0) return launch_likelihood_p<0>(waveform, n_det, d_ev, d_theta, n, d_lnl, d_status, s);
  if (precision == 1) return launch_likelihood_p<1>(waveform, n_det, d_ev, d_theta, n, d_lnl, d_status, s);
  return launch_likelihood_p<2>(waveform, n_det, d_ev, d_theta, n, d_lnl, d_status, s);
}

cudaError_t launch_unit_likelihood(int precision, int waveform, int n_det, const EventDev* d_ev, const double* d_u,
                                   int n, double* d_lnl, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (precision == 0) return launch_unit_likelihood_p<0>(waveform, n_det, d_ev, d_u, n, d_lnl, s);
  if (precision == 1) return launch_unit_likelihood_p<1>(waveform, n_det, d_ev, d_u, n, d_lnl, s);
  return launch_unit_likelihood_p<2>(waveform, n_det, d_ev, d_u, n, d_lnl, s);
}

cudaError_t launch_walk(int precision, int waveform, int n_det, const EventDev* d_evs, WalkTask* d_tasks,
                        const int32_t* d_blk_task, const int32_t* d_blk_local, int n_blocks, cudaStream_t s,
                        bool extras) {
  if (n_blocks <= 0) return cudaSuccess;
  if (precision == 0)
    return launch_walk_p<0>(waveform, n_det, d_evs, d_tasks, d_blk_task, d_blk_local, n_blocks, s, extras);
  if (precision == 1)
    return launch_walk_p<1>(waveform, n_det, d_evs, d_tasks, d_blk_task, d_blk_local, n_blocks, s, extras);
  return launch_walk_p<2>(waveform, n_det, d_evs, d_tasks, d_blk_task, d_blk_local, n_blocks, s, extras);
}

cudaError_t launch_hrss(int precision, int waveform, int n_det, const EventDev* d_evs, WalkTask* d_tasks,
                        const int32_t* d_blk_task, const int32_t* d_blk_local, int n_blocks, cudaStream_t s) {
  if (n_blocks <= 0) return cudaSuccess;
  if (precision == 0) return launch_hrss_p<0>(waveform, n_det, d_evs, d_tasks, d_blk_task, d_blk_local, n_blocks, s);
  if (precision == 1) return launch_hrss_p<1>(waveform, n_det, d_evs, d_tasks, d_blk_task, d_blk_local, n_blocks, s);
  return launch_hrss_p<2>(waveform, n_det, d_evs, d_tasks, d_blk_task, d_blk_local, n_blocks, s);
}

}  // namespace gwns
