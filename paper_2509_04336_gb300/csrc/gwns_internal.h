// gwns_internal.h -- host-side declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gwns_model.cuh"

namespace gwns {

constexpr int kThreads = 128;   // threads per walker CTA

// Per-event descriptor of one walk batch, read by the walk kernel.  The nested-sampling
// kernels rewrite lnl_star, n_steps and iteration between batches, so a captured graph
// replays without host involvement.
struct WalkTask {
  const double* surv;      // [n_s][D] survivors
  const float2* survf;     // [n_s][D] float-float copy (h, l) of surv (may be null)
  const double* u0;        // [n][D] starts
  const double* lnl0;      // [n]
  double* u_out;           // [n][D]
  double* lnl_out;         // [n]
  int32_t* n_acc;          // [n]
  int32_t* n_like;         // [n]
  int64_t* n_bins;         // [n] active bins evaluated per walker (may be null)
  int64_t* n_spec;         // [n] likelihoods evaluated speculatively, used or not (may be null)
  int32_t* n_acc_flow;     // [n] accepted flow steps, of n_acc (may be null)
  double lnl_star;
  int64_t iteration;
  int64_t walker_offset;
  uint64_t key0, key1;
  int32_t n_s;
  int32_t n;
  int32_t n_steps;
  int32_t done;
  int32_t event;           // index into the event table
  int32_t spec;            // proposals evaluated per round (1 .. kSpecMax)
  // flow steps (null flow: DE only).  Step t of walker w is a flow step when Philox word
  // (t, walker_offset + w, iteration, 6)[0] gives U < p_flow; its proposal and log q are
  // entry (w, t) of the proposal table [n][f_stride].
  const struct FlowDev* flow;
  const double* fu;        // [n][f_stride][D]
  const double* flq;       // [n][f_stride]
  double p_flow;
  int32_t f_stride;
  int32_t pad_;
  // hit-and-run slice sampling (HRSS) tasks: the lower Cholesky factor [D][D] of the
  // survivors' covariance; n_steps counts moves
  const double* chol;
  // watchdog: a walk ends after the round in which *abort is nonzero or more than budget_ns
  // nanoseconds (globaltimer) have passed since its CTA started (0: no budget); it then sets
  // bit 0 of *status (null pointers: no watchdog)
  const int32_t* abort;
  int32_t* status;
  uint64_t budget_ns;
};

constexpr int kSpecMax = 32;   // speculation depth limit (one warp of proposals)

// Launch wrappers (kernels.cu).  Every wrapper returns the launch error.  precision:
// NS_PREC_*; waveform: NS_WAVEFORM_*.
cudaError_t launch_likelihood(int precision, int waveform, int n_det, const EventDev* d_ev, const double* d_theta,
                              int n, double* d_lnl, int32_t* d_status, cudaStream_t s);
cudaError_t launch_unit_likelihood(int precision, int waveform, int n_det, const EventDev* d_ev, const double* d_u,
                                   int n, double* d_lnl, cudaStream_t s);
cudaError_t launch_unit_to_theta(const EventDev* d_ev, const double* d_u, int64_t n, double* d_theta,
                                 cudaStream_t s);
// no_cutoff: continue the template above its cutoff (the relative-binning fiducial).
cudaError_t launch_waveform(int waveform, int n_det, const EventDev* d_ev, const double* d_theta, int n, int n_bins,
                            double* d_hre, double* d_him, cudaStream_t s, int no_cutoff = 0);
// Block b makes the HRSS moves of walker blk_local[b] of task blk_task[b] (the task's chol,
// n_steps moves; n_acc receives the moves made).
cudaError_t launch_hrss(int precision, int waveform, int n_det, const EventDev* d_evs, WalkTask* d_tasks,
                        const int32_t* d_blk_task, const int32_t* d_blk_local, int n_blocks, cudaStream_t s);
// Fills the FP64 path's angle table on the current device (before any FP64 likelihood runs).
cudaError_t turn_table_upload(cudaStream_t s);
// Block b walks walker blk_local[b] of task blk_task[b].  extras: some task of the launch uses
// flow proposals or the relative-binning likelihood (false lets mode 2 run a walk kernel
// compiled without those paths).
cudaError_t launch_walk(int precision, int waveform, int n_det, const EventDev* d_evs, WalkTask* d_tasks,
                        const int32_t* d_blk_task, const int32_t* d_blk_local, int n_blocks, cudaStream_t s,
                        bool extras);

}  // namespace gwns
