// api_internal.h -- the handle behind the C ABI.
#pragma once

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/gwns.h"
#include "flow_internal.h"
#include "gwns_internal.h"

namespace gwns {

constexpr int kMaxLive = 4096;     // live points per event (one CTA sorts them in shared memory)

struct Scratch {
  void* ptr = nullptr;
  size_t bytes = 0;
};

// Device-resident nested-sampling state of one event.  The batch kernels read and write
// it in place, so a captured graph replays batches without host round trips.  The buffer
// pointers come last, from live_u on: a checkpoint restores the fields before them.
struct NsState {
  double log_x, log_z, lnl_star, dlogz, mean_accept, lnl_max, delay_k, term_value;
  double spec_mult, spec_p;   // speculation rule m = spec_mult / p; p of the last batch
  double flow_w;              // weight of an accepted flow step in the walk-length retune
  double mean_accept_flow;    // mean accepted flow steps per walker, last batch
  int64_t n_dead, n_like, iteration, max_iter, dead_cap, n_bins_eval, n_spec_eval;
  int32_t n_live, k, D, n_steps, naccept, maxmcmc, term_kind, done, zero_accept, overflow;
  int32_t spec, spec_auto, spec_cap, spec_rule;   // spec = min(spec_rule, spec_cap)
  int32_t hrss;        // HRSS inner kernel: moves per walker and batch (0: the DE walk)
  int32_t chol_bad;    // HRSS: the survivors' covariance was not positive definite
  uint64_t key0, key1;
  double* live_u;      // [n_live][D]
  double* live_lnl;    // [n_live]
  double* surv_u;      // [n_live - k][D]
  float2* survf;       // [n_live - k][D] float-float copy (h, l) of surv_u
  double* w_u0;        // [k][D]
  double* w_lnl0;      // [k]
  double* w_uo;        // [k][D]
  double* w_lo;        // [k]
  int32_t* w_na;       // [k]
  int32_t* w_nl;       // [k]
  int32_t* slot;       // [k]
  int64_t* w_nb;       // [k] active bins evaluated per walker
  int64_t* w_ns;       // [k] likelihoods evaluated per walker, speculative ones included
  int32_t* w_naf;      // [k] accepted flow steps per walker (of w_na)
  double* dead_u;      // [dead_cap][D]
  double* dead_lnl;    // [dead_cap]
  double* dead_logw;   // [dead_cap]
  int32_t* dead_nlive; // [dead_cap]
  double* chol;        // HRSS: [D][D] lower Cholesky factor of the survivors' covariance
};

struct EventHost {
  ns_config cfg;
  int n_det = 0, n_bins = 0, n_dim = 0;
  EventDev dev;
  double* d_basis64 = nullptr;
  float2* d_basis_ff = nullptr;
  double2* d_z64 = nullptr;
  float2* d_z32 = nullptr;
  double* d_hh_prefix = nullptr;
  double* d_gw64 = nullptr;
  float* d_gw32 = nullptr;
  float* d_hhp32 = nullptr;
  int32_t* d_rb_edges = nullptr;   // relative binning (relbin.cu)
  float2* d_rb_q0 = nullptr;
  float2* d_rb_a = nullptr;
  float4* d_rb_b = nullptr;
  NsState ns;            // host mirror of the device pointers and static fields
  FlowHost flow;         // flow proposal (enabled for NS_PROPOSAL_DE_FLOW)
};

}  // namespace gwns

struct ns_handle {
  int device = 0;
  int precision = 0;
  int waveform = 0;
  int max_det = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t aux_stream = nullptr;   // ns_set_abort's writes, not ordered with the walks
  bool hrss = false;                   // every event uses the HRSS inner kernel
  uint64_t budget_ns = 0;              // watchdog time budget of a walk (0: none)
  std::vector<gwns::EventHost> events;
  gwns::EventDev* d_events = nullptr;
  int32_t* d_status = nullptr;
  gwns::Scratch scratch_in, scratch_out, scratch_map, scratch_flow, scratch_shard;
  bool batch_open = false;   // ns_batch_begin ran; ns_batch_end closes the batch
  // nested sampling
  gwns::NsState* d_ns = nullptr;
  gwns::WalkTask* d_tasks = nullptr;
  int32_t* d_blk_task = nullptr;
  int32_t* d_blk_local = nullptr;
  int n_walk_blocks = 0;
  cudaGraphExec_t graph_exec[9] = {};   // instantiated batch graphs, indexed by batches per replay
  std::vector<cudaEvent_t> walk_events;  // [2 * batches in the graph]: start, end of each walk
  double walk_ms = 0.0;
  int64_t kernel_launches = 0;
  int64_t launches_per_batch[9] = {};   // kernels in each cached graph, per batch count
  // speculation-depth autotuner (all events in automatic mode): picks the cap
  bool tune = false;
  bool tune_guessed = false;         // first cap set from the cost structure (after batch 1)
  int tune_next = 64;                // iteration at which the next tuning pass starts
  int tune_idx = -1;                 // step of the tuning pass, -1 when not tuning
  double tune_ms[8] = {0}, tune_calls[8] = {0};   // per candidate, summed over its trials
  int tune_best = 32;
  std::vector<gwns::NsState> host_ns;   // last progress snapshot
  std::string err;
};

int set_error(ns_handle* h, int code, const char* fmt, ...);
void watchdog_fields(ns_handle* h, gwns::WalkTask& T);
int watchdog_report(ns_handle* h);
int cuda_fail(ns_handle* h, cudaError_t e, const char* what);
// A copy (fill) ordered on the handle's stream -- after the work enqueued there, before the work
// enqueued later -- and complete on return.  The handle's stream is non-blocking, so a plain
// cudaMemcpy / cudaMemset (legacy default stream) is ordered with neither, and it returns before
// a device-to-device copy, a fill or the DMA of a host-to-device copy has landed.
cudaError_t copy_on(ns_handle* h, void* dst, const void* src, size_t bytes, cudaMemcpyKind kind);
cudaError_t fill_on(ns_handle* h, void* dst, int value, size_t bytes);
int ensure_scratch(ns_handle* h, gwns::Scratch& s, size_t bytes);
int nested_init(ns_handle* h);
int default_spec(int precision);
int hrss_default_spec(int waveform);
// Whether a walk of event e (of any event of the handle) uses flow proposals or the
// relative-binning likelihood: launch_walk's extras.
bool walk_extras(const ns_handle* h, int e);
bool walk_extras(const ns_handle* h);
void nested_free(ns_handle* h);
void relbin_free(gwns::EventHost& E);
// flow proposal (flow_api.cu)
int flow_check_config(const ns_config& c, int e);
int flow_setup(ns_handle* h, int e);
void flow_free(gwns::EventHost& E);
void flow_task_fields(const gwns::EventHost& E, gwns::WalkTask& T);
int flow_enqueue_train(ns_handle* h, int e, cudaStream_t s, int64_t* launches);
int flow_enqueue_table(ns_handle* h, int e, cudaStream_t s, int64_t* launches);
int flow_attach(ns_handle* h, int event, gwns::WalkTask& T, int n, int n_steps, gwns::Scratch* table, cudaStream_t s);
bool flow_state_write(ns_handle* h, int e, FILE* f);
// A checkpoint's flow record, read and checked against the handle before anything is applied.
struct FlowBlob {
  bool present = false;
  gwns::FlowDev F;
  std::vector<float> buf;   // master weights, Adam m, Adam v
};
bool flow_state_parse(ns_handle* h, int e, FILE* f, FlowBlob& b);
bool flow_state_apply(ns_handle* h, int e, const FlowBlob& b);
