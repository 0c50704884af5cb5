// noalloc.cu -- ns_walk_batch_noalloc: the acceptance walk of ns_walk_batch for callers
// that must not allocate device memory after start-up.
//
// ns_walk_batch keeps the walk's task descriptor and its block -> walker map in device
// scratch that it grows with cudaMalloc on demand.  Some callers cannot let a library do
// that in the middle of a run: a process that reserves a fixed device-memory budget at
// start-up and forbids any later cudaMalloc, or a latency-critical loop that cannot absorb
// the implicit device synchronisation of cudaMalloc/cudaFree.  This entry point puts the
// same scratch in a file-scope __device__ array instead, so a call allocates nothing.
//
// Notes for users:
//  * The array holds one task descriptor and block maps for at most kNoAllocMaxWalkers
//    walkers; every GPU that loads the library holds it (about 64 KB) until the process exits.
//  * The array's address is looked up with cudaGetSymbolAddress on the first call made on
//    each device (with that device current).  Make that first call before any stream
//    capture that should contain a later call.
//  * Every call shares the one array.  Calls whose kernels overlap on the GPU (different
//    streams, or different handles on the same device) race on it: order them on one stream.
//  * All array arguments are device pointers; the work is enqueued on `stream` (NULL: the
//    handle's stream) and the call returns without waiting for it.
//  * An event with flow proposals (NS_PROPOSAL_DE_FLOW, p_flow > 0) writes its proposal table
//    into the handle's own batch table, which ns_step also uses: then n <= num_delete and
//    n_steps <= maxmcmc, and a call must not overlap an ns_step of the same handle.
#include <cstring>
#include <mutex>

#include "api_internal.h"

using namespace gwns;

namespace {

constexpr int kNoAllocMaxWalkers = 8192;
constexpr int kMaxDevices = 64;
constexpr size_t kTaskBytes = 256;   // WalkTask slot, padded to keep the maps 256-byte aligned
static_assert(sizeof(WalkTask) <= kTaskBytes, "WalkTask must fit its slot");
constexpr size_t kScratchBytes = kTaskBytes + 2 * sizeof(int32_t) * kNoAllocMaxWalkers;

// Walk scratch: [WalkTask | blk_task[kNoAllocMaxWalkers] | blk_local[kNoAllocMaxWalkers]].
static __device__ __align__(256) unsigned char g_walk_scratch[kScratchBytes];

void* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

// Writes the task descriptor and the block maps (one task, walker j on block j).  Nothing
// in the scratch needs to start at zero: every field the walk reads is written here.
__global__ void fill_walk_scratch(unsigned char* scratch, WalkTask task, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  int32_t* blk_task = (int32_t*)(scratch + kTaskBytes);
  int32_t* blk_local = blk_task + kNoAllocMaxWalkers;
  if (i == 0) *(WalkTask*)scratch = task;
  if (i < n) {
    blk_task[i] = 0;
    blk_local[i] = i;
  }
}

// Device address of g_walk_scratch on `device` (looked up once per device).
int scratch_for_device(ns_handle* h, int device, unsigned char** out) {
  if (device < 0 || device >= kMaxDevices) return set_error(h, NS_EINVAL, "device %d out of range", device);
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_walk_scratch);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGetSymbolAddress(g_walk_scratch)");
    g_scratch_ptr[device] = p;
  }
  *out = (unsigned char*)g_scratch_ptr[device];
  return NS_OK;
}

}  // namespace

extern "C" int ns_walk_batch_noalloc(ns_handle* h, int event, const double* live_u, int n_live_pts,
                                     const double* u0, const double* lnl0, double lnl_star, int n, int n_steps,
                                     int64_t iteration, int64_t walker_offset, double* u_out, double* lnl_out,
                                     int32_t* n_accept, int32_t* n_like, void* stream) {
  if (!h) return set_error(nullptr, NS_EINVAL, "handle is NULL");
  if (event < 0 || event >= (int)h->events.size()) return set_error(h, NS_EINVAL, "event out of range");
  if (n < 0 || n_steps < 0 || n_live_pts < 2 || iteration < 0 || walker_offset < 0)
    return set_error(h, NS_EINVAL, "need n >= 0, n_steps >= 0, n_live_pts >= 2, iteration >= 0, walker_offset >= 0");
  if (n > kNoAllocMaxWalkers)
    return set_error(h, NS_EINVAL, "ns_walk_batch_noalloc takes at most %d walkers per call (got %d)",
                     kNoAllocMaxWalkers, n);
  if (n > 0 && (!live_u || !u0 || !lnl0 || !u_out || !lnl_out || !n_accept || !n_like))
    return set_error(h, NS_EINVAL, "null array");
  if (lnl_star != lnl_star) return set_error(h, NS_ENONFINITE, "lnl_star is NaN");
  if (n == 0) return NS_OK;
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
  cudaGetLastError();
  unsigned char* scratch = nullptr;
  int r = scratch_for_device(h, h->device, &scratch);
  if (r) return r;
  const EventHost& E = h->events[event];
  WalkTask T;
  std::memset(&T, 0, sizeof(T));
  T.surv = live_u; T.u0 = u0; T.lnl0 = lnl0; T.u_out = u_out; T.lnl_out = lnl_out;
  T.n_acc = n_accept; T.n_like = n_like; T.n_bins = nullptr;
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
  cudaStream_t s = stream ? (cudaStream_t)stream : h->stream;
  // the flow kernels' timeout flag and the walk watchdog's bit start clear, as in ns_walk_batch
  if ((e = cudaMemsetAsync(h->d_status + 1, 0, sizeof(int32_t) * 2, s)) != cudaSuccess)
    return cuda_fail(h, e, "status reset");
  // flow steps draw on the handle's own proposal table, allocated at ns_init
  r = flow_attach(h, event, T, n, n_steps, nullptr, s);
  if (r) return r;
  fill_walk_scratch<<<(n + 255) / 256, 256, 0, s>>>(scratch, T, n);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(h, e, "scratch fill launch");
  WalkTask* d_task = (WalkTask*)scratch;
  const int32_t* d_bt = (const int32_t*)(scratch + kTaskBytes);
  const int32_t* d_bl = d_bt + kNoAllocMaxWalkers;
  e = launch_walk(h->precision, h->waveform, E.n_det, h->d_events, d_task, d_bt, d_bl, n, s, walk_extras(h, event));
  return e == cudaSuccess ? NS_OK : cuda_fail(h, e, "walk launch");
}
