// flow_api.cu -- the flow proposal's buffers, its place in a sampler batch, and the ns_flow_*
// entry points of the C ABI.
//
// In a batch of an event configured with NS_PROPOSAL_DE_FLOW the graph runs, after the
// deletion, a flag kernel (retrain when iteration % flow_every == 0), the standardisation and
// flow_epochs pairs of (gradient, Adam) launches on the n_live - k survivors -- each returns
// at once when the flag is clear -- and then the proposal table of the batch's walks (one
// inverse-flow sample and its ln q for every (walker, step)).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "api_internal.h"

using namespace gwns;

namespace {

constexpr int kTilesCap = (kMaxLive + kGradRows - 1) / kGradRows;

__global__ void flow_train_flag_kernel(const NsState* S, int every, int32_t* flag) {
  if (threadIdx.x == 0) *flag = (!S->done && S->iteration % every == 0) ? 1 : 0;
}

int sm_count(ns_handle* h) {
  int n = 0;
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, h->device);
  return n > 0 ? n : 1;
}

int falloc(ns_handle* h, void** p, size_t bytes, const char* what) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) return set_error(h, NS_ENOMEM, "cudaMalloc %s (%zu bytes): %s", what, bytes, cudaGetErrorString(e));
  return NS_OK;
}

int check_flow_event(ns_handle* h, int event) {
  if (!h) return set_error(nullptr, NS_EINVAL, "handle is NULL");
  if (event < 0 || event >= (int)h->events.size()) return set_error(h, NS_EINVAL, "event out of range");
  if (!h->events[event].flow.enabled) return set_error(h, NS_ESTATE, "event %d has no flow proposal", event);
  cudaSetDevice(h->device);
  cudaGetLastError();
  return NS_OK;
}

// FlowDev as the host sees it (pointers and sizes), for uploads that must keep them.
FlowDev host_flowdev(const EventHost& E) {
  const FlowHost& Fh = E.flow;
  FlowDev F;
  std::memset(&F, 0, sizeof(F));
  F.n_layers = Fh.n_layers;
  F.n_dim = E.n_dim;
  F.n_params = Fh.n_params;
  F.p_flow = (float)Fh.p_flow;
  for (int d = 0; d < kFlowP; ++d) { F.mu[d] = 0.0f; F.sigma[d] = 1.0f; }
  F.log_sigma_sum = 0.0f;
  F.adam_t = 0;
  F.lr = (float)Fh.lr;
  F.img = Fh.d_img;
  F.bias = Fh.d_bias;
  return F;
}

int check_err_flag(ns_handle* h, cudaStream_t s, const char* what) {
  int32_t st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, h->d_status + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(h, e, what);
  if (st) return set_error(h, NS_ETIMEOUT, "%s: a tensor-core wait timed out", what);
  return NS_OK;
}

}  // namespace

// ---------------------------------------------------------------- setup and teardown
int flow_check_config(const ns_config& c, int e) {
  if (c.proposal != NS_PROPOSAL_DE && c.proposal != NS_PROPOSAL_DE_FLOW && c.proposal != NS_PROPOSAL_HRSS)
    return set_error(nullptr, NS_EINVAL, "event %d: unknown proposal %d", e, c.proposal);
  const bool weight_set = c.flow_accept_weight != 0.0 && c.flow_accept_weight != 1.0;
  if (c.proposal != NS_PROPOSAL_DE_FLOW) {
    if (weight_set) return set_error(nullptr, NS_EINVAL, "event %d: flow_accept_weight is for NS_PROPOSAL_DE_FLOW", e);
    return NS_OK;
  }
  if (!(c.p_flow >= 0.0 && c.p_flow <= 1.0)) return set_error(nullptr, NS_EINVAL, "event %d: p_flow must be in [0, 1]", e);
  if (c.flow_accept_weight != 0.0 && !(c.flow_accept_weight >= 1.0 && c.flow_accept_weight <= 1e6))
    return set_error(nullptr, NS_EINVAL, "event %d: flow_accept_weight must be 0 or in [1, 1e6]", e);
  if (c.flow_layers < 0 || c.flow_layers > kFlowMaxLayers)
    return set_error(nullptr, NS_EINVAL, "event %d: flow_layers must be in 0..%d", e, kFlowMaxLayers);
  if (c.flow_every < 0 || c.flow_epochs < 0 || !(c.flow_lr >= 0.0) || !std::isfinite(c.flow_lr))
    return set_error(nullptr, NS_EINVAL, "event %d: flow_every, flow_epochs, flow_lr must be >= 0", e);
  return NS_OK;
}

int flow_setup(ns_handle* h, int e) {
  EventHost& E = h->events[e];
  const ns_config& c = E.cfg;
  FlowHost& Fh = E.flow;
  if (c.proposal != NS_PROPOSAL_DE_FLOW) return NS_OK;
  cudaError_t err = flow_kernel_setup();
  if (err != cudaSuccess) return cuda_fail(h, err, "flow kernel attributes");
  Fh.enabled = 1;
  Fh.n_layers = c.flow_layers > 0 ? c.flow_layers : 8;
  Fh.every = c.flow_every > 0 ? c.flow_every : 1;
  Fh.epochs = c.flow_epochs > 0 ? c.flow_epochs : 50;
  Fh.lr = c.flow_lr > 0.0 ? c.flow_lr : 3e-3;
  Fh.p_flow = c.p_flow;
  Fh.n_params = Fh.n_layers * flow_layer_params(E.n_dim);
  Fh.tiles_cap = kTilesCap;
  Fh.stride = c.maxmcmc;
  const size_t L = Fh.n_layers, NP = Fh.n_params, k = c.num_delete, D = E.n_dim;
  int r;
  if ((r = falloc(h, (void**)&Fh.d_flow, sizeof(FlowDev), "flow")) ||
      (r = falloc(h, (void**)&Fh.d_img, L * kImgLayer, "flow images")) ||
      (r = falloc(h, (void**)&Fh.d_bias, sizeof(float) * L * kBiasLayer, "flow biases")) ||
      (r = falloc(h, (void**)&Fh.d_master, sizeof(float) * NP, "flow weights")) ||
      (r = falloc(h, (void**)&Fh.d_m, sizeof(float) * NP, "adam m")) ||
      (r = falloc(h, (void**)&Fh.d_v, sizeof(float) * NP, "adam v")) ||
      (r = falloc(h, (void**)&Fh.d_partial, sizeof(float) * NP * Fh.tiles_cap, "flow partial gradients")) ||
      (r = falloc(h, (void**)&Fh.d_loss_part, sizeof(double) * Fh.tiles_cap, "flow losses")) ||
      (r = falloc(h, (void**)&Fh.d_zsave, sizeof(float) * Fh.tiles_cap * L * 128 * kFlowP, "flow layer inputs")) ||
      (r = falloc(h, (void**)&Fh.d_grad, sizeof(float) * NP, "flow gradient")) ||
      (r = falloc(h, (void**)&Fh.d_tab_u, sizeof(double) * k * Fh.stride * D, "flow proposal table")) ||
      (r = falloc(h, (void**)&Fh.d_tab_lq, sizeof(double) * k * Fh.stride, "flow proposal table")) ||
      (r = falloc(h, (void**)&Fh.d_train, sizeof(int32_t), "flow flag")))
    return r;
  if ((err = fill_on(h, Fh.d_img, 0, L * kImgLayer)) != cudaSuccess ||
      (err = fill_on(h, Fh.d_bias, 0, sizeof(float) * L * kBiasLayer)) != cudaSuccess)
    return cuda_fail(h, err, "flow image clear");
  FlowDev F = host_flowdev(E);
  if ((err = copy_on(h, Fh.d_flow, &F, sizeof(F), cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(h, err, "flow upload");
  if ((err = launch_flow_init(Fh.d_flow, Fh.d_master, Fh.d_m, Fh.d_v, (int)NP, c.seed, (uint64_t)e, h->stream)) ||
      (err = launch_flow_pack(Fh.d_flow, Fh.d_img, Fh.d_bias, Fh.d_master, (int)NP, h->stream)) ||
      (err = cudaStreamSynchronize(h->stream)))
    return cuda_fail(h, err, "flow initialisation");
  return NS_OK;
}

void flow_free(EventHost& E) {
  FlowHost& Fh = E.flow;
  void* ptrs[] = {Fh.d_flow, Fh.d_img, Fh.d_bias, Fh.d_master, Fh.d_m, Fh.d_v, Fh.d_partial, Fh.d_loss_part,
                  Fh.d_zsave, Fh.d_grad, Fh.d_tab_u, Fh.d_tab_lq, Fh.d_train};
  for (void* p : ptrs) cudaFree(p);
  Fh = FlowHost();
}

void flow_task_fields(const EventHost& E, WalkTask& T) {
  const FlowHost& Fh = E.flow;
  if (!Fh.enabled) return;
  T.flow = Fh.d_flow;
  T.fu = Fh.d_tab_u;
  T.flq = Fh.d_tab_lq;
  T.p_flow = Fh.p_flow;
  T.f_stride = Fh.stride;
}

// ---------------------------------------------------------------- batch stages
int flow_enqueue_train(ns_handle* h, int e, cudaStream_t s, int64_t* launches) {
  EventHost& E = h->events[e];
  FlowHost& Fh = E.flow;
  if (!Fh.enabled) return NS_OK;
  const NsState& S = E.ns;
  const int n_surv = S.n_live - S.k;   // the survivors sample the prior above the new L*
  flow_train_flag_kernel<<<1, 32, 0, s>>>(h->d_ns + e, Fh.every, Fh.d_train);
  cudaError_t err = cudaGetLastError();
  if (!err) err = launch_flow_standardise(Fh.d_flow, S.surv_u, n_surv, Fh.d_train, s);
  *launches += 2;
  for (int ep = 0; ep < Fh.epochs && !err; ++ep) {
    err = launch_flow_grad(Fh.d_flow, S.surv_u, n_surv, Fh.d_train, 1, Fh.d_partial, Fh.d_loss_part, Fh.d_zsave,
                           h->d_status + 1, s);
    if (!err)
      err = launch_flow_adam(Fh.d_flow, Fh.d_img, Fh.d_bias, Fh.d_master, Fh.d_m, Fh.d_v, Fh.d_partial, n_surv,
                             Fh.d_train, nullptr, Fh.n_params, s);
    *launches += 2;
  }
  return err == cudaSuccess ? NS_OK : cuda_fail(h, err, "flow training launch");
}

int flow_enqueue_table(ns_handle* h, int e, cudaStream_t s, int64_t* launches) {
  EventHost& E = h->events[e];
  FlowHost& Fh = E.flow;
  if (!Fh.enabled || !(Fh.p_flow > 0.0)) return NS_OK;
  cudaError_t err = launch_flow_table(Fh.d_flow, h->d_tasks + e, 0, 0, 0, 0, 0, 0, Fh.stride, Fh.d_tab_u, Fh.d_tab_lq,
                                      h->d_status + 1, sm_count(h), s);
  *launches += 1;
  return err == cudaSuccess ? NS_OK : cuda_fail(h, err, "flow table launch");
}

// Flow fields of a stand-alone walk (ns_walk_batch): the proposal table of its n walkers
// and n_steps steps goes to `table` (grown on demand) or, when `table` is null, to the
// handle's own batch table if it is large enough.
int flow_attach(ns_handle* h, int event, WalkTask& T, int n, int n_steps, Scratch* table, cudaStream_t s) {
  EventHost& E = h->events[event];
  FlowHost& Fh = E.flow;
  if (!Fh.enabled || !(Fh.p_flow > 0.0) || n == 0 || n_steps == 0) return NS_OK;
  const size_t D = E.n_dim;
  double *tu, *tl;
  int stride;
  if (table) {
    int r = ensure_scratch(h, *table, sizeof(double) * (size_t)n * n_steps * (D + 1));
    if (r) return r;
    tu = (double*)table->ptr;
    tl = tu + (size_t)n * n_steps * D;
    stride = n_steps;
  } else {
    if (n > E.ns.k || n_steps > Fh.stride)
      return set_error(h, NS_EINVAL, "flow walk without allocation needs n <= %d and n_steps <= %d", E.ns.k, Fh.stride);
    tu = Fh.d_tab_u;
    tl = Fh.d_tab_lq;
    stride = Fh.stride;
  }
  cudaError_t err = launch_flow_table(Fh.d_flow, nullptr, n, n_steps, T.walker_offset, T.iteration, T.key0, T.key1,
                                      stride, tu, tl, h->d_status + 1, sm_count(h), s);
  if (err != cudaSuccess) return cuda_fail(h, err, "flow table launch");
  T.flow = Fh.d_flow;
  T.fu = tu;
  T.flq = tl;
  T.p_flow = Fh.p_flow;
  T.f_stride = stride;
  return NS_OK;
}

// ---------------------------------------------------------------- checkpoint
bool flow_state_write(ns_handle* h, int e, FILE* f) {
  const FlowHost& Fh = h->events[e].flow;
  if (!Fh.enabled) return true;
  FlowDev F;
  std::vector<float> buf((size_t)Fh.n_params * 3);
  if (copy_on(h, &F, Fh.d_flow, sizeof(F), cudaMemcpyDeviceToHost) != cudaSuccess ||
      copy_on(h, buf.data(), Fh.d_master, sizeof(float) * Fh.n_params, cudaMemcpyDeviceToHost) != cudaSuccess ||
      copy_on(h, buf.data() + Fh.n_params, Fh.d_m, sizeof(float) * Fh.n_params, cudaMemcpyDeviceToHost) != cudaSuccess ||
      copy_on(h, buf.data() + 2 * (size_t)Fh.n_params, Fh.d_v, sizeof(float) * Fh.n_params, cudaMemcpyDeviceToHost) !=
          cudaSuccess)
    return false;
  return fwrite(&F, sizeof(F), 1, f) == 1 && fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
}

bool flow_state_parse(ns_handle* h, int e, FILE* f, FlowBlob& b) {
  const EventHost& E = h->events[e];
  const FlowHost& Fh = E.flow;
  b.present = Fh.enabled;
  if (!Fh.enabled) return true;
  b.buf.assign((size_t)Fh.n_params * 3, 0.0f);
  if (fread(&b.F, sizeof(b.F), 1, f) != 1 || fread(b.buf.data(), sizeof(float), b.buf.size(), f) != b.buf.size())
    return false;
  return b.F.n_params == Fh.n_params && b.F.n_layers == Fh.n_layers && b.F.n_dim == E.n_dim;
}

bool flow_state_apply(ns_handle* h, int e, const FlowBlob& b) {
  if (!b.present) return true;
  EventHost& E = h->events[e];
  FlowHost& Fh = E.flow;
  FlowDev cur = host_flowdev(E);
  std::memcpy(cur.mu, b.F.mu, sizeof(b.F.mu));
  std::memcpy(cur.sigma, b.F.sigma, sizeof(b.F.sigma));
  cur.log_sigma_sum = b.F.log_sigma_sum;
  cur.adam_t = b.F.adam_t;
  const float* buf = b.buf.data();
  return copy_on(h, Fh.d_flow, &cur, sizeof(cur), cudaMemcpyHostToDevice) == cudaSuccess &&
         copy_on(h, Fh.d_master, buf, sizeof(float) * Fh.n_params, cudaMemcpyHostToDevice) == cudaSuccess &&
         copy_on(h, Fh.d_m, buf + Fh.n_params, sizeof(float) * Fh.n_params, cudaMemcpyHostToDevice) == cudaSuccess &&
         copy_on(h, Fh.d_v, buf + 2 * (size_t)Fh.n_params, sizeof(float) * Fh.n_params, cudaMemcpyHostToDevice) ==
             cudaSuccess &&
         launch_flow_pack(Fh.d_flow, Fh.d_img, Fh.d_bias, Fh.d_master, Fh.n_params, h->stream) == cudaSuccess &&
         cudaStreamSynchronize(h->stream) == cudaSuccess;
}

// ---------------------------------------------------------------- C ABI
extern "C" int ns_flow_num_params(ns_handle* h, int event, int32_t* n_params) {
  int r = check_flow_event(h, event);
  if (r) return r;
  if (!n_params) return set_error(h, NS_EINVAL, "null argument");
  *n_params = h->events[event].flow.n_params;
  return NS_OK;
}

extern "C" int ns_flow_set(ns_handle* h, int event, const float* params, const double* mu, const double* sigma) {
  int r = check_flow_event(h, event);
  if (r) return r;
  if (!params || !mu || !sigma) return set_error(h, NS_EINVAL, "null argument");
  EventHost& E = h->events[event];
  FlowHost& Fh = E.flow;
  for (int i = 0; i < Fh.n_params; ++i)
    if (!std::isfinite(params[i])) return set_error(h, NS_ENONFINITE, "flow parameter %d not finite", i);
  FlowDev F = host_flowdev(E);
  float lss = 0.0f;
  for (int d = 0; d < E.n_dim; ++d) {
    if (!std::isfinite(mu[d]) || !(sigma[d] > 0.0) || !std::isfinite(sigma[d]))
      return set_error(h, NS_EINVAL, "mu must be finite and sigma positive");
    F.mu[d] = (float)mu[d];
    F.sigma[d] = (float)sigma[d];
    lss += logf(F.sigma[d]);
  }
  F.log_sigma_sum = lss;
  cudaError_t e;
  if ((e = cudaStreamSynchronize(h->stream)) ||
      (e = copy_on(h, Fh.d_flow, &F, sizeof(F), cudaMemcpyHostToDevice)) ||
      (e = copy_on(h, Fh.d_master, params, sizeof(float) * Fh.n_params, cudaMemcpyHostToDevice)) ||
      (e = fill_on(h, Fh.d_m, 0, sizeof(float) * Fh.n_params)) ||
      (e = fill_on(h, Fh.d_v, 0, sizeof(float) * Fh.n_params)) ||
      (e = launch_flow_pack(Fh.d_flow, Fh.d_img, Fh.d_bias, Fh.d_master, Fh.n_params, h->stream)) ||
      (e = cudaStreamSynchronize(h->stream)))
    return cuda_fail(h, e, "flow set");
  return NS_OK;
}

extern "C" int ns_flow_get(ns_handle* h, int event, float* params, double* mu, double* sigma) {
  int r = check_flow_event(h, event);
  if (r) return r;
  EventHost& E = h->events[event];
  FlowHost& Fh = E.flow;
  FlowDev F;
  cudaError_t e;
  if ((e = cudaStreamSynchronize(h->stream)) || (e = copy_on(h, &F, Fh.d_flow, sizeof(F), cudaMemcpyDeviceToHost)))
    return cuda_fail(h, e, "flow get");
  if (params && (e = copy_on(h, params, Fh.d_master, sizeof(float) * Fh.n_params, cudaMemcpyDeviceToHost)))
    return cuda_fail(h, e, "flow get");
  for (int d = 0; d < E.n_dim; ++d) {
    if (mu) mu[d] = F.mu[d];
    if (sigma) sigma[d] = F.sigma[d];
  }
  return NS_OK;
}

extern "C" int ns_flow_logq(ns_handle* h, int event, const double* u, int n, double* logq, int ptr_kind,
                            void* stream) {
  int r = check_flow_event(h, event);
  if (r) return r;
  if (n < 0 || (n > 0 && (!u || !logq))) return set_error(h, NS_EINVAL, "bad arrays");
  if (ptr_kind != NS_PTR_HOST && ptr_kind != NS_PTR_DEVICE) return set_error(h, NS_EINVAL, "bad ptr_kind");
  if (n == 0) return NS_OK;
  EventHost& E = h->events[event];
  const size_t D = E.n_dim;
  cudaStream_t s = stream ? (cudaStream_t)stream : h->stream;
  cudaError_t e;
  if ((e = cudaMemsetAsync(h->d_status + 1, 0, sizeof(int32_t), s))) return cuda_fail(h, e, "status reset");
  if (ptr_kind == NS_PTR_DEVICE) {
    e = launch_flow_logq(E.flow.d_flow, u, n, logq, h->d_status + 1, sm_count(h), s);
    return e == cudaSuccess ? NS_OK : cuda_fail(h, e, "flow logq launch");
  }
  for (size_t i = 0; i < (size_t)n * D; ++i)
    if (!(u[i] > 0.0 && u[i] < 1.0)) return set_error(h, NS_EINVAL, "u must lie strictly inside the unit cube");
  if ((r = ensure_scratch(h, h->scratch_in, sizeof(double) * (size_t)n * D))) return r;
  if ((r = ensure_scratch(h, h->scratch_out, sizeof(double) * (size_t)n))) return r;
  double* du = (double*)h->scratch_in.ptr;
  double* dl = (double*)h->scratch_out.ptr;
  if ((e = cudaMemcpyAsync(du, u, sizeof(double) * n * D, cudaMemcpyHostToDevice, s)) ||
      (e = launch_flow_logq(E.flow.d_flow, du, n, dl, h->d_status + 1, sm_count(h), s)) ||
      (e = cudaMemcpyAsync(logq, dl, sizeof(double) * n, cudaMemcpyDeviceToHost, s)))
    return cuda_fail(h, e, "flow logq");
  return check_err_flag(h, s, "flow logq");
}

extern "C" int ns_flow_sample(ns_handle* h, int event, int64_t iteration, int64_t walker_offset, int n, int n_steps,
                              double* u_out, double* logq_out, int ptr_kind, void* stream) {
  int r = check_flow_event(h, event);
  if (r) return r;
  if (n < 0 || n_steps < 0 || iteration < 0 || walker_offset < 0 || (n > 0 && n_steps > 0 && (!u_out || !logq_out)))
    return set_error(h, NS_EINVAL, "bad arguments");
  if (ptr_kind != NS_PTR_HOST && ptr_kind != NS_PTR_DEVICE) return set_error(h, NS_EINVAL, "bad ptr_kind");
  if (n == 0 || n_steps == 0) return NS_OK;
  EventHost& E = h->events[event];
  const size_t D = E.n_dim, rows = (size_t)n * n_steps;
  cudaStream_t s = stream ? (cudaStream_t)stream : h->stream;
  cudaError_t e;
  if ((e = cudaMemsetAsync(h->d_status + 1, 0, sizeof(int32_t), s))) return cuda_fail(h, e, "status reset");
  double *du = u_out, *dl = logq_out;
  if (ptr_kind == NS_PTR_HOST) {
    if ((r = ensure_scratch(h, h->scratch_out, sizeof(double) * rows * (D + 1)))) return r;
    du = (double*)h->scratch_out.ptr;
    dl = du + rows * D;
  }
  if ((e = launch_flow_table(E.flow.d_flow, nullptr, n, n_steps, walker_offset, iteration, E.cfg.seed,
                             (uint64_t)event, n_steps, du, dl, h->d_status + 1, sm_count(h), s)))
    return cuda_fail(h, e, "flow table launch");
  if (ptr_kind == NS_PTR_DEVICE) return NS_OK;
  if ((e = cudaMemcpyAsync(u_out, du, sizeof(double) * rows * D, cudaMemcpyDeviceToHost, s)) ||
      (e = cudaMemcpyAsync(logq_out, dl, sizeof(double) * rows, cudaMemcpyDeviceToHost, s)))
    return cuda_fail(h, e, "flow sample");
  return check_err_flag(h, s, "flow sample");
}

static int flow_points_upload(ns_handle* h, const EventHost& E, const double* u, int n, double** du, cudaStream_t s) {
  const size_t D = E.n_dim;
  if (n < 1 || n > kMaxLive) return set_error(h, NS_EINVAL, "need 1 <= n <= %d points", kMaxLive);
  for (size_t i = 0; i < (size_t)n * D; ++i)
    if (!(u[i] > 0.0 && u[i] < 1.0)) return set_error(h, NS_EINVAL, "u must lie strictly inside the unit cube");
  int r = ensure_scratch(h, h->scratch_in, sizeof(double) * (size_t)n * D);
  if (r) return r;
  *du = (double*)h->scratch_in.ptr;
  cudaError_t e = cudaMemcpyAsync(*du, u, sizeof(double) * n * D, cudaMemcpyHostToDevice, s);
  return e == cudaSuccess ? NS_OK : cuda_fail(h, e, "H2D points");
}

static int loss_sum(ns_handle* h, const FlowHost& Fh, int n, cudaStream_t s, double* loss) {
  std::vector<double> lp((n + kGradRows - 1) / kGradRows);
  cudaError_t e = cudaMemcpyAsync(lp.data(), Fh.d_loss_part, sizeof(double) * lp.size(), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(h, e, "flow loss");
  double acc = 0.0;
  for (double v : lp) acc += v;
  *loss = acc / n;
  return NS_OK;
}

extern "C" int ns_flow_grad(ns_handle* h, int event, const double* u, int n, float* grad, double* loss) {
  int r = check_flow_event(h, event);
  if (r) return r;
  if (!u || !grad) return set_error(h, NS_EINVAL, "null argument");
  EventHost& E = h->events[event];
  FlowHost& Fh = E.flow;
  cudaStream_t s = h->stream;
  double* du;
  if ((r = flow_points_upload(h, E, u, n, &du, s))) return r;
  cudaError_t e;
  if ((e = cudaMemsetAsync(h->d_status + 1, 0, sizeof(int32_t), s)) ||
      (e = launch_flow_grad(Fh.d_flow, du, n, nullptr, 0, Fh.d_partial, Fh.d_loss_part, Fh.d_zsave, h->d_status + 1, s)) ||
      (e = launch_flow_adam(Fh.d_flow, Fh.d_img, Fh.d_bias, Fh.d_master, Fh.d_m, Fh.d_v, Fh.d_partial, n, nullptr,
                            Fh.d_grad, Fh.n_params, s)) ||
      (e = cudaMemcpyAsync(grad, Fh.d_grad, sizeof(float) * Fh.n_params, cudaMemcpyDeviceToHost, s)))
    return cuda_fail(h, e, "flow gradient");
  if ((r = check_err_flag(h, s, "flow gradient"))) return r;
  if (loss) return loss_sum(h, Fh, n, s, loss);
  return NS_OK;
}

extern "C" int ns_flow_train(ns_handle* h, int event, const double* u, int n, int epochs, double* losses) {
  int r = check_flow_event(h, event);
  if (r) return r;
  if (!u || epochs < 0) return set_error(h, NS_EINVAL, "bad arguments");
  EventHost& E = h->events[event];
  FlowHost& Fh = E.flow;
  cudaStream_t s = h->stream;
  double* du;
  if ((r = flow_points_upload(h, E, u, n, &du, s))) return r;
  cudaError_t e;
  if ((e = cudaMemsetAsync(h->d_status + 1, 0, sizeof(int32_t), s)) ||
      (e = launch_flow_standardise(Fh.d_flow, du, n, nullptr, s)))
    return cuda_fail(h, e, "flow standardise");
  for (int ep = 0; ep < epochs; ++ep) {
    if ((e = launch_flow_grad(Fh.d_flow, du, n, nullptr, 1, Fh.d_partial, Fh.d_loss_part, Fh.d_zsave,
                              h->d_status + 1, s)) ||
        (e = launch_flow_adam(Fh.d_flow, Fh.d_img, Fh.d_bias, Fh.d_master, Fh.d_m, Fh.d_v, Fh.d_partial, n, nullptr,
                              nullptr, Fh.n_params, s)))
      return cuda_fail(h, e, "flow training launch");
    if (losses && (r = loss_sum(h, Fh, n, s, &losses[ep]))) return r;
  }
  return check_err_flag(h, s, "flow training");
}
