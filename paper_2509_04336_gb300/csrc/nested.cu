// nested.cu -- batched nested sampling on the device (Sec. 2.2.1, Sec. 2.2.3, Sec. 3.1,
// Sec. 3.2, Sec. 3.2.1) and the sampler entry points ns_step, ns_evidence, ns_posterior,
// ns_state_save and ns_state_load.
//
// One batch is three kernels that read and write the device-resident NsState:
//   select  (one CTA per event): sort the live points by (ln L, index) in shared memory;
//           the k lowest die and ln L* is the largest of them; their expected shrinkage
//           ln X_j = ln X_0 - sum_{i<=j} 1/(n - i) comes from a parallel prefix sum, their
//           weights L_j (X_{j-1} - X_j) enter Z through a block log-sum-exp; the survivors
//           are gathered in sorted order and each walker draws its start uniformly from
//           them (Philox block (0, j, it, 2), word 0);
//   walk    (one CTA per walker, all events in one grid): kernels.cu;
//   insert  (one CTA per event): the end points replace the dead slots, the walk length is
//           retuned from the batch mean accepted count, and the termination test runs.
// ns_step replays a CUDA graph of G batches and reads the small NsState back once per replay.
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <vector>

#include "api_internal.h"

using namespace gwns;

namespace {

constexpr int kSelThreads = 1024;

__device__ __forceinline__ bool key_less(const double* lnl, int a, int b) {
  // (ln L, index) lexicographic; index 0xFFFF pads the sort and compares greatest
  if (a == 0xFFFF) return false;
  if (b == 0xFFFF) return true;
  double la = lnl[a], lb = lnl[b];
  return la < lb || (la == lb && a < b);
}

// Block-wide inclusive scan of one double per thread (kSelThreads threads).
__device__ inline double block_scan(double v, double* warp_buf) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    double o = __shfl_up_sync(0xffffffffu, v, off);
    if (lane >= off) v += o;
  }
  if (lane == 31) warp_buf[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double w = (lane < kSelThreads / 32) ? warp_buf[lane] : 0.0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      double o = __shfl_up_sync(0xffffffffu, w, off);
      if (lane >= off) w += o;
    }
    warp_buf[lane] = w;
  }
  __syncthreads();
  double r = v + (warp > 0 ? warp_buf[warp - 1] : 0.0);
  __syncthreads();
  return r;
}

__device__ inline double block_max(double v, double* buf) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, off));
  if (lane == 0) buf[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = buf[0];
    for (int w = 1; w < kSelThreads / 32; ++w) m = fmax(m, buf[w]);
    buf[32] = m;
  }
  __syncthreads();
  double r = buf[32];
  __syncthreads();
  return r;
}

__device__ inline double block_sum(double v, double* buf) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if (lane == 0) buf[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < kSelThreads / 32; ++w) m += buf[w];
    buf[32] = m;
  }
  __syncthreads();
  double r = buf[32];
  __syncthreads();
  return r;
}

__device__ inline double logaddexp(double a, double b) {
  if (a == -INFINITY) return b;
  if (b == -INFINITY) return a;
  double m = fmax(a, b);
  return m + log1p(exp(-fabs(a - b)));
}

__global__ void __launch_bounds__(kSelThreads) select_kernel(NsState* states, WalkTask* tasks) {
  __shared__ double lnl[kMaxLive];
  __shared__ uint16_t idx[kMaxLive];
  __shared__ double buf[64];
  NsState& S = states[blockIdx.x];
  if (S.done) return;
  const int n = S.n_live, k = S.k, D = S.D, tid = threadIdx.x;
  if (S.n_dead + k > S.dead_cap) {      // the host keeps capacity ahead; never overrun
    if (tid == 0) { S.overflow = 1; S.done = 1; tasks[blockIdx.x].done = 1; }
    return;
  }
  int n2 = 1;
  while (n2 < n) n2 <<= 1;
  for (int i = tid; i < n2; i += kSelThreads) {
    if (i < n) { lnl[i] = S.live_lnl[i]; idx[i] = (uint16_t)i; }
    else idx[i] = 0xFFFF;
  }
  // bitonic sort of the index array by (ln L, index)
  for (int size = 2; size <= n2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      __syncthreads();
      for (int t = tid; t < n2 / 2; t += kSelThreads) {
        int i = 2 * t - (t & (stride - 1));
        int j = i + stride;
        bool up = (i & size) == 0;
        int a = idx[i], b = idx[j];
        if (key_less(lnl, b, a) == up) { idx[i] = (uint16_t)b; idx[j] = (uint16_t)a; }
      }
    }
  }
  __syncthreads();
  const double log_x0 = S.log_x;
  const int64_t n_dead = S.n_dead;
  // expected shrinkage and weights of the k dead points, in chunks of kSelThreads
  double carry = 0.0, m_all = -INFINITY;
  double logw_local[(kMaxLive + kSelThreads - 1) / kSelThreads];
  int c = 0;
  for (int base = 0; base < k; base += kSelThreads, ++c) {
    int j = base + tid;
    double inv = (j < k) ? 1.0 / (double)(n - j) : 0.0;
    double pre = block_scan(inv, buf) + carry;
    if (threadIdx.x == kSelThreads - 1) buf[40] = pre;
    __syncthreads();
    carry = buf[40];
    __syncthreads();
    double lw = -INFINITY;
    if (j < k) {
      int id = idx[j];
      double lx = log_x0 - pre;
      lw = lnl[id] + lx + log(expm1(inv));
      size_t row = (size_t)(n_dead + j);
      S.dead_lnl[row] = lnl[id];
      S.dead_logw[row] = lw;
      S.dead_nlive[row] = n - j;
      for (int d = 0; d < D; ++d) S.dead_u[row * D + d] = S.live_u[(size_t)id * D + d];
    }
    logw_local[c] = lw;
    m_all = fmax(m_all, lw);
  }
  const double m = block_max(m_all, buf);
  double acc = 0.0;
  c = 0;
  for (int base = 0; base < k; base += kSelThreads, ++c)
    if (base + tid < k) acc += exp(logw_local[c] - m);
  const double ssum = block_sum(acc, buf);
  // survivors in sorted order and the walkers' starts
  const int ns = n - k;
  for (int i = tid; i < ns; i += kSelThreads) {
    int id = idx[k + i];
    for (int d = 0; d < D; ++d) {
      double v = S.live_u[(size_t)id * D + d];
      S.surv_u[(size_t)i * D + d] = v;
      const float vh = __double2float_rn(v);
      S.survf[(size_t)i * D + d] = make_float2(vh, __double2float_rn(v - (double)vh));
    }
  }
  const uint64_t it = (uint64_t)S.iteration;
  for (int j = tid; j < k; j += kSelThreads) {
    Philox4 r = philox4x64(0ull, (uint64_t)j, it, 2ull, S.key0, S.key1);
    int sidx = (int)rand_index(r.v[0], (uint64_t)ns);
    int id = idx[k + sidx];
    for (int d = 0; d < D; ++d) S.w_u0[(size_t)j * D + d] = S.live_u[(size_t)id * D + d];
    S.w_lnl0[j] = lnl[id];
    S.slot[j] = idx[j];
  }
  __syncthreads();
  if (tid == 0) {
    S.lnl_star = lnl[idx[k - 1]];
    S.log_x = log_x0 - carry;
    double batch = (m == -INFINITY) ? -INFINITY : m + log(ssum);
    S.log_z = logaddexp(S.log_z, batch);
    S.n_dead = n_dead + k;
    WalkTask& T = tasks[blockIdx.x];
    T.lnl_star = S.lnl_star;
    T.iteration = S.iteration;
    T.n_steps = S.n_steps;
    T.done = 0;
  }
}

__global__ void __launch_bounds__(kSelThreads) insert_kernel(NsState* states, WalkTask* tasks) {
  __shared__ double buf[64];
  NsState& S = states[blockIdx.x];
  if (S.done) return;
  const int k = S.k, D = S.D, n = S.n_live, tid = threadIdx.x;
  double acc = 0.0, calls = 0.0, zero = 0.0, bins = 0.0, spec = 0.0, accf = 0.0;
  for (int j = tid; j < k; j += kSelThreads) {
    int s = S.slot[j];
    bins += (double)S.w_nb[j];
    spec += (double)S.w_ns[j];
    for (int d = 0; d < D; ++d) S.live_u[(size_t)s * D + d] = S.w_uo[(size_t)j * D + d];
    S.live_lnl[s] = S.w_lo[j];
    acc += (double)S.w_na[j];
    accf += (double)S.w_naf[j];
    calls += (double)S.w_nl[j];
    zero += (S.w_na[j] == 0) ? 1.0 : 0.0;
  }
  const double tot_acc = block_sum(acc, buf);
  const double tot_calls = block_sum(calls, buf);
  const double n_zero = block_sum(zero, buf);
  const double tot_bins = block_sum(bins, buf);
  const double tot_spec = block_sum(spec, buf);
  const double tot_accf = block_sum(accf, buf);
  __syncthreads();
  double mx = -INFINITY;
  for (int i = tid; i < n; i += kSelThreads) mx = fmax(mx, S.live_lnl[i]);
  const double lmax = block_max(mx, buf);
  double se = 0.0;
  for (int i = tid; i < n; i += kSelThreads) se += exp(S.live_lnl[i] - lmax);
  const double sum_live = block_sum(se, buf);
  if (tid == 0) {
    double mean_acc = tot_acc / (double)k;
    S.mean_accept = mean_acc;
    S.mean_accept_flow = tot_accf / (double)k;
    S.n_like += (int64_t)tot_calls;
    S.n_bins_eval += (int64_t)tot_bins;
    S.n_spec_eval += (int64_t)tot_spec;
    // speculation depth of the next batch: about c / p in-bounds proposals per round, p the
    // acceptance per likelihood call of this batch; c = 1.4 puts the first acceptance on
    // average in the first two thirds of a round (c = 0.7: halfway), a trade of discarded
    // proposals for fewer rounds, whose fixed costs dominate short likelihoods
    if (S.spec_auto) {
      double p = mean_acc / fmax(tot_calls / (double)k, 1.0);
      S.spec_p = p;
      double m = p > 0.0 ? floor(S.spec_mult / p + 0.5) : (double)kSpecMax;
      S.spec_rule = (int32_t)fmin(fmax(m, 1.0), (double)kSpecMax);
      S.spec = min(S.spec_rule, S.spec_cap);
    }
    if (n_zero > 0.0) S.zero_accept = 1;
    // walk-length retune (batch-scaled delay) on the mean of accepted DE steps plus flow_w
    // times accepted flow steps; HRSS keeps its fixed move count
    if (S.hrss == 0) {
      double ns = (double)S.n_steps;
      const double eff = (tot_acc + (S.flow_w - 1.0) * tot_accf) / (double)k;
      double x = (S.delay_k * ns + ns * (double)S.naccept / fmax(eff, 0.5)) / (S.delay_k + 1.0);
      double r = floor(x + 0.5);
      r = fmin(fmax(r, 1.0), (double)S.maxmcmc);
      S.n_steps = (int32_t)r;
    }
    S.iteration += 1;
    S.lnl_max = lmax;
    S.dlogz = logaddexp(S.log_z, lmax + S.log_x) - S.log_z;
    bool stop;
    if (S.term_kind == 0) {
      stop = S.dlogz < S.term_value;
    } else {
      double log_live = lmax + log(sum_live / (double)n) + S.log_x;
      stop = (log_live - S.log_z) < log(S.term_value);
    }
    if (stop || S.iteration >= S.max_iter) S.done = 1;
    tasks[blockIdx.x].done = S.done;
    tasks[blockIdx.x].n_steps = S.n_steps;
    tasks[blockIdx.x].spec = S.spec;
  }
}

// HRSS: the lower Cholesky factor of the survivors' sample covariance (divisor n_s - 1, unit-cube
// coordinates), one CTA per event, after the deletion: the direction factor of the batch's
// slice-sampling lines.  A pivot at the rounding level of its variance (the survivors span fewer
// than D directions) stops the event with chol_bad set.
__global__ void __launch_bounds__(kSelThreads) chol_kernel(NsState* states, WalkTask* tasks) {
  __shared__ double mean[kMaxDim];
  __shared__ double cov[kMaxDim * kMaxDim];
  NsState& S = states[blockIdx.x];
  if (S.done || S.hrss == 0) return;
  const int D = S.D, ns = S.n_live - S.k, tid = threadIdx.x;
  for (int i = tid; i < D; i += kSelThreads) {
    double a = 0.0;
    for (int p = 0; p < ns; ++p) a += S.surv_u[(size_t)p * D + i];
    mean[i] = a / (double)ns;
  }
  __syncthreads();
  for (int q = tid; q < D * D; q += kSelThreads) {
    const int i = q / D, k = q % D;
    if (k > i) continue;
    double a = 0.0;
    for (int p = 0; p < ns; ++p)
      a += (S.surv_u[(size_t)p * D + i] - mean[i]) * (S.surv_u[(size_t)p * D + k] - mean[k]);
    cov[q] = a / (double)(ns - 1);
  }
  __syncthreads();
  if (tid == 0) {
    double* L = S.chol;
    bool ok = true;
    for (int i = 0; i < D && ok; ++i)
      for (int k = 0; k <= i; ++k) {
        double a = cov[i * D + k];
        for (int m = 0; m < k; ++m) a -= L[i * D + m] * L[k * D + m];
        if (i == k) {
          if (!(a > 1e-12 * cov[i * D + i]) || !(a > 0.0)) { ok = false; break; }
          L[i * D + i] = sqrt(a);
        } else {
          L[i * D + k] = a / L[k * D + k];
        }
      }
    for (int i = 0; i < D; ++i)
      for (int k = i + 1; k < D; ++k) L[i * D + k] = 0.0;
    if (!ok) {
      S.chol_bad = 1;
      S.done = 1;
      tasks[blockIdx.x].done = 1;
    }
  }
}

// Initial live points: u[i][d] from Philox block (i, d / 4, 0, 3), word d % 4.
__global__ void init_live_kernel(NsState* states, int e) {
  NsState& S = states[e];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S.n_live) return;
  for (int d = 0; d < S.D; ++d) {
    Philox4 r = philox4x64((uint64_t)i, (uint64_t)(d / 4), 0ull, 3ull, S.key0, S.key1);
    S.live_u[(size_t)i * S.D + d] = rand_open_unit(r.v[d % 4]);
  }
}

// ln Z replays: replay r draws every shrinkage factor t_i ~ Beta(n_i, 1) as
// ln t_i = ln U / n_i (Philox block (i, r, 0, 4), word 0) and accumulates
// ln Z_r = logsumexp_i (ln L_i + ln X_{i-1} + ln(1 - t_i)) plus the live points at X_end / n.
__global__ void __launch_bounds__(kSelThreads) replay_kernel(const NsState* states, int e, double* out) {
  __shared__ double buf[64];
  const NsState& S = states[e];
  const int r = blockIdx.x, tid = threadIdx.x;
  double carry = 0.0, m_run = -INFINITY, s_run = 0.0;   // running logsumexp (valid in thread 0)
  for (int64_t base = 0; base < S.n_dead; base += kSelThreads) {
    int64_t i = base + tid;
    double lt = 0.0;
    if (i < S.n_dead) {
      Philox4 p = philox4x64((uint64_t)i, (uint64_t)r, 0ull, 4ull, S.key0, S.key1);
      lt = log(rand_open_unit(p.v[0])) / (double)S.dead_nlive[i];
    }
    double pre = block_scan(lt, buf) + carry;         // ln X_i (inclusive)
    double lw = -INFINITY;
    if (i < S.n_dead) {
      double lx_prev = pre - lt;
      lw = S.dead_lnl[i] + lx_prev + log(-expm1(lt));
    }
    if (threadIdx.x == kSelThreads - 1) buf[40] = pre;
    __syncthreads();
    carry = buf[40];
    __syncthreads();
    double m = block_max(lw, buf);
    double s = block_sum(lw == -INFINITY ? 0.0 : exp(lw - m), buf);
    if (tid == 0 && m != -INFINITY) {
      if (m > m_run) { s_run = s_run * exp(m_run - m) + s; m_run = m; }
      else s_run += s * exp(m - m_run);
    }
  }
  // final live points
  double mx = -INFINITY;
  for (int i = tid; i < S.n_live; i += kSelThreads) mx = fmax(mx, S.live_lnl[i]);
  double lm = block_max(mx, buf);
  double se = 0.0;
  for (int i = tid; i < S.n_live; i += kSelThreads) se += exp(S.live_lnl[i] - lm);
  double sl = block_sum(se, buf);
  if (tid == 0) {
    double live = lm + log(sl / (double)S.n_live) + carry;
    double lz = (m_run == -INFINITY) ? -INFINITY : m_run + log(s_run);
    out[r] = logaddexp(lz, live);
  }
}

int alloc(ns_handle* h, void** p, size_t bytes, const char* what) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) return set_error(h, NS_ENOMEM, "allocating %s (%zu bytes): %s", what, bytes, cudaGetErrorString(e));
  return NS_OK;
}

double batch_delay(double delay, int k) {
  if (delay <= 0.0) return 0.0;
  double r = std::pow(delay / (delay + 1.0), (double)k);
  return r / (1.0 - r);
}

int upload_states(ns_handle* h) {
  std::vector<NsState> st;
  for (auto& E : h->events) st.push_back(E.ns);
  cudaError_t e = copy_on(h, h->d_ns, st.data(), sizeof(NsState) * st.size(), cudaMemcpyHostToDevice);
  return e == cudaSuccess ? NS_OK : cuda_fail(h, e, "state upload");
}

int download_states(ns_handle* h) {
  h->host_ns.resize(h->events.size());
  cudaError_t e = cudaMemcpyAsync(h->host_ns.data(), h->d_ns, sizeof(NsState) * h->events.size(),
                                  cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? NS_OK : cuda_fail(h, e, "state download");
}

// Grow the dead store of event e to hold at least `need` rows (copying the rows so far).
int grow_dead(ns_handle* h, int e, int64_t need, int64_t rows) {
  NsState& S = h->events[e].ns;
  if (need <= S.dead_cap) return NS_OK;
  int64_t cap = S.dead_cap > 0 ? S.dead_cap : S.k;
  while (cap < need) cap *= 2;
  double *du = nullptr, *dl = nullptr, *dw = nullptr;
  int32_t* dn = nullptr;
  int r;
  if ((r = alloc(h, (void**)&du, sizeof(double) * cap * S.D, "dead_u")) ||
      (r = alloc(h, (void**)&dl, sizeof(double) * cap, "dead_lnl")) ||
      (r = alloc(h, (void**)&dw, sizeof(double) * cap, "dead_logw")) ||
      (r = alloc(h, (void**)&dn, sizeof(int32_t) * cap, "dead_nlive"))) {
    cudaFree(du); cudaFree(dl); cudaFree(dw); cudaFree(dn);
    return r;
  }
  size_t nd = (size_t)rows;
  cudaError_t err = cudaSuccess;
  if (nd) {
    if ((err = copy_on(h, du, S.dead_u, sizeof(double) * nd * S.D, cudaMemcpyDeviceToDevice)) ||
        (err = copy_on(h, dl, S.dead_lnl, sizeof(double) * nd, cudaMemcpyDeviceToDevice)) ||
        (err = copy_on(h, dw, S.dead_logw, sizeof(double) * nd, cudaMemcpyDeviceToDevice)) ||
        (err = copy_on(h, dn, S.dead_nlive, sizeof(int32_t) * nd, cudaMemcpyDeviceToDevice)))
      return cuda_fail(h, err, "dead store copy");
  }
  cudaFree(S.dead_u); cudaFree(S.dead_lnl); cudaFree(S.dead_logw); cudaFree(S.dead_nlive);
  S.dead_u = du; S.dead_lnl = dl; S.dead_logw = dw; S.dead_nlive = dn;
  S.dead_cap = cap;
  // patch the pointer and capacity fields of the device state
  NsState* d = h->d_ns + e;
  if ((err = copy_on(h, &d->dead_cap, &S.dead_cap, sizeof(int64_t), cudaMemcpyHostToDevice)) ||
      (err = copy_on(h, &d->dead_u, &S.dead_u, sizeof(double*), cudaMemcpyHostToDevice)) ||
      (err = copy_on(h, &d->dead_lnl, &S.dead_lnl, sizeof(double*), cudaMemcpyHostToDevice)) ||
      (err = copy_on(h, &d->dead_logw, &S.dead_logw, sizeof(double*), cudaMemcpyHostToDevice)) ||
      (err = copy_on(h, &d->dead_nlive, &S.dead_nlive, sizeof(int32_t*), cudaMemcpyHostToDevice)))
    return cuda_fail(h, err, "dead store patch");
  return NS_OK;
}

// Room for `batches` more batches of every event.
int ensure_dead_capacity(ns_handle* h, int batches) {
  for (size_t e = 0; e < h->events.size(); ++e) {
    const NsState& cur = h->host_ns[e];
    int r = grow_dead(h, (int)e, cur.n_dead + (int64_t)batches * h->events[e].ns.k, cur.n_dead);
    if (r) return r;
  }
  return NS_OK;
}

int enqueue_batch(ns_handle* h, int b, int64_t* launches) {
  const int ne = (int)h->events.size();
  int r;
  select_kernel<<<ne, kSelThreads, 0, h->stream>>>(h->d_ns, h->d_tasks);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "select launch");
  for (int ev = 0; ev < ne; ++ev)
    if ((r = flow_enqueue_train(h, ev, h->stream, launches)) || (r = flow_enqueue_table(h, ev, h->stream, launches)))
      return r;
  *launches += 3;
  // inside stream capture a plain event record is only a dependency marker; the external
  // flag makes it an event-record node that timestamps every replay
  if ((e = cudaEventRecordWithFlags(h->walk_events[2 * b], h->stream, cudaEventRecordExternal)) != cudaSuccess)
    return cuda_fail(h, e, "event");
  if (h->hrss) {
    chol_kernel<<<ne, kSelThreads, 0, h->stream>>>(h->d_ns, h->d_tasks);
    *launches += 1;
    e = launch_hrss(h->precision, h->waveform, h->max_det, h->d_events, h->d_tasks, h->d_blk_task, h->d_blk_local,
                    h->n_walk_blocks, h->stream);
  } else {
    e = launch_walk(h->precision, h->waveform, h->max_det, h->d_events, h->d_tasks, h->d_blk_task, h->d_blk_local,
                    h->n_walk_blocks, h->stream, walk_extras(h));
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "walk launch");
  if ((e = cudaEventRecordWithFlags(h->walk_events[2 * b + 1], h->stream, cudaEventRecordExternal)) != cudaSuccess)
    return cuda_fail(h, e, "event");
  insert_kernel<<<ne, kSelThreads, 0, h->stream>>>(h->d_ns, h->d_tasks);
  e = cudaGetLastError();
  return e == cudaSuccess ? NS_OK : cuda_fail(h, e, "insert launch");
}

int build_graph(ns_handle* h, int batches) {
  if (h->graph_exec[batches]) return NS_OK;
  cudaGraph_t g;
  cudaError_t e;
  while ((int)h->walk_events.size() < 2 * 8) {
    cudaEvent_t ev;
    if ((e = cudaEventCreate(&ev)) != cudaSuccess) return cuda_fail(h, e, "event create");
    h->walk_events.push_back(ev);
  }
  e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(h, e, "begin capture");
  int64_t launches = 0;
  for (int b = 0; b < batches; ++b) {
    int r = enqueue_batch(h, b, &launches);
    if (r) { cudaStreamEndCapture(h->stream, &g); return r; }
  }
  h->launches_per_batch[batches] = launches;
  e = cudaStreamEndCapture(h->stream, &g);
  if (e != cudaSuccess) return cuda_fail(h, e, "end capture");
  e = cudaGraphInstantiate(&h->graph_exec[batches], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(h, e, "graph instantiate");
  return NS_OK;
}

}  // namespace

int nested_init(ns_handle* h) {
  const int ne = (int)h->events.size();
  int r;
  int total_walkers = 0;
  std::vector<WalkTask> tasks(ne);
  for (int e = 0; e < ne; ++e) {
    EventHost& E = h->events[e];
    const ns_config& c = E.cfg;
    NsState& S = E.ns;
    std::memset(&S, 0, sizeof(S));
    S.n_live = c.n_live;
    S.k = c.num_delete;
    S.D = E.n_dim;
    S.naccept = c.naccept;
    S.maxmcmc = c.maxmcmc;
    S.term_kind = c.term_kind;
    S.term_value = c.term_value;
    S.max_iter = c.max_iter > 0 ? c.max_iter : 1000000;
    S.n_steps = c.n_steps0 > 0 ? c.n_steps0 : (int32_t)std::ceil(c.naccept / 0.25);
    if (S.n_steps > S.maxmcmc) S.n_steps = S.maxmcmc;
    double delay = c.delay < 0.0 ? (double)(c.naccept - 1) : c.delay;
    S.delay_k = batch_delay(delay, S.k);
    S.log_x = 0.0;
    S.log_z = -INFINITY;
    S.lnl_star = -INFINITY;
    S.dlogz = INFINITY;
    S.key0 = c.seed;
    S.key1 = (uint64_t)e;
    S.dead_cap = (int64_t)S.k * 64;
    S.hrss = c.proposal == NS_PROPOSAL_HRSS ? (c.hrss_moves > 0 ? c.hrss_moves : 2 * E.n_dim) : 0;
    if (S.hrss) S.n_steps = S.hrss;
    S.spec_auto = c.spec_depth == 0 && S.hrss == 0;
    S.spec_cap = h->precision == 0 ? 8 : kSpecMax;
    S.spec_rule = 4;
    S.spec = c.spec_depth > 0 ? c.spec_depth : (S.hrss ? hrss_default_spec(c.waveform) : 4);
    S.spec_mult = 1.4;
    S.spec_p = 0.0;
    S.flow_w = c.flow_accept_weight > 0.0 ? c.flow_accept_weight : 1.0;
    const size_t n = S.n_live, k = S.k, D = S.D;
    if ((r = alloc(h, (void**)&S.live_u, sizeof(double) * n * D, "live_u")) ||
        (r = alloc(h, (void**)&S.live_lnl, sizeof(double) * n, "live_lnl")) ||
        (r = alloc(h, (void**)&S.surv_u, sizeof(double) * (n - k) * D, "surv_u")) ||
        (r = alloc(h, (void**)&S.survf, sizeof(float2) * (n - k) * D, "survf")) ||
        (r = alloc(h, (void**)&S.w_u0, sizeof(double) * k * D, "w_u0")) ||
        (r = alloc(h, (void**)&S.w_lnl0, sizeof(double) * k, "w_lnl0")) ||
        (r = alloc(h, (void**)&S.w_uo, sizeof(double) * k * D, "w_uo")) ||
        (r = alloc(h, (void**)&S.w_lo, sizeof(double) * k, "w_lo")) ||
        (r = alloc(h, (void**)&S.w_na, sizeof(int32_t) * k, "w_na")) ||
        (r = alloc(h, (void**)&S.w_nl, sizeof(int32_t) * k, "w_nl")) ||
        (r = alloc(h, (void**)&S.slot, sizeof(int32_t) * k, "slot")) ||
        (r = alloc(h, (void**)&S.w_nb, sizeof(int64_t) * k, "w_nb")) ||
        (r = alloc(h, (void**)&S.w_ns, sizeof(int64_t) * k, "w_ns")) ||
        (r = alloc(h, (void**)&S.w_naf, sizeof(int32_t) * k, "w_naf")) ||
        (r = alloc(h, (void**)&S.dead_u, sizeof(double) * S.dead_cap * D, "dead_u")) ||
        (r = alloc(h, (void**)&S.dead_lnl, sizeof(double) * S.dead_cap, "dead_lnl")) ||
        (r = alloc(h, (void**)&S.dead_logw, sizeof(double) * S.dead_cap, "dead_logw")) ||
        (r = alloc(h, (void**)&S.dead_nlive, sizeof(int32_t) * S.dead_cap, "dead_nlive")) ||
        (S.hrss && (r = alloc(h, (void**)&S.chol, sizeof(double) * D * D, "chol"))))
      return r;
    // walks of the batch-phase calls fill only their own walker range
    if (cudaError_t err = fill_on(h, S.w_naf, 0, sizeof(int32_t) * k)) return cuda_fail(h, err, "w_naf clear");
    WalkTask& T = tasks[e];
    std::memset(&T, 0, sizeof(T));
    T.surv = S.surv_u; T.survf = S.survf; T.u0 = S.w_u0; T.lnl0 = S.w_lnl0; T.u_out = S.w_uo; T.lnl_out = S.w_lo;
    T.n_acc = S.w_na; T.n_like = S.w_nl; T.n_bins = S.w_nb; T.n_spec = S.w_ns; T.spec = S.spec;
    T.n_acc_flow = S.w_naf;
    T.lnl_star = -INFINITY; T.iteration = 0; T.walker_offset = 0;
    T.key0 = S.key0; T.key1 = S.key1; T.n_s = S.n_live - S.k; T.n = S.k; T.n_steps = S.n_steps;
    T.done = 0; T.event = e;
    T.chol = S.chol;
    watchdog_fields(h, T);
    flow_task_fields(E, T);
    total_walkers += S.k;
  }
  if ((r = alloc(h, (void**)&h->d_ns, sizeof(NsState) * ne, "states")) ||
      (r = alloc(h, (void**)&h->d_tasks, sizeof(WalkTask) * ne, "tasks")) ||
      (r = alloc(h, (void**)&h->d_blk_task, sizeof(int32_t) * total_walkers, "block map")) ||
      (r = alloc(h, (void**)&h->d_blk_local, sizeof(int32_t) * total_walkers, "block map")))
    return r;
  std::vector<int32_t> bt, bl;
  for (int e = 0; e < ne; ++e)
    for (int j = 0; j < h->events[e].ns.k; ++j) { bt.push_back(e); bl.push_back(j); }
  h->n_walk_blocks = total_walkers;
  cudaError_t err;
  if ((err = copy_on(h, h->d_tasks, tasks.data(), sizeof(WalkTask) * ne, cudaMemcpyHostToDevice)) ||
      (err = copy_on(h, h->d_blk_task, bt.data(), sizeof(int32_t) * bt.size(), cudaMemcpyHostToDevice)) ||
      (err = copy_on(h, h->d_blk_local, bl.data(), sizeof(int32_t) * bl.size(), cudaMemcpyHostToDevice)))
    return cuda_fail(h, err, "task upload");
  if ((r = upload_states(h))) return r;
  // initial live points and their likelihoods (Sec. 2.2.1)
  for (int e = 0; e < ne; ++e) {
    NsState& S = h->events[e].ns;
    init_live_kernel<<<(S.n_live + 127) / 128, 128, 0, h->stream>>>(h->d_ns, e);
    if ((err = launch_unit_likelihood(h->precision, h->waveform, h->events[e].n_det, h->d_events + e, S.live_u, S.n_live,
                                      S.live_lnl, h->stream)) != cudaSuccess)
      return cuda_fail(h, err, "initial likelihoods");
    int64_t nl = S.n_live;
    cudaMemcpyAsync(&h->d_ns[e].n_like, &nl, sizeof(int64_t), cudaMemcpyHostToDevice, h->stream);
  }
  if ((err = cudaStreamSynchronize(h->stream)) != cudaSuccess) return cuda_fail(h, err, "initial live points");
  return download_states(h);
}

void nested_free(ns_handle* h) {
  for (auto& g : h->graph_exec) if (g) { cudaGraphExecDestroy(g); g = nullptr; }
  for (cudaEvent_t ev : h->walk_events) cudaEventDestroy(ev);
  h->walk_events.clear();
  for (auto& E : h->events) {
    NsState& S = E.ns;
    void* ptrs[] = {S.live_u, S.live_lnl, S.surv_u, S.survf, S.w_u0, S.w_lnl0, S.w_uo, S.w_lo, S.w_na, S.w_nl,
                    S.slot, S.w_nb, S.w_ns, S.w_naf, S.dead_u, S.dead_lnl, S.dead_logw, S.dead_nlive, S.chol};
    for (void* p : ptrs) cudaFree(p);
    std::memset(&S, 0, sizeof(S));
  }
  cudaFree(h->d_ns);
  cudaFree(h->d_tasks);
  cudaFree(h->d_blk_task);
  cudaFree(h->d_blk_local);
  h->d_ns = nullptr;
  h->d_tasks = nullptr;
}

static void fill_progress(ns_handle* h, ns_progress* p) {
  for (size_t e = 0; e < h->events.size(); ++e) {
    const NsState& S = h->host_ns[e];
    p[e].iterations = S.iteration;
    p[e].n_like = S.n_like;
    p[e].log_z = S.log_z;
    p[e].dlogz = S.dlogz;
    p[e].log_x = S.log_x;
    p[e].lnl_star = S.lnl_star;
    p[e].mean_accept = S.mean_accept;
    p[e].n_steps = S.n_steps;
    p[e].done = S.done;
    p[e].n_bins = S.n_bins_eval;
    p[e].walk_ms = h->walk_ms;
    p[e].kernel_launches = h->kernel_launches;
    p[e].n_spec = S.n_spec_eval;
    p[e].spec_depth = S.spec;
    p[e].spec_cap = S.spec_cap;
    p[e].mean_accept_flow = S.mean_accept_flow;
  }
}

namespace {
// Candidate caps of the speculation depth tried by the autotuner (the rule m = c / p sets the
// depth below the cap): a small cap suits proposals with much work of their own, where each
// speculative one costs a full evaluation; short likelihoods, whose rounds are dominated by
// their fixed costs, take the largest.
const int kTuneCaps[] = {2, 4, 8, 16, 32};
const int kTuneCapsF64[] = {1, 2, 4, 8};

// Sets the speculation cap of every event, and the depth of the next walk to the rule value
// under that cap.
int set_spec_cap(ns_handle* h, int cap) {
  for (size_t e = 0; e < h->events.size(); ++e) {
    const NsState& S = h->host_ns[e];
    const int32_t spec = S.spec_rule < cap ? S.spec_rule : cap;
    NsState* d = h->d_ns + e;
    cudaError_t err;
    if ((err = copy_on(h, &d->spec_cap, &cap, sizeof(int32_t), cudaMemcpyHostToDevice)) ||
        (err = copy_on(h, &d->spec, &spec, sizeof(int32_t), cudaMemcpyHostToDevice)) ||
        (err = copy_on(h, &h->d_tasks[e].spec, &spec, sizeof(int32_t), cudaMemcpyHostToDevice)))
      return cuda_fail(h, err, "speculation cap");
  }
  return NS_OK;
}
}  // namespace

extern "C" int ns_step(ns_handle* h, int max_batches, ns_progress* progress) {
  if (!h) return set_error(nullptr, NS_EINVAL, "handle is NULL");
  if (max_batches < 0) return set_error(h, NS_EINVAL, "max_batches < 0");
  if (h->batch_open) return set_error(h, NS_ESTATE, "a batch is open (ns_batch_end)");
  cudaSetDevice(h->device);
  cudaGetLastError();   // a stale error of an earlier call must not be reported here
  int r;
  bool all_done = true;
  for (auto& S : h->host_ns) all_done = all_done && S.done;
  int left = all_done ? 0 : max_batches;
  const int G = 8;
  {
    cudaError_t e = cudaMemsetAsync(h->d_status + 2, 0, sizeof(int32_t), h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "watchdog reset");
  }
  bool all_auto = true;
  for (auto& E : h->events) all_auto = all_auto && E.ns.spec_auto;
  h->tune = all_auto;
  const int* caps = h->precision == 0 ? kTuneCapsF64 : kTuneCaps;
  const int n_caps = h->precision == 0 ? 4 : 5;
  while (left > 0) {
    int b = left < G ? left : G;
    // Autotuning of the speculation cap: from iteration tune_next, one batch per candidate
    // in the order c_0 .. c_{n-1}, c_{n-1} .. c_0 (the sampler's regime drifts from
    // batch to batch; the mirrored order cancels a linear drift), scored by summed walk-kernel
    // device time per likelihood call; the best is kept until the next pass 64 iterations
    // later.  Any depth gives the chain of the one-step walk (exactly in FP64), so this only
    // moves time.
    int64_t it_now = h->host_ns.empty() ? 0 : h->host_ns[0].iteration;
    // First cap, from the cost structure once a batch has run: a proposal of fewer than ~1k
    // active bins (with relative binning: edges plus exact-range bins) is a short likelihood whose rounds are dominated by fixed costs (largest
    // cap); a longer one costs a full evaluation per speculative proposal (small cap).
    if (h->tune && !h->tune_guessed && it_now >= 1) {
      double bins = 0.0, evals = 0.0;
      for (auto& S : h->host_ns) { bins += (double)S.n_bins_eval; evals += (double)S.n_spec_eval; }
      const bool short_lik = evals > 0.0 && bins < 1024.0 * evals;
      const int cap = h->precision == 0 ? (short_lik ? 8 : 2) : (short_lik ? 32 : 4);
      if ((r = set_spec_cap(h, cap))) return r;
      h->tune_best = cap;
      h->tune_guessed = true;
    }
    int64_t like0 = 0;
    double ms0 = h->walk_ms;
    bool trial = false;
    int cand = 0;
    if (h->tune && (h->tune_idx >= 0 || it_now >= h->tune_next)) {
      if (h->tune_idx < 0) {
        h->tune_idx = 0;
        for (int i = 0; i < n_caps; ++i) h->tune_ms[i] = h->tune_calls[i] = 0.0;
      }
      cand = h->tune_idx < n_caps ? h->tune_idx : 2 * n_caps - 1 - h->tune_idx;
      if ((r = set_spec_cap(h, caps[cand]))) return r;
      for (auto& S : h->host_ns) like0 += S.n_like;
      b = 1;
      trial = true;
    }
    if ((r = ensure_dead_capacity(h, b))) return r;
    if ((r = build_graph(h, b))) return r;
    cudaError_t e = cudaGraphLaunch(h->graph_exec[b], h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "graph launch");
    if ((r = download_states(h))) return r;
    for (int i = 0; i < b; ++i) {
      float ms = 0.f;
      e = cudaEventElapsedTime(&ms, h->walk_events[2 * i], h->walk_events[2 * i + 1]);
      if (e != cudaSuccess) return cuda_fail(h, e, "walk timing");
      h->walk_ms += ms;
    }
    h->kernel_launches += h->launches_per_batch[b];
    if (trial) {
      int64_t like1 = 0;
      for (auto& S : h->host_ns) like1 += S.n_like;
      h->tune_ms[cand] += h->walk_ms - ms0;
      h->tune_calls[cand] += (double)(like1 - like0);
      if (++h->tune_idx == 2 * n_caps) {
        int best = 0;
        double best_cost = INFINITY;
        for (int i = 0; i < n_caps; ++i) {
          const double cost = h->tune_ms[i] / (h->tune_calls[i] > 0.0 ? h->tune_calls[i] : 1.0);
          if (cost < best_cost) { best_cost = cost; best = i; }
        }
        h->tune_best = caps[best];
        if ((r = set_spec_cap(h, h->tune_best))) return r;
        h->tune_idx = -1;
        h->tune_next = (int)h->host_ns[0].iteration + 64;
      }
    }
    left -= b;
    all_done = true;
    for (auto& S : h->host_ns) all_done = all_done && S.done;
    if (all_done) break;
  }
  if (progress) fill_progress(h, progress);
  for (auto& S : h->host_ns)
    if (S.overflow) return set_error(h, NS_ENOMEM, "dead-point store overflow");
  for (size_t e = 0; e < h->host_ns.size(); ++e)
    if (h->host_ns[e].chol_bad)
      return set_error(h, NS_EINVAL, "event %zu: the survivors' covariance is not positive definite (HRSS)", e);
  if ((r = watchdog_report(h))) return r;
  bool warn = false;
  for (auto& S : h->host_ns) warn = warn || S.zero_accept;
  return warn ? NS_WMAXMCMC : NS_OK;
}

extern "C" int ns_evidence(ns_handle* h, int event, double* log_z, double* log_z_err, double* info_h,
                           int64_t* n_like) {
  if (!h) return set_error(nullptr, NS_EINVAL, "handle is NULL");
  if (event < 0 || event >= (int)h->events.size()) return set_error(h, NS_EINVAL, "event out of range");
  cudaSetDevice(h->device);
  int r = download_states(h);
  if (r) return r;
  const NsState& S = h->host_ns[event];
  const int64_t nd = S.n_dead;
  std::vector<double> dl(nd), dw(nd), ll(S.n_live);
  cudaError_t e;
  if ((e = copy_on(h, dl.data(), S.dead_lnl, sizeof(double) * nd, cudaMemcpyDeviceToHost)) ||
      (e = copy_on(h, dw.data(), S.dead_logw, sizeof(double) * nd, cudaMemcpyDeviceToHost)) ||
      (e = copy_on(h, ll.data(), S.live_lnl, sizeof(double) * S.n_live, cudaMemcpyDeviceToHost)))
    return cuda_fail(h, e, "evidence download");
  // ln Z = logsumexp(dead ln w, live ln L + ln X - ln n), in FP64
  double m = -INFINITY;
  for (double v : dw) m = std::fmax(m, v);
  const double lxn = S.log_x - std::log((double)S.n_live);
  for (double v : ll) m = std::fmax(m, v + lxn);
  double s = 0.0;
  for (double v : dw) s += std::exp(v - m);
  for (double v : ll) s += std::exp(v + lxn - m);
  const double lz = m + std::log(s);
  double hsum = 0.0;
  for (int64_t i = 0; i < nd; ++i) hsum += std::exp(dw[i] - lz) * dl[i];
  for (double v : ll) hsum += std::exp(v + lxn - lz) * v;
  // replays on the device
  const int R = 200;
  double* d_out;
  if ((r = alloc(h, (void**)&d_out, sizeof(double) * R, "replays"))) return r;
  replay_kernel<<<R, kSelThreads, 0, h->stream>>>(h->d_ns, event, d_out);
  std::vector<double> rep(R);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(rep.data(), d_out, sizeof(double) * R, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cudaFree(d_out);
  if (e != cudaSuccess) return cuda_fail(h, e, "replays");
  double mean = 0.0;
  for (double v : rep) mean += v;
  mean /= R;
  double var = 0.0;
  for (double v : rep) var += (v - mean) * (v - mean);
  if (log_z) *log_z = lz;
  if (log_z_err) *log_z_err = std::sqrt(var / R);
  if (info_h) *info_h = hsum - lz;
  if (n_like) *n_like = S.n_like;
  return NS_OK;
}

extern "C" int ns_posterior(ns_handle* h, int event, double* theta_out, double* logw_out, int64_t cap,
                            int64_t* n_out) {
  if (!h) return set_error(nullptr, NS_EINVAL, "handle is NULL");
  if (event < 0 || event >= (int)h->events.size()) return set_error(h, NS_EINVAL, "event out of range");
  if (cap < 0 || (cap > 0 && (!theta_out || !logw_out))) return set_error(h, NS_EINVAL, "bad output arrays");
  cudaSetDevice(h->device);
  double lz;
  int r = ns_evidence(h, event, &lz, nullptr, nullptr, nullptr);
  if (r) return r;
  const NsState& S = h->host_ns[event];
  const int64_t total = S.n_dead + S.n_live;
  if (n_out) *n_out = total;
  const int64_t m = cap < total ? cap : total;
  if (m == 0) return NS_OK;
  const int D = S.D;
  double *d_u, *d_th;
  if ((r = alloc(h, (void**)&d_u, sizeof(double) * m * D, "posterior u"))) return r;
  if ((r = alloc(h, (void**)&d_th, sizeof(double) * m * kParams, "posterior theta"))) { cudaFree(d_u); return r; }
  const int64_t from_dead = m < S.n_dead ? m : S.n_dead;
  cudaError_t e = copy_on(h, d_u, S.dead_u, sizeof(double) * from_dead * D, cudaMemcpyDeviceToDevice);
  if (e == cudaSuccess && m > from_dead)
    e = copy_on(h, d_u + from_dead * D, S.live_u, sizeof(double) * (m - from_dead) * D, cudaMemcpyDeviceToDevice);
  if (e == cudaSuccess) e = launch_unit_to_theta(h->d_events + event, d_u, m, d_th, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) e = copy_on(h, theta_out, d_th, sizeof(double) * m * kParams, cudaMemcpyDeviceToHost);
  std::vector<double> dw(from_dead), ll(S.n_live);
  if (e == cudaSuccess) e = copy_on(h, dw.data(), S.dead_logw, sizeof(double) * from_dead, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = copy_on(h, ll.data(), S.live_lnl, sizeof(double) * S.n_live, cudaMemcpyDeviceToHost);
  cudaFree(d_u);
  cudaFree(d_th);
  if (e != cudaSuccess) return cuda_fail(h, e, "posterior");
  const double lxn = S.log_x - std::log((double)S.n_live);
  for (int64_t i = 0; i < m; ++i)
    logw_out[i] = (i < S.n_dead ? dw[i] : ll[i - S.n_dead] + lxn) - lz;
  return NS_OK;
}

// ---------------------------------------------------------------- checkpoint / resume
namespace {
const char kMagic[8] = {'G', 'W', 'N', 'S', 'S', 'T', '0', '4'};

bool wr(FILE* f, const void* p, size_t n) { return fwrite(p, 1, n, f) == n; }
bool rd(FILE* f, void* p, size_t n) { return fread(p, 1, n, f) == n; }

template <class T>
bool dev_write(ns_handle* h, FILE* f, const T* d, size_t n) {
  std::vector<T> v(n);
  if (n && copy_on(h, v.data(), d, sizeof(T) * n, cudaMemcpyDeviceToHost) != cudaSuccess) return false;
  return wr(f, v.data(), sizeof(T) * n);
}
}  // namespace

extern "C" int ns_state_save(ns_handle* h, const char* path) {
  if (!h || !path) return set_error(h, NS_EINVAL, "null argument");
  if (h->batch_open) return set_error(h, NS_ESTATE, "a batch is open (ns_batch_end)");
  cudaSetDevice(h->device);
  int r = download_states(h);
  if (r) return r;
  FILE* f = fopen(path, "wb");
  if (!f) return set_error(h, NS_EIO, "cannot open %s for writing", path);
  bool ok = wr(f, kMagic, 8);
  int32_t ne = (int32_t)h->events.size();
  ok = ok && wr(f, &ne, sizeof(ne));
  for (int e = 0; e < ne && ok; ++e) {
    const NsState& S = h->host_ns[e];
    ok = ok && wr(f, &S, sizeof(S));
    ok = ok && dev_write(h, f, S.live_u, (size_t)S.n_live * S.D) && dev_write(h, f, S.live_lnl, (size_t)S.n_live);
    ok = ok && dev_write(h, f, S.dead_u, (size_t)S.n_dead * S.D) && dev_write(h, f, S.dead_lnl, (size_t)S.n_dead);
    ok = ok && dev_write(h, f, S.dead_logw, (size_t)S.n_dead) && dev_write(h, f, S.dead_nlive, (size_t)S.n_dead);
    ok = ok && flow_state_write(h, e, f);
  }
  ok = (fclose(f) == 0) && ok;
  return ok ? NS_OK : set_error(h, NS_EIO, "writing %s failed", path);
}

extern "C" int ns_state_load(ns_handle* h, const char* path) {
  if (!h || !path) return set_error(h, NS_EINVAL, "null argument");
  if (h->batch_open) return set_error(h, NS_ESTATE, "a batch is open (ns_batch_end)");
  cudaSetDevice(h->device);
  FILE* f = fopen(path, "rb");
  if (!f) return set_error(h, NS_EIO, "cannot open %s", path);
  // 1. read and check the whole file on the host; the handle is untouched until it all fits
  struct Rec {
    NsState S;
    std::vector<double> live_u, live_lnl, dead_u, dead_lnl, dead_logw;
    std::vector<int32_t> dead_nlive;
    FlowBlob flow;
  };
  char magic[8];
  int32_t ne = 0;
  bool ok = rd(f, magic, 8) && std::memcmp(magic, kMagic, 8) == 0 && rd(f, &ne, sizeof(ne)) &&
            ne == (int32_t)h->events.size();
  std::vector<Rec> recs(ok ? ne : 0);
  auto rdv = [&](auto& v, size_t n) {
    v.resize(n);
    return rd(f, v.data(), sizeof(v[0]) * n);
  };
  for (int e = 0; e < ne && ok; ++e) {
    Rec& R = recs[e];
    const NsState& cur = h->events[e].ns;
    ok = rd(f, &R.S, sizeof(R.S)) && R.S.n_live == cur.n_live && R.S.k == cur.k && R.S.D == cur.D &&
         R.S.n_dead >= 0 && R.S.n_dead <= (int64_t)1 << 40;
    if (!ok) break;
    const size_t nl = (size_t)R.S.n_live, nd = (size_t)R.S.n_dead, D = (size_t)R.S.D;
    ok = rdv(R.live_u, nl * D) && rdv(R.live_lnl, nl) && rdv(R.dead_u, nd * D) && rdv(R.dead_lnl, nd) &&
         rdv(R.dead_logw, nd) && rdv(R.dead_nlive, nd) && flow_state_parse(h, e, f, R.flow);
  }
  fclose(f);
  if (!ok) return set_error(h, NS_EIO, "reading %s failed or it does not match this handle", path);
  // 2. apply
  for (int e = 0; e < ne; ++e) {
    Rec& R = recs[e];
    int r = grow_dead(h, e, R.S.n_dead, 0);
    if (r) return r;
    EventHost& E = h->events[e];
    const size_t nl = (size_t)R.S.n_live, nd = (size_t)R.S.n_dead, D = (size_t)R.S.D;
    cudaError_t err;
    if ((err = copy_on(h, E.ns.live_u, R.live_u.data(), sizeof(double) * nl * D, cudaMemcpyHostToDevice)) ||
        (err = copy_on(h, E.ns.live_lnl, R.live_lnl.data(), sizeof(double) * nl, cudaMemcpyHostToDevice)) ||
        (nd && (err = copy_on(h, E.ns.dead_u, R.dead_u.data(), sizeof(double) * nd * D, cudaMemcpyHostToDevice))) ||
        (nd && (err = copy_on(h, E.ns.dead_lnl, R.dead_lnl.data(), sizeof(double) * nd, cudaMemcpyHostToDevice))) ||
        (nd && (err = copy_on(h, E.ns.dead_logw, R.dead_logw.data(), sizeof(double) * nd, cudaMemcpyHostToDevice))) ||
        (nd && (err = copy_on(h, E.ns.dead_nlive, R.dead_nlive.data(), sizeof(int32_t) * nd, cudaMemcpyHostToDevice))))
      return cuda_fail(h, err, "state upload");
    if (!flow_state_apply(h, e, R.flow)) return set_error(h, NS_ECUDA, "flow state upload failed");
    // the checkpoint's scalar state (every field before the buffer pointers); this handle keeps
    // its own buffers and dead-store capacity
    NsState S = E.ns;
    std::memcpy(&S, &R.S, offsetof(NsState, live_u));
    S.dead_cap = E.ns.dead_cap;
    WalkTask* dt = h->d_tasks + e;
    if ((err = copy_on(h, h->d_ns + e, &S, sizeof(S), cudaMemcpyHostToDevice)) ||
        (err = copy_on(h, &dt->done, &S.done, sizeof(int32_t), cudaMemcpyHostToDevice)) ||
        (err = copy_on(h, &dt->n_steps, &S.n_steps, sizeof(int32_t), cudaMemcpyHostToDevice)) ||
        (err = copy_on(h, &dt->spec, &S.spec, sizeof(int32_t), cudaMemcpyHostToDevice)))
      return cuda_fail(h, err, "state upload");
  }
  return download_states(h);
}

// ---------------------------------------------------------------- the batch in phases
// ns_step runs deletion, walk and insertion of a batch as one graph.  These calls run the same
// kernels one phase at a time, so that the walkers of a batch can be spread over processes (one
// GPU each) that exchange the walk outputs between the phases: every process holds the same
// handle state, runs the deletion and the insertion itself (deterministic and identical) and
// walks its own range of walkers.
namespace {
int batch_checks(ns_handle* h, bool want_open) {
  if (!h) return set_error(nullptr, NS_EINVAL, "handle is NULL");
  if (h->batch_open != want_open)
    return set_error(h, NS_ESTATE, want_open ? "no batch is open (ns_batch_begin)" : "a batch is open (ns_batch_end)");
  cudaSetDevice(h->device);
  cudaGetLastError();
  return NS_OK;
}
}  // namespace

extern "C" int ns_batch_begin(ns_handle* h) {
  int r = batch_checks(h, false);
  if (r) return r;
  for (const auto& E : h->events)
    if (E.ns.flow_w != 1.0)
      return set_error(h, NS_EINVAL, "the batch-phase calls need flow_accept_weight 1 (they do not carry flow "
                                     "acceptance counts)");
  bool all_done = true;
  for (auto& S : h->host_ns) all_done = all_done && S.done;
  if (all_done) return set_error(h, NS_ESTATE, "every event has finished");
  if ((r = ensure_dead_capacity(h, 1))) return r;
  const int ne = (int)h->events.size();
  cudaError_t e;
  if ((e = cudaMemsetAsync(h->d_status + 2, 0, sizeof(int32_t), h->stream)) != cudaSuccess)
    return cuda_fail(h, e, "watchdog reset");
  int64_t launches = 0;
  select_kernel<<<ne, kSelThreads, 0, h->stream>>>(h->d_ns, h->d_tasks);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(h, e, "select launch");
  for (int ev = 0; ev < ne; ++ev)
    if ((r = flow_enqueue_train(h, ev, h->stream, &launches)) || (r = flow_enqueue_table(h, ev, h->stream, &launches)))
      return r;
  launches += 1;
  if (h->hrss) {
    chol_kernel<<<ne, kSelThreads, 0, h->stream>>>(h->d_ns, h->d_tasks);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(h, e, "covariance launch");
    launches += 1;
  }
  if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return cuda_fail(h, e, "batch begin");
  h->kernel_launches += launches;
  h->batch_open = true;
  return NS_OK;
}

extern "C" int ns_batch_walk(ns_handle* h, int64_t walker_begin, int64_t walker_end) {
  int r = batch_checks(h, true);
  if (r) return r;
  if (walker_begin < 0 || walker_end < walker_begin) return set_error(h, NS_EINVAL, "bad walker range");
  std::vector<int32_t> bt, bl;
  for (size_t ev = 0; ev < h->events.size(); ++ev) {
    const int64_t k = h->events[ev].ns.k;
    for (int64_t j = walker_begin; j < walker_end && j < k; ++j) {
      bt.push_back((int32_t)ev);
      bl.push_back((int32_t)j);
    }
  }
  const int nb = (int)bt.size();
  if (nb == 0) return NS_OK;
  if ((r = ensure_scratch(h, h->scratch_shard, sizeof(int32_t) * 2 * (size_t)nb))) return r;
  int32_t* d_bt = (int32_t*)h->scratch_shard.ptr;
  int32_t* d_bl = d_bt + nb;
  bt.insert(bt.end(), bl.begin(), bl.end());
  cudaError_t e;
  if ((e = cudaMemcpyAsync(d_bt, bt.data(), sizeof(int32_t) * bt.size(), cudaMemcpyHostToDevice, h->stream)))
    return cuda_fail(h, e, "walker map upload");
  if (h->walk_events.size() < 2) {
    for (int i = 0; i < 2; ++i) {
      cudaEvent_t ev;
      if ((e = cudaEventCreate(&ev)) != cudaSuccess) return cuda_fail(h, e, "event create");
      h->walk_events.push_back(ev);
    }
  }
  if ((e = cudaEventRecord(h->walk_events[0], h->stream)) != cudaSuccess) return cuda_fail(h, e, "event");
  e = h->hrss ? launch_hrss(h->precision, h->waveform, h->max_det, h->d_events, h->d_tasks, d_bt, d_bl, nb, h->stream)
              : launch_walk(h->precision, h->waveform, h->max_det, h->d_events, h->d_tasks, d_bt, d_bl, nb, h->stream,
                            walk_extras(h));
  if (e != cudaSuccess) return cuda_fail(h, e, "walk launch");
  if ((e = cudaEventRecord(h->walk_events[1], h->stream)) != cudaSuccess) return cuda_fail(h, e, "event");
  if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return cuda_fail(h, e, "walk");
  float ms = 0.f;
  if ((e = cudaEventElapsedTime(&ms, h->walk_events[0], h->walk_events[1])) != cudaSuccess)
    return cuda_fail(h, e, "walk timing");
  h->walk_ms += ms;
  h->kernel_launches += 1;
  return NS_OK;
}

extern "C" int ns_batch_walk_io(ns_handle* h, int event, int64_t walker_begin, int64_t walker_end, double* u,
                                double* lnl, int32_t* n_accept, int32_t* n_like, int64_t* n_bins, int64_t* n_spec,
                                int ptr_kind, int write) {
  int r = batch_checks(h, true);
  if (r) return r;
  if (event < 0 || event >= (int)h->events.size()) return set_error(h, NS_EINVAL, "event out of range");
  const NsState& S = h->events[event].ns;
  if (walker_begin < 0 || walker_end < walker_begin || walker_end > S.k)
    return set_error(h, NS_EINVAL, "walker range must lie in [0, num_delete = %d]", S.k);
  if (ptr_kind != NS_PTR_HOST && ptr_kind != NS_PTR_DEVICE) return set_error(h, NS_EINVAL, "bad ptr_kind");
  const size_t n = (size_t)(walker_end - walker_begin), D = S.D, j0 = (size_t)walker_begin;
  if (n == 0) return NS_OK;
  if (!u || !lnl || !n_accept || !n_like || !n_bins || !n_spec) return set_error(h, NS_EINVAL, "null array");
  const cudaMemcpyKind kind = write ? (ptr_kind == NS_PTR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice)
                                    : (ptr_kind == NS_PTR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice);
  struct Part { void* dev; void* user; size_t bytes; };
  const Part parts[6] = {{S.w_uo + j0 * D, u, sizeof(double) * n * D},
                         {S.w_lo + j0, lnl, sizeof(double) * n},
                         {S.w_na + j0, n_accept, sizeof(int32_t) * n},
                         {S.w_nl + j0, n_like, sizeof(int32_t) * n},
                         {S.w_nb + j0, n_bins, sizeof(int64_t) * n},
                         {S.w_ns + j0, n_spec, sizeof(int64_t) * n}};
  cudaError_t e = cudaSuccess;
  for (const Part& p : parts) {
    e = write ? cudaMemcpyAsync(p.dev, p.user, p.bytes, kind, h->stream)
              : cudaMemcpyAsync(p.user, p.dev, p.bytes, kind, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "walk output copy");
  }
  if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return cuda_fail(h, e, "walk output copy");
  return NS_OK;
}

extern "C" int ns_batch_end(ns_handle* h, ns_progress* progress) {
  int r = batch_checks(h, true);
  if (r) return r;
  const int ne = (int)h->events.size();
  insert_kernel<<<ne, kSelThreads, 0, h->stream>>>(h->d_ns, h->d_tasks);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "insert launch");
  h->kernel_launches += 1;
  h->batch_open = false;
  if ((r = download_states(h))) return r;
  if (progress) fill_progress(h, progress);
  for (auto& S : h->host_ns)
    if (S.overflow) return set_error(h, NS_ENOMEM, "dead-point store overflow");
  for (size_t ev = 0; ev < h->host_ns.size(); ++ev)
    if (h->host_ns[ev].chol_bad)
      return set_error(h, NS_EINVAL, "event %zu: the survivors' covariance is not positive definite (HRSS)", ev);
  if ((r = watchdog_report(h))) return r;
  bool warn = false;
  for (auto& S : h->host_ns) warn = warn || S.zero_accept;
  return warn ? NS_WMAXMCMC : NS_OK;
}
