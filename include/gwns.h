/*
 * gwns.h -- C ABI of libgwns, a GB300 (sm_103a) implementation of the batched
 * acceptance-walk nested sampler for gravitational-wave inference described in
 * arXiv 2509.04336 ("Gravitational-wave inference at GPU speed: a bilby-like nested
 * sampling kernel within blackjax-ns").
 *
 * What the library computes (the paper's statement of the problem):
 *   evidence     Z = int L(d|theta) pi(theta) dtheta                     (Eq. 2, Sec. 2.1)
 *   posterior    P(theta|d) = L pi / Z, as weighted dead + live points   (Eq. 1; Sec. 3.2 weights)
 *   likelihood   ln L = -1/2 sum_det <d - h_det | d - h_det>,
 *                <a|b> = 4 df Re sum_k conj(a_k) b_k / S_n(f_k)          (Sec. 3.3)
 *   sampler      batched nested sampling: delete the k lowest live points, L* = max of
 *                the deleted, evolve k constrained chains in parallel     (Sec. 2.2.3)
 *   inner kernel differential-evolution acceptance walk in the unit cube,
 *                accepting iff L > L*, walk length tuned per batch        (Sec. 3.1, Sec. 3.2)
 *
 * Conventions (all entry points):
 *   - Return 0 (NS_OK) on success, a negative NS_E* code on failure, NS_WMAXMCMC (> 0)
 *     as a warning.  No C++ exception crosses the ABI.  ns_last_error() returns a
 *     message for the last failure of a handle (or of ns_init when handle is NULL).
 *   - Physical parameter vectors theta are 11 doubles in this order:
 *       chirp mass [Msun, detector frame], mass ratio q = m2/m1 <= 1, chi_1, chi_2,
 *       luminosity distance [Mpc], theta_jn [rad], psi [rad], phase phi_c [rad],
 *       geocentre coalescence time t_c [s, relative to the segment reference],
 *       right ascension [rad], declination [rad].
 *   - Unit-cube vectors u hold the D sampled (non-FIXED) parameters in the same order.
 *   - Arrays are row-major and densely packed.  ptr_kind says whether the caller's
 *     pointers are host (NS_PTR_HOST, pageable or pinned) or device (NS_PTR_DEVICE)
 *     memory.  Caller buffers are borrowed for the duration of the call only; with
 *     device pointers the work is enqueued on `stream` and the call returns after
 *     enqueueing (the caller synchronises); with host pointers the call blocks.
 *   - stream == NULL means the handle's own stream (created non-blocking, so it is not ordered
 *     with the legacy default stream); to order a call with work on the legacy default stream
 *     pass cudaStreamLegacy.
 *   - The library owns every buffer it allocates; ns_free releases them.
 *   - One handle per host thread; a handle is bound to the device given to ns_init.
 */
#ifndef GWNS_H
#define GWNS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GWNS_N_PARAMS 11
#define GWNS_MAX_DET 4
#define GWNS_MAX_EVENTS 256

/* status codes */
#define NS_OK 0
#define NS_EINVAL (-1)      /* bad argument or configuration                          */
#define NS_ECUDA (-2)       /* a CUDA runtime call failed                             */
#define NS_ENOMEM (-3)      /* device or host allocation failed                       */
#define NS_ENONFINITE (-4)  /* non-finite input (theta, data, PSD) or result           */
#define NS_ETIMEOUT (-5)    /* a device loop hit its iteration/clock budget            */
#define NS_ESTATE (-6)      /* call not valid in the current state (e.g. run finished) */
#define NS_EIO (-7)         /* checkpoint file could not be written or read            */
#define NS_WMAXMCMC 1       /* warning: a walk batch reached maxmcmc steps with no     */
                            /* accepted move for some walker (its start is returned)   */

/* prior kinds (Table 1) */
#define NS_PRIOR_UNIFORM 0   /* x = lo + u (hi - lo)                                   */
#define NS_PRIOR_POWERLAW 1  /* density ~ x^alpha on [lo, hi], alpha != -1             */
#define NS_PRIOR_SINE 2      /* density ~ sin x on [lo, hi] within [0, pi]              */
#define NS_PRIOR_COSINE 3    /* density ~ cos x on [lo, hi] within [-pi/2, pi/2]        */
#define NS_PRIOR_FIXED 4     /* held at `value`, not sampled                            */

#define NS_WAVEFORM_TAYLORF2 0      /* 3.5PN aligned-spin TaylorF2, zero above f_ISCO  */
#define NS_WAVEFORM_PHENOMD_FORM 1  /* IMRPhenomD-form inspiral-merger-ringdown        */

#define NS_PREC_FP64 0      /* every step in FP64 (the plain walk)                              */
#define NS_PREC_MIXED 1     /* FP32 amplitude and inner products with compensated sums; the     */
                            /* phase, its reduction and the time shift in FP64; FP64 lnL         */
                            /* assembly and evidence                                             */
#define NS_PREC_MIXED_FF 2  /* as NS_PREC_MIXED, but the phase is carried as a float-float pair  */
                            /* (about 48-bit significand) on the FP32 pipe and the time shift is */
                            /* reduced exactly through a 9-bit head; per-walker constants FP64   */

#define NS_TERM_DLOGZ 0           /* stop when ln(Z + L_max X) - ln Z < term_value (Sec. 4.1.1)   */
#define NS_TERM_FRAC_REMAINING 1  /* stop when L_mean X < term_value * Z (Sec. 4.2)              */

#define NS_PROPOSAL_DE 0        /* differential-evolution steps only (Sec. 3.1)            */
#define NS_PROPOSAL_DE_FLOW 1   /* DE steps mixed with flow independence proposals          */
#define NS_PROPOSAL_HRSS 2      /* hit-and-run slice sampling as the inner kernel (Sec. 2.2, */
                                /* Sec. 5; see ns_hrss_batch): hrss_moves moves a batch     */

#define NS_PTR_HOST 0
#define NS_PTR_DEVICE 1

typedef struct ns_prior {
    int32_t kind;      /* NS_PRIOR_*                                  */
    int32_t periodic;  /* nonzero: wrap u into [0, 1) in the walk      */
    double lo, hi;     /* support                                      */
    double alpha;      /* power-law index (NS_PRIOR_POWERLAW)          */
    double value;      /* NS_PRIOR_FIXED value                         */
} ns_prior;

/* Sampler settings of one event (Sec. 3.2; values of Sec. 4.1.1 and Sec. 4.2). */
typedef struct ns_config {
    ns_prior prior[GWNS_N_PARAMS];
    int32_t n_live;       /* live points                                            */
    int32_t num_delete;   /* k, points deleted and replaced per batch (1 <= k < n_live) */
    int32_t naccept;      /* target accepted steps per walk                         */
    int32_t maxmcmc;      /* cap on the walk length                                 */
    double delay;         /* sequential smoothing of the walk-length update; < 0 means
                             naccept - 1.  The batch uses delay_k with
                             delay_k/(delay_k+1) = (delay/(delay+1))^k              */
    int32_t use_ratio;    /* nonzero: sample ln L + 1/2 sum <d|d> (likelihood ratio)  */
    int32_t term_kind;    /* NS_TERM_*                                              */
    double term_value;    /* dlogZ threshold or evidence fraction                   */
    int32_t precision;    /* NS_PREC_*; the same for every event of a handle        */
    int32_t waveform;     /* NS_WAVEFORM_*; the same for every event of a handle    */
    int32_t max_iter;     /* hard cap on batches (0: 1000000)                       */
    int32_t n_steps0;     /* first walk length (0: ceil(naccept / 0.25))            */
    uint64_t seed;        /* Philox key word 0; key word 1 is the event index      */
    int32_t spec_depth;   /* walk steps evaluated per round (1..32); 0: chosen per batch
                             from the acceptance rate.  Any value gives the same chain.  */
    int32_t proposal;     /* NS_PROPOSAL_DE, or NS_PROPOSAL_DE_FLOW: DE steps mixed with
                             independence proposals from a normalising flow trained on the
                             live points (see "Flow proposal" below)                  */
    double p_flow;        /* DE_FLOW: probability that a walk step is a flow step, [0, 1] */
    int32_t flow_layers;  /* DE_FLOW: affine coupling layers, 1..16 (0: 8)            */
    int32_t flow_every;   /* DE_FLOW: retrain the flow every this many batches (0: 1)  */
    int32_t flow_epochs;  /* DE_FLOW: full-batch Adam steps per retraining (0: 50)     */
    int32_t hrss_moves;   /* HRSS: slice-sampling moves per walker and batch, fixed (no
                             walk-length retune; 0: 2 D).  Every event of a handle uses
                             HRSS or none does.  Needs n_live - num_delete > D.          */
    double flow_lr;       /* DE_FLOW: Adam learning rate (0: 3e-3)                  */
    double flow_accept_weight; /* DE_FLOW: weight of an accepted flow step in the walk-length
                             retune, in [1, 1e6] (0: 1).  The retune aims the batch mean of
                             (accepted DE steps + w x accepted flow steps) at naccept: an
                             accepted independence proposal moves a walker as far as w DE
                             acceptances.  1 counts both kinds alike.  Weights above 1 are an
                             experiment: they shorten the walks, and on an 11-parameter event
                             they were measured to bias ln Z.  A handle with a weight other
                             than 1 cannot use the batch-phase calls (ns_batch_*), which do
                             not carry the flow acceptance counts.                       */
} ns_config;

/* One detector's data.  Pointers are HOST arrays of n_bins doubles, copied by ns_init. */
typedef struct ns_detector {
    double vertex[3];     /* Earth-fixed position [m]                               */
    double x_arm[3];      /* unit vector of the x arm                               */
    double y_arm[3];      /* unit vector of the y arm                               */
    const double* d_re;   /* Re d(f_k) [1/Hz]                                       */
    const double* d_im;   /* Im d(f_k) [1/Hz]                                       */
    const double* psd;    /* one-sided S_n(f_k) [1/Hz], > 0                          */
} ns_detector;

/* One event: data on the grid f_k = f_min + k df, k = 0 .. n_bins-1. */
typedef struct ns_event {
    int32_t n_det;        /* 1 .. GWNS_MAX_DET                                      */
    int32_t n_bins;       /* >= 1                                                   */
    double f_min;         /* [Hz] > 0                                               */
    double df;            /* [Hz] > 0 (1 / segment duration)                        */
    double gmst;          /* Greenwich sidereal angle of the event [rad]           */
    ns_detector det[GWNS_MAX_DET];
} ns_event;

/* Progress of one event after ns_step. */
typedef struct ns_progress {
    int64_t iterations;   /* batches completed                                      */
    int64_t n_like;       /* likelihood evaluations so far                          */
    double log_z;         /* ln Z of the dead points so far                         */
    double dlogz;         /* ln(Z + L_max X) - ln Z                                 */
    double log_x;         /* expected ln X of the live set                          */
    double lnl_star;      /* threshold of the last batch                            */
    double mean_accept;   /* mean accepted steps per walker, last batch             */
    int32_t n_steps;      /* walk length of the next batch                          */
    int32_t done;         /* termination reached                                    */
    int64_t n_bins;       /* active (walker, bin) pairs evaluated by walks so far    */
                          /* (relative binning: the edges and exact-range bins)    */
    double walk_ms;       /* device time of this handle's walk launches so far [ms], */
                          /* from CUDA events on the launching stream (all events)  */
    int64_t kernel_launches; /* kernels launched by ns_step so far (all events)     */
    int64_t n_spec;       /* likelihoods evaluated by walks so far, including those   */
                          /* evaluated ahead and dropped after an earlier acceptance  */
    int32_t spec_depth;   /* speculation depth of the next batch                    */
    int32_t spec_cap;     /* the cap on it in force (chosen by the autotuner when the
                             configuration leaves the depth automatic)                */
    double mean_accept_flow; /* mean accepted flow steps per walker, last batch (of
                             mean_accept)                                             */
} ns_progress;

typedef struct ns_handle ns_handle;

/* Create a sampler for n_events events on CUDA device `device`.  cfg and ev are
 * arrays of n_events.  Copies and preprocesses all inputs (whitening, basis tables,
 * prefix sums), allocates the live/dead stores and draws the initial live points
 * (Sec. 2.2.1: n_live draws from the prior).  On failure *out is NULL and
 * ns_last_error(NULL) describes the problem. */
int ns_init(const ns_config* cfg, const ns_event* ev, int n_events, int device, ns_handle** out);

/* Detector strain of the waveform model for n parameter vectors (the projection of
 * Sec. 3.3 / Sec. 4.1.1 network): h_re, h_im are [n][n_det][n_bins] in physical units
 * (1/Hz), FP64.  theta is [n][11]. */
int ns_waveform(ns_handle* h, int event, const double* theta, int n,
                double* h_re, double* h_im, int ptr_kind, void* stream);

/* ln L (or ln Lambda under use_ratio) of n parameter vectors theta [n][11]
 * (Sec. 3.3), computed in the handle's precision.  lnl is [n]. */
int ns_likelihood_batch(ns_handle* h, int event, const double* theta, int n,
                        double* lnl, int ptr_kind, void* stream);

/* One walk batch of the inner kernel (Sec. 3.1): n walkers start at u0 [n][D] with
 * ln L lnl0 [n] and take n_steps DE steps against the survivor set live_u [n_live_pts][D],
 * accepting iff ln L > lnl_star.  Random numbers come from Philox4x64-10 with key
 * (seed, event) and counters (step, walker_offset + w, iteration, tag), so a call is a
 * pure function of its arguments.  Outputs: u_out [n][D], lnl_out [n], n_accept [n],
 * n_like [n] (likelihood calls; out-of-bounds proposals are rejected without a call).
 * n_live_pts >= 2.  Returns NS_WMAXMCMC when a walker accepted nothing. */
int ns_walk_batch(ns_handle* h, int event, const double* live_u, int n_live_pts,
                  const double* u0, const double* lnl0, double lnl_star,
                  int n, int n_steps, int64_t iteration, int64_t walker_offset,
                  double* u_out, double* lnl_out, int32_t* n_accept, int32_t* n_like,
                  int ptr_kind, void* stream);

/* ns_walk_batch for callers that cannot allocate device memory after start-up (no
 * counterpart in the paper).  Processes that reserve a fixed device-memory budget at
 * start-up, or latency-critical loops that cannot absorb the device synchronisation of
 * cudaMalloc/cudaFree, need a walk that allocates nothing: this call keeps the walk's task
 * descriptor and block map in a fixed static device array (about 64 KB per GPU, held until
 * the process exits) instead of growing scratch with cudaMalloc, and calls no allocation
 * routine.  All arrays are DEVICE pointers with ns_walk_batch's layouts; the work is
 * enqueued on `stream` and the call returns without waiting.  At most 8192 walkers per
 * call (NS_EINVAL beyond).  The first call on a device looks up the array's address; make
 * it before any stream capture.  Calls whose kernels overlap on the GPU share the array and
 * race: order them on one stream.  Results equal ns_walk_batch's for the same arguments.
 * An event with flow proposals (NS_PROPOSAL_DE_FLOW, p_flow > 0) writes its proposal table
 * into the handle's own batch table, which ns_step also uses: there n <= num_delete and
 * n_steps <= maxmcmc (NS_EINVAL beyond), and the call must not overlap an ns_step of the
 * same handle on the GPU. */
int ns_walk_batch_noalloc(ns_handle* h, int event, const double* live_u, int n_live_pts,
                          const double* u0, const double* lnl0, double lnl_star,
                          int n, int n_steps, int64_t iteration, int64_t walker_offset,
                          double* u_out, double* lnl_out, int32_t* n_accept, int32_t* n_like,
                          void* stream);

/* Run up to max_batches batches of the sampler on every unfinished event (Sec. 2.2.3,
 * Sec. 3.2): deletion, evidence update, walk, insertion, walk-length retune and the
 * termination test all run on the device.  progress is [n_events] (may be NULL).
 * Returns NS_OK when it ran; progress[e].done reports termination.  NS_ETIMEOUT: the watchdog
 * (ns_set_watchdog, ns_set_abort) ended walks early in a batch of this call; the batches ran to
 * completion with the truncated walks (every walker still at a point above L*), the state is
 * consistent and a later call continues the run.  With HRSS (NS_PROPOSAL_HRSS) each batch also
 * forms the Cholesky factor of the survivors' covariance on the device; NS_EINVAL if it is not
 * positive definite. */
int ns_step(ns_handle* h, int max_batches, ns_progress* progress);

/* ---- a batch in phases: walker sharding of one event over processes (one GPU each) ----
 * ns_step runs a batch (Sec. 2.2.3) as deletion, walk and insertion on the device.  These calls
 * run the same kernels one phase at a time, so that R processes holding identical handles (same
 * events, configurations and seeds) can split the k walkers of a batch -- the walks are
 * independent and each walker's chain depends only on its index (its Philox counters) -- and
 * exchange the k walk outputs, k x (D + 1) FP64 plus counters, before the insertion:
 *   ns_batch_begin   deletion, evidence update, starts (and the flow training or the HRSS
 *                    covariance of the batch); blocks until done
 *   ns_batch_walk    the walks of walkers [walker_begin, walker_end) of every event (clipped
 *                    to each event's num_delete)
 *   ns_batch_walk_io copies the walk outputs of walkers [walker_begin, walker_end) of one event
 *                    out of the handle (write = 0) or into it (write = 1): u [n][D], lnl [n],
 *                    n_accept [n], n_like [n], n_bins [n], n_spec [n] (n = end - begin), host or
 *                    device pointers per ptr_kind (on the handle's stream; returns when done)
 *   ns_batch_end     insertion, walk-length retune, termination; progress as ns_step's
 * Every walker's outputs must be in the handle (walked here or written in) before ns_batch_end;
 * run on every process, the sequence leaves every handle in the state ns_step would, bit for bit.
 * Between ns_batch_begin and ns_batch_end, ns_step and checkpoints are refused (NS_ESTATE). */
int ns_batch_begin(ns_handle* h);
int ns_batch_walk(ns_handle* h, int64_t walker_begin, int64_t walker_end);
int ns_batch_walk_io(ns_handle* h, int event, int64_t walker_begin, int64_t walker_end, double* u, double* lnl,
                     int32_t* n_accept, int32_t* n_like, int64_t* n_bins, int64_t* n_spec, int ptr_kind, int write);
int ns_batch_end(ns_handle* h, ns_progress* progress);

/* Watchdog of the walks (failure detection on the device).  Every walk -- ns_walk_batch,
 * ns_walk_batch_noalloc, ns_hrss_batch and the walks of ns_step -- checks between its rounds
 * (HRSS: between moves) a time budget and an abort flag, and when either has run out it stops
 * after the current round, keeps its current point (which satisfies L > L*) and reports
 * NS_ETIMEOUT (host-pointer calls and ns_step; device-pointer walks return before the kernel
 * runs, so their timeout shows in the next ns_step or host-pointer walk of the handle).
 * ns_set_watchdog: budget_seconds > 0 bounds each walker's walk in wall time (GPU global timer,
 * from the start of its thread block); 0 switches the budget off (the default).
 * ns_set_abort: flag != 0 makes every running and later walk of the handle stop after its
 * current round, until it is called again with 0.  ns_set_abort may be called from another host
 * thread while ns_step runs (it writes the flag through a stream of its own and returns when the
 * flag is on the device). */
int ns_set_watchdog(ns_handle* h, double budget_seconds);
int ns_set_abort(ns_handle* h, int flag);

/* Final evidence of an event: the dead points plus the final live points, each with
 * weight L_i X / n_live.  log_z_err is the standard deviation of ln Z over replays
 * with shrinkage factors t ~ Beta(n_i, 1); info_h is the information H. */
int ns_evidence(ns_handle* h, int event, double* log_z, double* log_z_err,
                double* info_h, int64_t* n_like);

/* Posterior samples of an event (dead then final live points): theta_out [cap][11]
 * physical parameters and logw_out [cap] normalised log weights (Eq. 1).  *n_out is
 * the number of points available; at most cap are written.  Host pointers. */
int ns_posterior(ns_handle* h, int event, double* theta_out, double* logw_out,
                 int64_t cap, int64_t* n_out);

/* Checkpoint / resume of the whole sampler state (live sets, dead stores, evidence
 * accumulators, walk lengths, iteration counters).  A resumed run continues the
 * same Philox streams and so replays bit-identically. */
int ns_state_save(ns_handle* h, const char* path);
int ns_state_load(ns_handle* h, const char* path);

/* ---------------------------------------------------------------- Flow proposal
 * The paper (Sec. 5) motivates normalising-flow proposals for a batched GPU nested sampler
 * without fixing a design; this library's reading (an event configured with
 * NS_PROPOSAL_DE_FLOW):
 *   q(u) on the unit cube: z0 = (logit(u) - mu) / sigma, then L RealNVP affine coupling
 *   layers (Dinh et al. 2017), layer l conditioning on the dimensions d with (d + l) even
 *   through a tanh MLP D -> 128 -> 128 -> 2 D that gives log-scales s = 2 tanh(s_raw / 2)
 *   and shifts t; base density N(0, I).  Matrix products run on the tensor cores with
 *   bf16 operands and FP32 accumulation.
 *   Walk: step t of walker w is a flow step with probability p_flow (Philox word
 *   (t, walker_offset + w, iteration, 6)[0]); it proposes u' = F^-1(x), x ~ N(0, I) from
 *   Philox blocks (t, walker_offset + w, iteration, 16 + c), and accepts iff
 *   ln U < ln q(u) - ln q(u') (word 1) and ln L(u') > ln L* -- a Metropolis-Hastings step
 *   that keeps the prior restricted to L > L* invariant.  The q test comes first, so a
 *   rejected flow step costs no likelihood call.
 *   Training: maximum likelihood on the n_live - k survivors (samples of the prior above
 *   the new L*) of every flow_every-th batch, after the deletion: mu, sigma re-estimated,
 *   flow_epochs full-batch Adam steps (beta (0.9, 0.999), eps 1e-8); weights and Adam state
 *   carry over from batch to batch.
 * Parameters are a flat FP32 vector, per layer W1 [128][D], b1 [128], W2 [128][128],
 * b2 [128], W3 [2D][128] (rows: s_0..s_{D-1}, t_0..t_{D-1}), b3 [2D]; ns_flow_num_params
 * gives its length.  Every call below returns NS_ESTATE for an event without a flow.
 * Host pointers unless a ptr_kind says otherwise. */
int ns_flow_num_params(ns_handle* h, int event, int32_t* n_params);
/* Replace the flow's weights and standardisation (mu, sigma [D]); resets Adam. */
int ns_flow_set(ns_handle* h, int event, const float* params, const double* mu, const double* sigma);
int ns_flow_get(ns_handle* h, int event, float* params, double* mu, double* sigma);
/* ln q(u) of n points u [n][D] strictly inside the unit cube. */
int ns_flow_logq(ns_handle* h, int event, const double* u, int n, double* logq, int ptr_kind, void* stream);
/* The proposal table a walk batch would use: for walkers w < n (walker ids walker_offset + w)
 * and steps t < n_steps, u_out [n][n_steps][D] = F^-1(x) and logq_out [n][n_steps] = ln q. */
int ns_flow_sample(ns_handle* h, int event, int64_t iteration, int64_t walker_offset, int n, int n_steps,
                   double* u_out, double* logq_out, int ptr_kind, void* stream);
/* Mean of -ln q over n points u [n][D] and its gradient grad [n_params] (no update). */
int ns_flow_grad(ns_handle* h, int event, const double* u, int n, float* grad, double* loss);
/* Re-estimate mu, sigma on u [n][D] (n <= 4096) and take `epochs` Adam steps on the mean of
 * -ln q; losses [epochs] (may be NULL) receives the loss before each step. */
int ns_flow_train(ns_handle* h, int event, const double* u, int n, int epochs, double* losses);

/* ---- hit-and-run slice sampling (the inner kernel named in Sec. 2.2 and Sec. 5; Neal 2003) ----
 * One batch of the alternative inner kernel (the handle's precision), host arrays: n walkers
 * start at u0 [n][D] (unit cube) with ln L lnl0 [n] and each make n_steps slice-sampling moves
 * under ln L > lnl_star.  A move draws a line through the walker with direction C z / |z|
 * (z standard normal; C C^T the sample covariance of the survivors live_u [n_live_pts][D]),
 * places a bracket one unit of the line wide at random around the walker, steps out by one unit
 * while the bracket's ends satisfy the constraint (at most 9 steps, split at random between the
 * sides), then shrinks it around uniform draws until one satisfies the constraint (at most 100
 * draws, after which the walker stays).  Points outside the cube cost no likelihood call;
 * periodic coordinates wrap.  Random numbers: Philox4x64-10, key (seed, event), counters
 * (step, walker_offset + w, iteration, tag), tags 32..34 normals, 40 bracket, 48.. shrinkage.
 * Outputs: u_out [n][D], lnl_out [n], n_move [n] (moves made), n_like [n] (likelihood calls).
 * The walkers run on the GPU one CTA each, every candidate's likelihood summed by the whole CTA.
 * Errors: NS_EINVAL (bad sizes, a survivor covariance that is not positive definite:
 * n_live_pts must exceed D), NS_ENONFINITE, NS_ENOMEM, NS_ECUDA, NS_ETIMEOUT (watchdog). */
int ns_hrss_batch(ns_handle* h, int event, const double* live_u, int n_live_pts,
                  const double* u0, const double* lnl0, double lnl_star, int n, int n_steps,
                  int64_t iteration, int64_t walker_offset, double* u_out, double* lnl_out,
                  int32_t* n_move, int32_t* n_like);

/* ---- relative binning (Sec. 3.3 and Sec. 5: the likelihood compression for long signals;
 * Zackay, Dai & Venumadhav 2018) ----
 * Switches event `event` of an NS_PREC_MIXED_FF handle to the relative-binning likelihood.
 * edges [n_edges]: host int32 grid-bin indices of the coarse-bin edges, strictly increasing,
 * edges[0] = 0 and edges[n_edges - 1] = n_bins (the caller keeps ownership).  theta0 [11]:
 * host, the fiducial parameters.  The fiducial template h0 is the template at theta0 continued
 * above its cutoff; per coarse bin and detector the call computes (FP64, stored FP32) the
 * summary data A0 = sum conj(d) h0 w, A1 = sum conj(d) h0 w x, B0, B1, B2 = sum |h0|^2 w x^{0,1,2}
 * (w = 4 df / S_n, x = f - f_edge).  A proposal's ln L then takes r = h / h0 at the edges and,
 * for every coarse bin wholly below its cutoff whose right edge is a grid bin,
 * <d|h> = Re(A0 r + A1 r'), <h|h> = B0 |r|^2 + 2 B1 Re(conj(r) r') + B2 |r'|^2 (r' the slope
 * between the edges); from the first other coarse bin up to the cutoff it sums the bins exactly.
 * ns_likelihood_batch, ns_walk_batch and ns_step of the event use it from then on; n_edges = 0
 * restores the full likelihood.  Call before the first ns_step of the event: the initial live
 * points are re-evaluated.  The setting is not part of a checkpoint.
 * Errors: NS_EINVAL (other precision, bad edges, after the first step, a fiducial that vanishes
 * at an edge), NS_ENONFINITE (theta0 or the summary data), NS_ENOMEM, NS_ECUDA. */
int ns_relbin_set(ns_handle* h, int event, const int32_t* edges, int n_edges, const double* theta0);

/* Coarse-bin edges for ns_relbin_set on the grid f_k = f_min + k df, k < n_bins (the bin-width
 * rule of Zackay, Dai & Venumadhav 2018, which the paper's Sec. 3.3 and Sec. 5 name): with
 * dpsi(f) = 2 pi sum_g sign(g) (f / f_g)^g over g = -5/3, -2/3, 1, 5/3, 7/3 (f_g = f_min for
 * g < 0, the top bin's frequency for g > 0), a bound on how far any template's phase can drift
 * from the fiducial's, each edge after 0 is the first grid bin whose dpsi differs from the
 * previous edge's by more than eps radians; the last edge is n_bins.  Host arithmetic only, no
 * handle and no device: edges [cap] (host, caller-owned) receives min(cap, *n_edges) edges.
 * Returns NS_EINVAL for f_min, df or eps not positive and finite, n_bins < 1, a null n_edges,
 * or cap < *n_edges (then *n_edges still holds the count needed). */
int ns_relbin_edges(double f_min, double df, int n_bins, double eps, int32_t* edges, int cap, int32_t* n_edges);

void ns_free(ns_handle* h);
const char* ns_last_error(ns_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* GWNS_H */
