/*
 * pm.h -- C ABI of the B300 (sm_103a) sparse-matrix permanent estimator.
 *
 * The library estimates per(A) = sum_{pi in S_n} prod_v A_{v,pi(v)} (Eq. 1)
 * of a sparse nonnegative n x n matrix with the adaptive sequential
 * importance sampler of "The Quick and the Dead" (Algorithm 2): many
 * independent trajectories, each picking the active row or column of minimum
 * live degree (Sec. 3.2), drawing a partner from the scaled proposal of
 * Eq. 3, multiplying its weight by the correction B_vu / q(u|v), eliminating
 * the pair with degree updates, and running the scheduled SK / Local scaling
 * (Sec. 3.3, Eq. 5) and DM support filtering (Sec. 2, Sec. 3.3) between steps.
 *
 * Conventions for every function:
 *  - returns pm_status; PM_OK (0) on success.  No function aborts the process
 *    or traps the device; device-side failures come back through a status
 *    word read after the stream synchronises (PM_EDEVICE).
 *  - outputs are written only when the call returns PM_OK, or PM_ETIMEOUT /
 *    PM_ECANCELLED from a call that stopped early (time budget, cancel):
 *    then they describe the trajectories that ran (pm_result.stop says why
 *    a matrix stopped).
 *  - all pointers are caller-owned and not retained after the call returns,
 *    except the handles the library allocates (pm_context, pm_matrix).
 *  - a context serialises its work on one CUDA stream; calls on one context
 *    must not overlap in time from several host threads.
 *  - per(A) = 0 is not an error: PM_OK with log_estimate = -INFINITY,
 *    estimate = 0 and p_match = 0.
 */
#ifndef PM_H_
#define PM_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PM_OK = 0,
    PM_EINVAL = 1,         /* malformed matrix, size mismatch, bad schedule, NULL argument */
    PM_ENOMEM = 2,         /* device or pinned-host allocation failed */
    PM_ECUDA = 3,          /* a CUDA runtime call failed (the message is kept, see pm_last_error) */
    PM_ETIMEOUT = 4,       /* the call's time budget (pm_schedule.time_budget_s) ran out first */
    PM_ECANCELLED = 5,     /* pm_context_cancel stopped the call */
    PM_EUNSUPPORTED = 6,   /* size or option outside what this build supports */
    PM_EDEVICE = 7         /* a kernel reported an internal error through the status word */
} pm_status;

/* Sparse matrix in CSR form.  row_ptr[0] = 0, row_ptr nondecreasing,
 * row_ptr[n] = nnz; col_idx strictly increasing inside each row, in [0, n);
 * values > 0 (float32) or NULL for a 0/1 matrix.  on_device = 1: the three
 * arrays are device pointers of the context's device; 0: host pointers. */
typedef struct {
    int32_t n;
    int32_t on_device;
    int64_t nnz;
    const int64_t* row_ptr;   /* [n + 1] */
    const int32_t* col_idx;   /* [nnz] */
    const float* values;      /* [nnz] or NULL */
} pm_csr;

/* Vertex rule R_V (Alg. 2): two-sided minimum degree over active rows and
 * columns, ties to the lowest unified id (row i -> i, column j -> n + j); or
 * the fixed row order of Alg. 1. */
typedef enum { PM_VR_MIN_DEGREE_2SIDED = 0, PM_VR_ROW_ORDER = 1 } pm_vertex_rule;
/* SK policy P_SK (Sec. 3.3); NONE keeps the outer scaling for the whole trajectory. */
typedef enum { PM_SK_NONE = 0, PM_SK_FIXED = 1, PM_SK_ADAPTIVE = 2, PM_SK_LOCAL = 3 } pm_sk_policy;
/* DM policy P_DM (Sec. 3.3). */
typedef enum { PM_DM_NONE = 0, PM_DM_ALL = 1, PM_DM_THRS = 2, PM_DM_TRCK = 3 } pm_dm_policy;
/* FP32_PROPOSAL: scaling vectors and proposal scores in binary32, log-weights
 * and statistics in binary64.  FP64: everything in binary64. */
typedef enum { PM_PREC_FP32_PROPOSAL = 0, PM_PREC_FP64 = 1 } pm_precision;

/* Inputs of Algorithm 2.  Presets of Sec. 4: two-sided MD, initial_dm = 1,
 * K0 = 100, K = 10, theta = 0.33 with (sk, dm) = fixed_all (FIXED, ALL),
 * adaptive_threshold (ADAPTIVE, THRS), local_threshold (LOCAL, THRS),
 * adaptive_tracked (ADAPTIVE, TRCK), local_tracked (LOCAL, TRCK). */
typedef struct {
    int32_t vertex_rule;   /* pm_vertex_rule */
    int32_t initial_dm;    /* 1: InitialDM before the outer SK (Alg. 2 preprocessing) */
    int32_t K0;            /* outer SK iterations, >= 0 */
    int32_t K;             /* inner SK iteration cap, >= 0 */
    int32_t sk;            /* pm_sk_policy */
    int32_t dm;            /* pm_dm_policy */
    int32_t precision;     /* pm_precision */
    int32_t local_cap;     /* 0: the Local repair of Eq. 5.  L > 0: a bounded-work variant
                              (Sec. 3.3 leaves its design open; no counterpart in the paper's
                              results): the two-hop expansion skips vertices whose adjacency
                              list in B^(0) (A after the initial DM) holds more than L entries,
                              and the normalisation sum of such
                              a vertex is estimated from a systematic sample of L list positions
                              ((o + q floor(len / L)) mod len, o from a Philox draw of the step)
                              scaled by deg / (live samples).  Scales only shape the proposal,
                              so the estimate stays unbiased. */
    double theta;          /* Thrs / Trck threshold theta_th = theta_tr */
    const struct pm_model* learned;  /* NULL: the scaled proposal of Eq. 3.  Otherwise the
                              learned proposal (no counterpart in the paper): candidate l
                              of v gets score B_vl * e^{f(x_vl)} where f is the model and
                              x_vl the edge features; requires sk = PM_SK_NONE and
                              precision = PM_PREC_FP32_PROPOSAL.  The correction still
                              uses the realised probability, so the estimate stays
                              unbiased. */
    /* Run control (Sec. 4: runs stop at a relative-error target or a time
     * cap).  0 switches each off; both >= 0 and finite.
     *   rse_target     estimate_permanent(_batch) / pm_estimate_batch_ex run
     *                  rounds of trajectories until each matrix's RSE is at
     *                  most rse_target (with at least min(1024, n_traj)
     *                  trajectories and two alive) or its n_traj ran; the
     *                  rounds use consecutive trajectory ids, so n_traj is
     *                  an upper bound.  pm_batch_create rejects it (a
     *                  resident batch runs fixed counts).
     *   time_budget_s  the call starts no trajectory once this much time has
     *                  passed (host clock between rounds, the device clock
     *                  %globaltimer inside a launch); trajectories already
     *                  started run to their end.  If matrices are still
     *                  short of their target or n_traj, the call returns
     *                  PM_ETIMEOUT with the results of what ran.
     * pm_trace, training teachers and pm_server (whose requests carry their
     * own targets) ignore or reject them: the server requires 0. */
    double rse_target;
    double time_budget_s;
} pm_schedule;

/* Why a matrix's run ended (pm_result.stop). */
enum { PM_STOP_COMPLETE = 0,   /* all n_traj trajectories ran */
       PM_STOP_TARGET = 1,     /* RSE reached rse_target */
       PM_STOP_TIME = 2,       /* the time budget ran out */
       PM_STOP_CANCELLED = 3 };

typedef struct {
    double log_estimate;   /* ln(mean X); -INFINITY if every X = 0 */
    double estimate;       /* exp(log_estimate); +INFINITY if it overflows binary64 */
    double ess;            /* (sum X)^2 / sum X^2 (Sec. 2) */
    double p_match;        /* #{X > 0} / M */
    double rel_spread;     /* s_X / |mean X|, s_X with M - 1 (Sec. 3.2) */
    double rse;            /* rel_spread / sqrt(M) (Sec. 4 "Metrics") */
    double log_sum_x;      /* ln sum X    (for merging runs on the host) */
    double log_sum_x2;     /* ln sum X^2 */
    uint64_t n_traj;       /* M */
    uint64_t n_alive;
    uint64_t n_dm_calls;   /* inner DM calls over all trajectories */
    uint64_t n_full_sk;    /* full SK iterations over all trajectories */
    uint64_t n_local_sk;   /* Local repairs over all trajectories */
    double seconds;        /* wall time of the call on the host clock */
    uint64_t alg_bytes;    /* algorithmic bytes the trajectories of this matrix touched
                              (the method's own traffic, whatever the memory level):
                              16 B per vertex at initialisation; per step 8 B per
                              adjacency entry of the picked vertex and of its partner
                              (index + liveness check) and 16 B of list pointers,
                              32 B per degree decrement (read-modify-write + the
                              minimum-degree structure), the scale (4 or 8 B) and value
                              (4 B) per candidate of a scaled / weighted proposal; the
                              learned proposal's features 8 B per adjacency entry of
                              each live candidate + 16 B per candidate; 16 B per live
                              edge per full SK iteration, 16 B per vertex of each Local
                              repair, 16 B per live edge + 48 B per active row per DM */
    double kernel_ms;      /* device time of the trajectory kernel of the call (CUDA events
                              on the context's stream; shared by all matrices of a batch) */
    uint64_t mlp_rows;     /* learned proposal: network evaluations of live candidates
                              (2 * (8*64 + 64*64 + 64) = 9344 multiply-add flops each) */
    uint64_t traj_ns;      /* sum over this matrix's trajectories of their device
                              durations (%globaltimer, start to end); trajectories of a
                              launch overlap, so a matrix's share of the launch's time
                              is its traj_ns over the launch's total */
    double dev_ms;         /* this matrix's share of the trajectory kernels' device time:
                              per launch, the launch's time x traj_ns of this matrix / the
                              launch's total traj_ns; summed over the launches merged */
    uint32_t rounds;       /* trajectory launches the result merges */
    int32_t stop;          /* PM_STOP_* */
} pm_result;

/* Layout of one matrix in a trajectory launch (see pm_batch_create). */
typedef struct {
    int32_t g;               /* warps per trajectory */
    int32_t groups;          /* trajectories in flight per CTA (one CTA per SM) */
    int32_t staged;          /* matrix adjacency staged in shared memory */
    int32_t rc_smem;         /* scaling vectors in shared memory */
    int32_t gstate;          /* trajectory state in global memory (large n) */
    int32_t dm_smem;         /* inner DM's workspace and edge mask in shared memory */
    int32_t tuned;           /* 1 if the autotuner chose this layout */
    int32_t pair;            /* two trajectories per warp, one per 16-lane half (schedules
                                without inner SK or DM; `groups` counts trajectories) */
    double probe_traj_per_s;      /* the chosen layout's probe rate (-1: not probed) */
    double heuristic_traj_per_s;  /* the heuristic layout's probe rate (-1: not probed) */
} pm_plan_info;

/* Bookkeeping of the most recent estimate / trace / batch call of a context. */
typedef struct {
    uint64_t h2d_bytes;       /* host -> device bytes the call copied */
    uint64_t d2h_bytes;       /* device -> host bytes the call copied */
    double traj_kernel_ms;    /* device time of the trajectory kernel */
    double prep_kernel_ms;    /* device time of the preprocessing kernel */
    int32_t grid;             /* CTAs of the trajectory launch */
    int32_t warps_per_cta;    /* warps (trajectory slots) per CTA */
    pm_plan_info first_plan;  /* layout of the call's first matrix (g = 0: no launch;
                                 tuned and the probe rates are not filled in) */
    double grad_kernel_ms;    /* device time of the most recent pm_mlp_gradient's kernels
                                 (residual pass, tensor-core gradient, reduction; 0: none) */
} pm_call_info;

typedef struct pm_context pm_context;

/* Create a context on CUDA device `device` that issues all work on
 * `cuda_stream` (a cudaStream_t; NULL = a new non-blocking stream owned by
 * the context).  Device workspaces are allocated lazily and grown as needed. */
pm_status pm_context_create(pm_context** ctx, int device, void* cuda_stream);
pm_status pm_context_destroy(pm_context* ctx);

/* Ask the context's running estimate call (or resident-batch run) to stop:
 * safe to call from any host thread at any time.  It sets a flag in pinned
 * host memory that the trajectory kernel reads before it starts each chunk
 * of trajectories; started trajectories run to their end, and the call
 * returns PM_ECANCELLED with the results of what ran.  Every estimate call
 * and batch run clears the flag when it starts, so a cancel that arrives
 * between calls is dropped. */
pm_status pm_context_cancel(pm_context* ctx);

/* Merge the results of disjoint trajectory sets of one matrix (other ranks,
 * earlier rounds or resumed runs with other trajectory ids) through their
 * sufficient statistics: M, #alive, ln sum X and ln sum X^2, from which the
 * estimate, ESS, p_match (Sec. 2), relative spread and RSE (Sec. 4
 * "Metrics") follow exactly; operation counts, bytes, times and rounds are
 * summed, stop is the largest.  Host arithmetic only (no device needed).
 * parts[count], count >= 1; out may alias no part. */
pm_status pm_merge_results(const pm_result* parts, int32_t count, pm_result* out);

/* Estimate per(csr) from n_traj trajectories with Philox4x32-10 seed `seed`;
 * trajectory k draws from counter (k, matrix index 0, step, attempt), so any
 * trajectory can be replayed on its own.  n must equal csr->n. */
pm_status estimate_permanent(pm_context* ctx, const pm_csr* csr, int32_t n, uint64_t n_traj,
                             uint64_t seed, const pm_schedule* schedule, pm_result* out);

/* The same for `count` matrices in one persistent launch (matrix k uses
 * matrix index k in the Philox counter, n_traj[k] trajectories); outs[count]. */
pm_status estimate_permanent_batch(pm_context* ctx, const pm_csr* mats, int32_t count,
                                   const uint64_t* n_traj, uint64_t seed,
                                   const pm_schedule* schedule, pm_result* outs);

/* estimate_permanent_batch with two extras: trajectories of matrix k are
 * first_traj .. first_traj + n_traj[k] - 1, and, when log_x is not NULL, the
 * per-trajectory ln X (host buffer of sum_k n_traj[k] doubles, matrix-major,
 * -INFINITY for dead trajectories) is copied out.  Same launch as
 * estimate_permanent_batch. */
pm_status pm_estimate_batch_ex(pm_context* ctx, const pm_csr* mats, int32_t count,
                               const uint64_t* n_traj, uint64_t first_traj, uint64_t seed,
                               const pm_schedule* schedule, pm_result* outs, double* log_x);

/* Replay trajectories first_traj .. first_traj + count - 1 of matrix index
 * `matrix_index` and return their paths (host buffers, any may be NULL):
 *   chosen[count][n][2]  unified ids (v, u) of step t, -1 after death
 *   deg_v[count][n]      live degree of v when it was picked, -1 after death
 *   dead_step[count]     step at which the trajectory died, -1 if it completed
 *   log_x[count]         ln X, -INFINITY for a dead trajectory
 *   logits[count][n][logit_stride]
 *                        learned proposal only: network output of the q-th live
 *                        candidate (adjacency order) of step t, q < logit_stride
 *                        (0 where a step has fewer candidates; a stride of the
 *                        largest row or column length of csr keeps every
 *                        candidate of every step).  logit_stride is ignored when
 *                        logits is NULL, else 1 .. 65535 (PM_EINVAL otherwise).
 * The trajectory kernel runs in the layout the context's autotuner chose for
 * this matrix's size class and schedule (pm_batch_create with
 * PM_BATCH_AUTOTUNE), else in the heuristic layout. */
pm_status pm_trace(pm_context* ctx, const pm_csr* csr, uint32_t matrix_index,
                   uint64_t first_traj, uint32_t count, uint64_t seed,
                   const pm_schedule* schedule, int32_t* chosen, int32_t* deg_v,
                   int32_t* dead_step, double* log_x, float* logits, uint32_t logit_stride);

/* Preprocessing only (InitialDM + K0 outer SK): host outputs, any may be NULL:
 * ok (1 if a perfect matching exists), keep[nnz] (1 = edge survives the
 * initial DM, CSR order of the input), r[n], c[n] (outer scaling, binary64
 * copies of the mode's values). */
pm_status pm_preprocess(pm_context* ctx, const pm_csr* csr, const pm_schedule* schedule,
                        int32_t* ok, uint8_t* keep, double* r, double* c);

/* Philox4x32-10 blocks for `count` consecutive counters starting at ctr
 * (ctr[0] incremented per block), computed on the device (host output
 * out[count][4]); for checking the generator against published vectors. */
pm_status pm_philox_blocks(pm_context* ctx, const uint32_t ctr[4], const uint32_t key[2],
                           uint32_t count, uint32_t* out);

/* Measure the device's on-chip read bandwidth (a diagnostic with no
 * counterpart in the paper; the roofline denominators of traffic that stays
 * on chip): *l2_read_gbs from 200 passes of 16-byte L2-cached reads over a
 * 64 MiB buffer (smaller than L2, so every pass after the first hits L2),
 * *smem_read_gbs from conflict-free 16-byte reads of 96 KiB of shared memory
 * per CTA on two CTAs per SM; GB/s = bytes read / CUDA-event time.
 * Allocates and frees a 64 MiB device buffer. */
pm_status pm_probe_bandwidth(pm_context* ctx, double* l2_read_gbs, double* smem_read_gbs);

/* Copy the bookkeeping of the context's most recent call into *info. */
pm_status pm_last_call_info(const pm_context* ctx, pm_call_info* info);

/* ---- resident batches (no counterpart in the paper) -----------------------
 * A batch is a set of matrices estimated together again and again, each run
 * with a fresh trajectory range: the serving and benchmarking pattern.  It
 * owns device copies of its matrices (taken at creation from host or device
 * CSR; the caller's arrays are not retained) and a workspace sized once.
 * Every run executes the whole path of Algorithm 2 (preprocessing, one
 * persistent trajectory launch over all matrices, statistics) and returns
 * what pm_estimate_batch_ex returns for the same arguments: ln X of every
 * trajectory is identical whatever the layout.
 *   PM_BATCH_GRAPH     the launch sequence is captured once as a CUDA graph;
 *                      a run sets the trajectory kernel's range and seed in
 *                      the instantiated graph and launches it.
 *   PM_BATCH_AUTOTUNE  for each size class (half-octave of n) the layout --
 *                      staging of the matrix in shared memory, placement of
 *                      the trajectory state, warps per trajectory -- is chosen
 *                      by timing every candidate layout on a probe launch of
 *                      the class's largest matrix (fastest trajectories/s);
 *                      with inner DM, also whether the DM workspace and edge
 *                      mask sit in shared memory (fewer trajectories per SM,
 *                      faster DM);
 *                      the choice is cached in the context per class and
 *                      schedule.  Without it a fixed heuristic decides.
 * The context (and a learned model in the schedule) must outlive the batch;
 * runs of one batch must not overlap.  Errors: as pm_estimate_batch_ex;
 * PM_ECUDA if capture or instantiation fails. */
typedef struct pm_batch pm_batch;
enum { PM_BATCH_GRAPH = 1, PM_BATCH_AUTOTUNE = 2 };

pm_status pm_batch_create(pm_context* ctx, const pm_csr* mats, int32_t count,
                          const uint64_t* n_traj, const pm_schedule* schedule, uint32_t flags,
                          pm_batch** out);
/* One run over trajectories first_traj .. first_traj + n_traj[k] - 1 of every
 * matrix k: outs[count] as pm_estimate_batch_ex, log_x (host, may be NULL) the
 * per-trajectory ln X, matrix-major. */
pm_status pm_batch_run(pm_batch* batch, uint64_t first_traj, uint64_t seed, pm_result* outs,
                       double* log_x);
/* The layout matrix k runs with. */
pm_status pm_batch_plan_info(const pm_batch* batch, int32_t k, pm_plan_info* info);

/* Cost-aware choice of the Thrs / Trck threshold (the paper leaves theta's
 * tuning open, Sec. 4): for each of thetas[count], one probe estimate of csr
 * with schedule->theta = thetas[k] on a time budget of probe_s seconds (disjoint
 * trajectory ids per candidate); its score is the work-normalised relative
 * variance RSE^2 x device seconds (scores[k], may be NULL; +INFINITY when fewer
 * than two trajectories stayed alive).  schedule->theta is set to the best
 * candidate (unchanged if none scored).  schedule->dm must be PM_DM_THRS or
 * PM_DM_TRCK; its rse_target and time_budget_s are ignored by the probes. */
pm_status pm_tune_theta(pm_context* ctx, const pm_csr* csr, pm_schedule* schedule, const double* thetas,
                        int32_t count, double probe_s, uint64_t seed, double* scores);

/* Pin the layout (g, staged, rc_smem, gstate, dm_smem, pair of *layout; the other
 * fields are ignored) that every later call of this context uses for
 * matrices of n's size class (half-octave of n) under this schedule, as the
 * autotuner's cached choice does (no counterpart in the paper: for callers who
 * tuned offline, and to run a given layout).  A later autotune of the same
 * class replaces it.  PM_EUNSUPPORTED if the layout does not fit a matrix of
 * order n with nnz entries under this schedule; a matrix of the class that it
 * does not fit runs in the heuristic layout. */
pm_status pm_layout_set(pm_context* ctx, const pm_schedule* schedule, int32_t n, int64_t nnz,
                        const pm_plan_info* layout);
pm_status pm_batch_destroy(pm_batch* batch);

/* ---- serving (no counterpart in the paper) --------------------------------
 * A server estimates a stream of requests, each until its RSE (Sec. 4
 * "Metrics") reaches the request's target or its trajectory budget is spent.
 * pm_server_submit copies a matrix to the device and queues it.  Every
 * pm_server_round
 *   1. admits queued requests first come first served while the device bytes
 *      of the admitted requests stay within cfg.device_budget_bytes (a request
 *      larger than the whole budget is refused) and prepares each once
 *      (InitialDM, outer SK, degrees, tree: Algorithm 2's preprocessing);
 *   2. runs one persistent trajectory launch over all admitted requests,
 *      max(steps_per_round / n, the request's share of the GPU's trajectory
 *      slots) trajectories each (clamped to [traj_min, traj_max] and to what
 *      is left of the request's budget), with ids disjoint from every earlier
 *      round;
 *   3. merges each request's statistics with its earlier rounds and returns
 *      the requests that are finished (target met with at least
 *      min_traj_done trajectories and two alive, budget spent, refused).
 * Times are seconds on the server's clock (pm_server_clock, from creation).
 * The context (and a learned model) must outlive the server. */
typedef struct pm_server pm_server;
enum { PM_REQ_DONE = 0, PM_REQ_BUDGET = 1, PM_REQ_REFUSED = 2, PM_REQ_FAILED = 3 };

typedef struct {
    pm_schedule schedule;         /* estimator of every request */
    uint64_t seed;                /* Philox seed of all rounds */
    uint64_t device_budget_bytes; /* admission limit */
    uint64_t steps_per_round;     /* trajectory steps per request per round (T = steps / n) */
    uint32_t traj_min, traj_max;  /* per request and round; 1 <= traj_min <= traj_max < 2^24 */
    uint64_t min_traj_done;       /* trajectories before the RSE target may end a request */
} pm_server_cfg;

typedef struct {
    uint64_t id;
    int32_t status;               /* PM_REQ_* */
    uint32_t rounds;
    pm_result result;             /* merged over all rounds (seconds, kernel_ms, alg_bytes: 0) */
    double submit_time, done_time;
} pm_request_done;

pm_status pm_server_create(pm_context* ctx, const pm_server_cfg* cfg, pm_server** out);
/* target_rse > 0; max_traj >= 1.  *id identifies the request in later results. */
pm_status pm_server_submit(pm_server* server, const pm_csr* csr, double target_rse, uint64_t max_traj,
                           uint64_t* id);
/* done[cap] (host) receives the finished requests, *n_done of them; n_active,
 * n_queued (may be NULL) the requests still admitted / waiting. */
pm_status pm_server_round(pm_server* server, pm_request_done* done, uint32_t cap, uint32_t* n_done,
                          uint32_t* n_active, uint32_t* n_queued);
double pm_server_clock(const pm_server* server);
pm_status pm_server_destroy(pm_server* server);

/* ---- learned proposal (no counterpart in the paper) ----------------------
 * A small network f: 8 edge features -> 64 -> 64 (GELU) -> 1 predicts
 * ln(r_v c_l), the scale product an SK-scheduled run would use for edge
 * (v, l).  Features of candidate l of the picked vertex v at step t:
 * log1p deg(v), log1p deg(l), log1p of the degree sum over v's live
 * candidates, log1p of the degree sum over l's live neighbours, t / n, ln of
 * the outer scales of v and l, ln B_vl.  Weights are BF16 on the device
 * (FP32 master copy for training); parameter vector layout: W1[64][8], b1[64],
 * W2[64][64], b2[64], W3[64], b3 (4801 floats). */
typedef struct pm_model pm_model;

typedef struct {
    uint64_t n_pairs;        /* (features, target) pairs to train on: whole steps, at most this many */
    uint64_t seed;           /* Philox seed of the teacher trajectories and of the shuffle */
    int32_t epochs;          /* passes over the recorded pairs */
    int32_t batch;           /* rows per Adam step */
    float lr, beta1, beta2, eps;   /* Adam */
    pm_schedule teacher;     /* SK-scheduled estimator producing the targets (sk FIXED or
                                ADAPTIVE, FP32 proposal); its current scales at each step
                                are the targets */
    int32_t objective;       /* PM_OBJ_MSE or PM_OBJ_CENTRED */
    int32_t reserved;        /* must be 0 */
} pm_train_cfg;

/* Training losses over the recorded pairs (e = network output - target):
 * PM_OBJ_MSE      mean of e^2;
 * PM_OBJ_CENTRED  mean of (e - mean of e over the pair's step)^2.  Eq. 3
 *                 normalises the scores of a step, so only the differences of
 *                 a step's logits reach the proposal; this loss ignores the
 *                 part of the target (ln r_v) that all candidates share. */
enum { PM_OBJ_MSE = 0, PM_OBJ_CENTRED = 1 };

typedef struct {
    double loss_first;       /* loss of the first Adam step's batch */
    double loss_last;        /* mean loss over the last epoch */
    uint64_t n_pairs;        /* pairs recorded */
    int32_t steps;           /* Adam steps taken */
    int32_t reserved;
    double seconds_record, seconds_train;
} pm_train_report;

/* Create a model on the context's device: params (host, 4801 floats) or NULL
 * for a seeded random initialisation. */
pm_status pm_model_create(pm_context* ctx, const float* params, uint64_t seed, pm_model** out);
pm_status pm_model_destroy(pm_model* model);
/* Write the FP32 master parameters to `path` (8-byte magic "PMMODEL1",
 * uint32 version 1, uint32 count 4801, the parameters, a 64-bit FNV-1a
 * checksum of their bytes; little-endian), through a temporary file renamed
 * into place.  PM_EINVAL if the file cannot be written. */
pm_status pm_model_save(pm_context* ctx, const pm_model* model, const char* path);
/* Create a model on the context's device from a file written by
 * pm_model_save.  PM_EINVAL for a missing, truncated, foreign or corrupted
 * file (magic, version, count, length and checksum are all checked). */
pm_status pm_model_load(pm_context* ctx, const char* path, pm_model** out);
/* FP32 master parameters (host out, 4801 floats) / replace them. */
pm_status pm_model_get_params(pm_context* ctx, const pm_model* model, float* params);
pm_status pm_model_set_params(pm_context* ctx, pm_model* model, const float* params);
/* Train on pairs recorded from cfg->teacher running on mats[count] (matrix k
 * uses matrix index k): record (one run sized for about 1.5 x n_pairs, into a
 * buffer that cannot overflow), keep whole steps in a fixed order up to
 * n_pairs, shuffle (whole steps for PM_OBJ_CENTRED), then epochs of Adam on
 * cfg->objective, gradients from the tensor-core backward kernel reduced in a
 * fixed order.  The same arguments give bit-identical parameters. */
pm_status pm_model_train(pm_context* ctx, pm_model* model, const pm_csr* mats, int32_t count,
                         const pm_train_cfg* cfg, pm_train_report* report);
/* Network outputs for B feature rows (host X[B][8] -> host out[B]). */
pm_status pm_mlp_forward(pm_context* ctx, const pm_model* model, const float* X, uint64_t B,
                         float* out);
/* Gradient of the training loss over (X[B][8], T[B]) w.r.t. the parameters
 * (host grad[4801]) and the loss, from the training kernel.  group == NULL:
 * PM_OBJ_MSE.  Otherwise PM_OBJ_CENTRED with group[B] (host) = index within
 * the step << 16 | the step's row count, the rows of a step consecutive and
 * complete; codes that do not tile [0, B) that way give PM_EINVAL. */
pm_status pm_mlp_gradient(pm_context* ctx, const pm_model* model, const float* X, const float* T,
                          const uint32_t* group, uint64_t B, float* grad, double* loss);
/* Record (features, target) pairs along trajectories first_traj ..
 * first_traj + count - 1 of `teacher` on one matrix; key = traj << 28 |
 * step << 14 | candidate (live-candidate index).  A pair is kept if all its
 * values are finite; a step's kept pairs are stored consecutively, and only
 * if there are at least two; group (may be NULL) = index within the step's
 * pairs << 16 | their count.  Host outputs of capacity cap (a step that does
 * not fit is dropped, the order of steps is not deterministic); *n_out =
 * pairs stored. */
pm_status pm_record_pairs(pm_context* ctx, const pm_csr* csr, uint32_t matrix_index,
                          uint64_t first_traj, uint32_t count, uint64_t seed,
                          const pm_schedule* teacher, uint64_t cap, float* feat, float* target,
                          uint64_t* key, uint32_t* group, uint64_t* n_out);

/* Statistics of a set of log-weights; fields as in pm_result. */
typedef struct {
    double log_estimate, ess, p_match, rel_spread, rse, log_sum_x, log_sum_x2;
    uint64_t n_traj, n_alive;
} pm_weight_stats;

/* Allocation-free statistics of M log-weights (no counterpart in the paper;
 * a library service).  Some callers cannot allocate device memory when they
 * call in: hosts whose own allocator has reserved the device's memory, and
 * latency-bound loops that cannot take the device-wide synchronisation that
 * cudaMalloc / cudaFree may cause.  This function allocates nothing: its
 * scratch (partial sums, about 50 KB) is a fixed device array that every GPU
 * loading the library holds until the process exits.
 *   log_x  device pointer (current device) to M binary64 ln X values,
 *          -INFINITY for dead trajectories
 *   M      1 .. 2^26; larger M returns PM_EUNSUPPORTED (the scratch holds the
 *          partial sums of at most 2^26 values)
 *   out    device pointer (current device) receiving one pm_weight_stats
 *   cuda_stream  stream the two kernels run on; the call does not
 *          synchronise, out is valid once the stream has reached this point.
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress), so make that first call before any stream capture.
 * Every call shares the same scratch: calls whose kernels overlap on the GPU
 * (other streams, other host threads) race; serialise them.  Errors:
 * PM_EINVAL for NULL pointers or M = 0, PM_ECUDA if a launch fails. */
pm_status pm_log_weight_stats_noalloc(const double* log_x, uint64_t M, pm_weight_stats* out,
                                      void* cuda_stream);

/* Human-readable name of a status, and the last error message of a context. */
const char* pm_status_string(pm_status s);
const char* pm_last_error(const pm_context* ctx);

#ifdef __cplusplus
}
#endif
#endif /* PM_H_ */
