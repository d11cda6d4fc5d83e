/*
 * hjcd.h -- C ABI of the GB300 (sm_103a) batched HJCD-IK library.
 *
 * HJCD-IK (arXiv 2510.07514) solves inverse kinematics for serial revolute
 * chains by running many seeds per target pose through three stages
 * (Sec. V, Alg. 2): an orientation-aware greedy coordinate descent (PO-CCD,
 * Alg. 3), a Jacobian damped-least-squares polish (PJ-IK, Alg. 4) and a
 * sphere-based collision filter (Sec. V-C); the collision-free survivors are
 * ranked by residual.  Every stage runs in this library's own CUDA kernels.
 *
 * Conventions shared by every entry point
 *   - Status: every call returns HJCD_OK (0) or a negative HJCD_E* code and
 *     records a message readable with hjcd_last_error().  Nothing is written
 *     to outputs when a call fails validation.
 *   - Precision: all device arithmetic is IEEE binary32.
 *   - Poses: 7 floats px py pz qw qx qy qz (metres; Hamilton quaternion).
 *     Quaternions are normalised on entry; a zero quaternion is HJCD_EINVAL.
 *   - Joint vectors on the device are structure-of-arrays: joint j of
 *     candidate c lives at theta[j * ld + c] (ld >= number of candidates).
 *   - Ownership: the caller owns every buffer it passes.  Robot and scene
 *     tables are copied into device memory owned by the context when they are
 *     created; later changes to the caller's arrays have no effect.
 *   - Streams: `stream` is a cudaStream_t (NULL = the legacy default stream).
 *     Calls taking device buffers only enqueue work and return before it
 *     completes; hjcd_solve with host buffers returns after its results have
 *     been copied back.
 *   - Threads: a context is used by one host thread at a time; while a
 *     server runs (hjcd_server_start), its scheduler thread launches work on
 *     the same context, and the caller may still submit, poll, wait and
 *     change the launch configuration and collision mode.
 *   - Random draws: Philox4x32-10 keyed by the request seed, counter
 *     (candidate, target, phase << 24 | iteration, block), so results do not
 *     depend on how work is batched.
 */
#ifndef HJCD_H
#define HJCD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t hjcd_status;
#define HJCD_OK 0
#define HJCD_EINVAL (-1)    /* bad argument: size, pointer kind, id, limits */
#define HJCD_ENOMEM (-2)    /* device (or host pinned) allocation failed */
#define HJCD_ECUDA (-3)     /* a CUDA runtime call or kernel launch failed */
#define HJCD_ETIMEOUT (-4)  /* a bounded device wait ran out; results invalid */
#define HJCD_ENOTFOUND (-5) /* unknown robot or scene id */

#define HJCD_MAX_DOF 24        /* joints per chain */
#define HJCD_MAX_SPHERES 256   /* link spheres per robot */
#define HJCD_MAX_SAMPLES 8192  /* seeds per target */
#define HJCD_MAX_TOPK 64
#define HJCD_MAX_BATCH_ROBOTS 16  /* distinct robots in one hjcd_solve_batch call */

typedef struct hjcd_ctx hjcd_ctx;

/* Parameter table of Alg. 2-4 (symbols of the paper in brackets).  Values
 * are readings of the paper, which names them only symbolically. */
typedef struct hjcd_params {
    int32_t cd_max_iters;   /* PO-CCD iteration cap [max_iters] */
    float cd_eps_pos2;      /* PO-CCD coarse break on |e_p|^2, m^2 [epsilon] */
    float cd_eps_ori2;      /* PO-CCD coarse break on |omega|^2, rad^2 [nu] */
    float cd_gamma_pos;     /* acceptance: position improvement, m [gamma] */
    float cd_gamma_ori;     /* acceptance: orientation improvement, rad [gamma] */
    float cd_sigma;         /* std of the PO-CCD rejection perturbation, rad [Sigma] */
    float cd_delta0;        /* annealing delta(k) = delta0 * rho^k (Eq. ori_update) */
    float cd_rho;
    float proj_eps;         /* relative projected length below which Eq. theta_proj gives 0 */
    int32_t dup_ratio;      /* K = max(1, floor(B / dup_ratio)) seeds kept [K] */
    float dup_sigma;        /* std of the duplication perturbation, rad [Sigma] */
    int32_t lm_max_iters;   /* PJ-IK iteration cap [max_iters] */
    float lm_lambda;        /* damping of Eq. normal-eqs [lambda] */
    float lm_trust_R;       /* trust region, rad [R] */
    float lm_beta;          /* line-search ratio [beta] */
    int32_t lm_A;           /* line-search depth [A], 0..31 */
    float lm_sigma;         /* std of the PJ-IK perturbation, rad [Sigma] */
    float lm_gn_reg;        /* regulariser of the minimum-norm Gauss-Newton step (Eq. dogleg) */
    float cd_tie;           /* greedy joint choice: a later joint wins only if its score is lower by this fraction */
    int32_t cd_variant;     /* 0: PO-CCD (Alg. 3), each seed breaking on its own; 1: position-only CCD
                               (Alg. 1: joints n..1, each rotated at once by Eq. theta_proj, break on the
                               squared position error), a baseline; 2: PO-CCD with the target-wide break
                               (all seeds of a target stop after the first iteration that leaves any of
                               them inside the coarse tolerance; whole solves only, not hjcd_po_ccd or
                               hjcd_solve_noalloc) */
} hjcd_params;

typedef struct hjcd_solve_opts {
    float eps_pos;          /* success / PJ-IK break tolerance on |e_p|, m */
    float eps_ori;          /* success / PJ-IK break tolerance on |omega|, rad */
    int32_t n_samples;      /* seeds per target, M = B (Alg. 2); 1..HJCD_MAX_SAMPLES */
    int32_t top_k;          /* ranked solutions returned per target, 1..HJCD_MAX_TOPK */
    uint64_t seed;          /* request seed (Philox key) */
    const hjcd_params* params;           /* NULL => hjcd_default_params() */
    const int32_t* samples_per_target;   /* NULL => n_samples for all; else HOST array [n_targets] */
} hjcd_solve_opts;

/* ---- context -------------------------------------------------------------- */

/* Create a context on CUDA device `device` (made current on this thread). */
hjcd_status hjcd_init(int device, hjcd_ctx** out);
/* Free every device buffer of the context.  NULL is ignored. */
void hjcd_destroy(hjcd_ctx* ctx);
/* Message of the last failed call on this context ("" if none).  The string
 * stays valid until the next call on the context. */
const char* hjcd_last_error(const hjcd_ctx* ctx);
const char* hjcd_status_string(hjcd_status s);
void hjcd_default_params(hjcd_params* out);

/* ---- resident tables -------------------------------------------------------- */

/* Register a serial revolute chain (Eq. fk).  Joint i contributes, in the
 * modified-DH (Craig) convention, Rx(dh_alpha[i]) Tx(dh_a[i])
 * Rz(theta_i + dh_theta_off[i]) Tz(dh_d[i]); `flange` (row-major 4x4 rigid
 * transform) follows joint n.  Limits: q_lo[i] < q_hi[i].
 * Collision model (Sec. V-C): n_spheres spheres; sphere s is attached to
 * body sph_link[s] in 0..n+1 (0 = base, i = the body moved by joint i,
 * n+1 = the flange frame) at sph_xyzr[4s..4s+2] in that body's frame with
 * radius sph_xyzr[4s+3] > 0.  ignore_pairs: (n+2)x(n+2) row-major bytes,
 * nonzero = the body pair is never checked for self-collision (either entry
 * of a pair marks it); NULL ignores exactly the pairs with |i - j| <= 1.
 * All arrays are HOST memory.
 * Returns the new robot id in *robot_id. */
hjcd_status hjcd_create_robot(hjcd_ctx* ctx, int n_dof,
                              const float* dh_a, const float* dh_alpha, const float* dh_d,
                              const float* dh_theta_off, const float flange[16],
                              const float* q_lo, const float* q_hi,
                              int n_spheres, const int32_t* sph_link, const float* sph_xyzr,
                              const uint8_t* ignore_pairs, int32_t* robot_id);

/* Create (scene_id_or_new < 0) or replace an obstacle scene: n_sph spheres
 * (x y z r, r > 0) and n_box axis-aligned boxes (lo xyz, hi xyz, lo <= hi),
 * HOST arrays.  Returns the id in *scene_id. */
hjcd_status hjcd_set_scene(hjcd_ctx* ctx, int32_t scene_id_or_new, int n_sph, const float* sph_xyzr,
                           int n_box, const float* box_lohi, int32_t* scene_id);

/* ---- the whole method (Alg. 2) ------------------------------------------- */

/* Solve n_targets poses (targets_pq, 7 floats each).  Per target: M seeds
 * through PO-CCD, top-K + perturbed duplication to B, PJ-IK, the collision
 * filter (self-collision when the robot has spheres, plus the scene when
 * scene_id >= 0) and the ranking of the collision-free candidates: those within the
 * tolerances first, each group by the score
 * (|e_p|/eps_pos)^2 + (|omega|/eps_ori)^2.
 * Outputs: out_q [n_targets][top_k][n] joint vectors, out_err
 * [n_targets][top_k][2] (|e_p| m, |omega| rad), out_count [n_targets] the
 * number of collision-free solutions written (0..top_k; 0 is not an error).
 * Rows past out_count are NaN.
 * targets_pq and the three outputs may each be host or device pointers
 * (detected per pointer).  With any host output the call synchronises the
 * stream before returning. */
hjcd_status hjcd_solve(hjcd_ctx* ctx, int32_t robot_id, int32_t scene_id, int n_targets,
                       const float* targets_pq, const hjcd_solve_opts* opts,
                       float* out_q, float* out_err, int32_t* out_count, void* stream);

/* One request of a batch.  scene_id >= 0 names a resident scene; with
 * scene_id < 0 the request brings its own obstacles (HOST arrays, copied with
 * the batch): n_inline_spheres x y z r (r > 0) and n_inline_boxes lo xyz,
 * hi xyz (zero of both: no obstacles).  opts as for hjcd_solve; of
 * opts.params only the iteration caps cd_max_iters and lm_max_iters are taken
 * (the other parameters are the batch's). */
typedef struct hjcd_batch_item {
    int32_t robot_id;
    int32_t scene_id;
    int32_t n_inline_spheres;
    int32_t n_inline_boxes;
    const float* inline_spheres;
    const float* inline_boxes;
    int32_t n_targets;
    int32_t pad_;
    const float* targets_pq;
    hjcd_solve_opts opts;
    float* out_q;
    float* out_err;
    int32_t* out_count;
    const float* q_current;  /* NULL, or [n_targets][n] (host or device): rank as hjcd_solve_nearest */
} hjcd_batch_item;

/* Alg. 2 for several requests at once -- different robots (at most
 * HJCD_MAX_BATCH_ROBOTS distinct), scenes, seed counts, tolerances, top_k and
 * iteration caps -- packed into one launch per phase.  Every request's
 * results are those hjcd_solve gives it alone with the same parameters: each
 * target row keys its random streams by its request's seed and its index
 * inside the request.  Outputs per item as for hjcd_solve; with any host
 * output the call synchronises the stream. */
hjcd_status hjcd_solve_batch(hjcd_ctx* ctx, int n_items, const hjcd_batch_item* items,
                             const hjcd_params* params, void* stream);

/* ---- a batch captured as a CUDA graph ----------------------------------------- */

/* A fixed batch (robots, scenes, seed counts, tolerances, seeds, top_k and
 * caps as in hjcd_solve_batch) captured once, with its own workspace, as one
 * CUDA graph of the whole launch sequence; each hjcd_graph_launch replays it
 * on `stream`, reading the targets from the items' buffers at replay time and
 * writing their outputs, so a control loop that re-solves new poses of the
 * same shape pays no planning or launch overhead.  Targets and outputs must be
 * DEVICE buffers that stay valid for the graph's life; the inline obstacles
 * and seed-count arrays are copied at creation.  Replays of one graph must not
 * overlap in time (they share the workspace).  The paper has no counterpart. */
typedef struct hjcd_graph hjcd_graph;
hjcd_status hjcd_graph_create(hjcd_ctx* ctx, int n_items, const hjcd_batch_item* items,
                              const hjcd_params* params, hjcd_graph** out);
hjcd_status hjcd_graph_launch(hjcd_graph* graph, void* stream);
/* Wait for the last replay and report a bounded device wait that ran out. */
hjcd_status hjcd_graph_check(hjcd_graph* graph);
void hjcd_graph_destroy(hjcd_graph* graph);

/* ---- launch configuration and autotuning --------------------------------------- */

/* Candidates per CTA of the PO-CCD kernel (64, 128 or 256; default 64) and
 * warps per CTA of the PJ-IK kernel (2, 4 or 8; default 8; a PJ-IK launch of
 * at most 64 candidates per SM always takes 2) for every later launch of the
 * context.  Results do not depend on them. */
hjcd_status hjcd_set_launch_config(hjcd_ctx* ctx, int32_t ccd_block, int32_t lm_warps);

typedef struct hjcd_tune_report {
    int32_t ccd_block, lm_warps;        /* launch configuration picked (now set on the context) */
    int32_t cd_max_iters, lm_max_iters; /* iteration caps picked (in *tuned) */
    float success_rate;                 /* of the picked caps on the calibration batch */
    float best_success_rate;            /* best rate of any swept caps */
    double ms;                          /* median time of the calibration batch with the picks */
    int32_t trials;                     /* configurations timed */
} hjcd_tune_report;

/* Autotune on a calibration batch (items as for hjcd_solve_batch; their
 * outputs are not written, top_k is taken as 1).  First every launch
 * configuration is timed and the fastest set on the context; then PO-CCD
 * sweep counts {8, 12, 16, 24, 32, 48} x PJ-IK caps {8, 12, 16, 20, 30} are
 * timed and the fastest pair whose success rate is within success_tol of the
 * best swept rate goes to *tuned (base, or the defaults, with those caps).
 * Each configuration: one warm-up and the median of `repeats` (0: 3) solves.
 * The paper tunes nothing; it states its iteration caps as parameters. */
hjcd_status hjcd_autotune(hjcd_ctx* ctx, int n_items, const hjcd_batch_item* items, const hjcd_params* base,
                          float success_tol, int32_t repeats, hjcd_params* tuned, hjcd_tune_report* report);

/* ---- the seeds of a target sharded across devices -------------------------------- */

/* Alg. 2 with each target's M = opts->n_samples seeds split across devices
 * (one exchange step; the paper runs one device).  Each device runs PO-CCD on
 * seeds [seed_begin, seed_end) of every target (random streams keyed by the
 * global seed index) and keeps its K = max(1, floor(M / dup_ratio)) best:
 * hjcd_shard_topk writes, per target, scores [T][K], seed indices [T][K] (-1
 * past its seeds) and joint vectors [T][K][n], best first.  The lists of all
 * shards, gathered in any order, are merged by hjcd_topk_merge (input
 * [L][T][K] and [L][T][K][n]; output the K best per target, ties to the lower
 * seed index).  hjcd_solve_from_topk runs the rest of Alg. 2 from the merged
 * joint vectors [T][K][n] (duplication, PJ-IK, collision filter, ranking)
 * for targets_pq[0 .. n_targets), which are targets first_target ..
 * first_target + n_targets - 1 of the request (their indices key the random
 * streams, so each device may polish any consecutive range of the targets):
 * the results equal hjcd_solve's on the same targets and options, bit for bit.
 * All arrays are DEVICE memory; targets and options must be the same on every
 * device; opts->samples_per_target must be NULL; cd_variant 2 is refused. */
hjcd_status hjcd_shard_topk(hjcd_ctx* ctx, int32_t robot_id, int n_targets, const float* targets_pq,
                            const hjcd_solve_opts* opts, int32_t seed_begin, int32_t seed_end,
                            float* out_score, int32_t* out_index, float* out_theta, void* stream);
hjcd_status hjcd_topk_merge(hjcd_ctx* ctx, int n_targets, int n_lists, int K, int n, const float* in_score,
                            const int32_t* in_index, const float* in_theta, float* out_score,
                            int32_t* out_index, float* out_theta, void* stream);
hjcd_status hjcd_solve_from_topk(hjcd_ctx* ctx, int32_t robot_id, int32_t scene_id, int n_targets,
                                 const float* targets_pq, int32_t first_target, const hjcd_solve_opts* opts,
                                 const float* kept_theta, float* out_q, float* out_err, int32_t* out_count,
                                 void* stream);

/* ---- serving: continuous batching ------------------------------------------ */

/* Serving loop of a context (Sec. I and Sec. VI motivate interactive use; the
 * paper has no serving layer).  One scheduler thread packs the pending
 * requests, in arrival order, into batches (one launch per phase, as
 * hjcd_solve_batch) and runs each batch on one of max_inflight streams as
 * soon as one is free: requests arriving while others run are admitted as
 * streams and memory free up, and their work overlaps on the device.  A
 * batch holds at most max_batch_requests requests, max_batch_seeds PO-CCD
 * seeds and memory_budget / max_inflight bytes of device workspace; a request
 * that does not fit that share alone fails with HJCD_ENOMEM.  Zero fields take
 * the defaults (2 streams, 256 requests, 2^20 seeds, a quarter of the free
 * device memory).  params: the batch parameters (NULL: defaults); a request's
 * own opts.params contributes its iteration caps.  With max_inflight = 1 and
 * max_batch_requests = 1 the loop is the plain one-request-per-launch path. */
typedef struct hjcd_server_opts {
    int32_t max_inflight;
    int32_t max_batch_requests;
    int64_t max_batch_seeds;
    uint64_t memory_budget;
    const hjcd_params* params;
} hjcd_server_opts;

/* Outcome and timing of a finished request (host steady clock). */
typedef struct hjcd_request_info {
    hjcd_status status;        /* HJCD_OK, or why the request failed */
    int32_t batch_requests;    /* requests in the batch it ran in */
    double queued_ms;          /* submit -> launch of its batch */
    double total_ms;           /* submit -> results in the caller's buffers */
} hjcd_request_info;

hjcd_status hjcd_server_start(hjcd_ctx* ctx, const hjcd_server_opts* opts);
/* Finish every submitted request, then stop (hjcd_destroy does the same). */
hjcd_status hjcd_server_stop(hjcd_ctx* ctx);
/* Queue one request (fields as for hjcd_solve_batch; targets, outputs HOST
 * memory).  The inputs are copied before the call returns; the outputs must
 * stay valid until the request is reported done.  *request_id identifies it. */
hjcd_status hjcd_submit(hjcd_ctx* ctx, const hjcd_batch_item* req, int64_t* request_id);
/* *done = 1 once the request's results are in its buffers (info, if not NULL,
 * then filled); a finished request is reported once, after which its id is
 * unknown. */
hjcd_status hjcd_poll(hjcd_ctx* ctx, int64_t request_id, int32_t* done, hjcd_request_info* info);
/* Block until the request is done (HJCD_ETIMEOUT after timeout_s seconds). */
hjcd_status hjcd_wait(hjcd_ctx* ctx, int64_t request_id, double timeout_s, hjcd_request_info* info);

/* How the whole-method entry points apply the collision filter (Alg. 2):
 * 1 (default), in rank order -- each target's candidates are sorted by score
 * first and checked in that order until top_k collision-free ones are found,
 * which returns exactly the top_k of filtering every candidate; 0, every
 * polished candidate is checked, then the survivors are ranked.  Results are
 * identical; the work counters differ. */
hjcd_status hjcd_set_collision_mode(hjcd_ctx* ctx, int32_t mode);

/* Device workspace one hjcd_solve / hjcd_solve_batch call may use (0, the
 * default: unlimited).  A call needing more runs in waves: each request's
 * targets are cut into consecutive chunks whose seeds fit the budget, run one
 * after another through the same workspace; results equal one whole solve
 * (each chunk keeps its targets' indices inside the request). */
hjcd_status hjcd_set_memory_budget(hjcd_ctx* ctx, uint64_t bytes);

/* hjcd_solve for tracking (the paper's real-time use moves the arm toward the
 * returned solution nearest its current configuration): the collision-free
 * solutions within the request's tolerances come first, ordered by squared
 * joint-space distance to q_current[t] ([n_targets][n], host or device),
 * then the other collision-free candidates by score.  Everything else as for
 * hjcd_solve. */
hjcd_status hjcd_solve_nearest(hjcd_ctx* ctx, int32_t robot_id, int32_t scene_id, int n_targets,
                               const float* targets_pq, const float* q_current, const hjcd_solve_opts* opts,
                               float* out_q, float* out_err, int32_t* out_count, void* stream);

/* ---- the whole method without allocation ------------------------------------- */

/* Bytes of the file-scope device array that serves as the scratch of
 * hjcd_solve_noalloc.  A call needs 64 T + 16 (T + 1) + 12 for the targets,
 * offsets and flags, plus (4 n + 4) M + (4 n + 13) B bytes and a little
 * alignment for T targets of M seeds (B per hjcd_topk_dup, B = M for the
 * default ratio) and n joints: about 200k candidates of a 7-joint arm. */
#define HJCD_NOALLOC_SCRATCH_BYTES (16u << 20)

/* hjcd_solve for callers that cannot allocate device memory while they run:
 * real-time control loops whose latency budget rules out cudaMalloc (it may
 * block until the device is idle), and processes whose device memory belongs
 * to another allocator.  The paper has no counterpart.
 * Same arguments and results as hjcd_solve, with these differences:
 *   - targets_pq, out_q, out_err and out_count must be DEVICE pointers, and
 *     opts->samples_per_target must be NULL (every target uses n_samples);
 *   - the scratch is one file-scope device array of
 *     HJCD_NOALLOC_SCRATCH_BYTES that every GPU loading this library holds
 *     until the process exits; a call needing more returns HJCD_EINVAL;
 *   - the call allocates nothing (no cudaMalloc, cudaFree, pinned or pooled
 *     memory): it only enqueues work on `stream` and returns;
 *   - every call shares that array and finds the previous call's contents in
 *     it (what must start at zero is cleared on the stream), so calls that
 *     overlap on the GPU -- on different streams, or from several contexts --
 *     race and corrupt each other's results;
 *   - the first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current and keeps it for the
 *     life of the process; make that first call before any stream capture
 *     begins, and make no call on a device after cudaDeviceReset there (the
 *     kept address then refers to a module that is gone);
 *   - rows past out_count are NaN, as hjcd_solve leaves them;
 *   - work counters are not updated, and a staging wait of the collision
 *     kernel that runs out is not reported (the call does not synchronise):
 *     the candidates of a collision CTA that gave up count as colliding, so
 *     such a call returns fewer solutions, never a colliding one. */
hjcd_status hjcd_solve_noalloc(hjcd_ctx* ctx, int32_t robot_id, int32_t scene_id, int n_targets,
                               const float* targets_pq, const hjcd_solve_opts* opts,
                               float* out_q, float* out_err, int32_t* out_count, void* stream);

/* ---- stages (device buffers only) -------------------------------------------
 * Candidates are described by `tgt[c]` (row of `targets_pq`) and `cand[c]`
 * (index of the candidate inside its target, which keys its random streams).
 * All pointers below are DEVICE pointers. */

/* Eq. fk: flange pose of each candidate. */
hjcd_status hjcd_fk(hjcd_ctx* ctx, int32_t robot_id, int64_t n_cand, const float* theta, int64_t ld,
                    float* out_pq, void* stream);

/* Alg. 3, seeding: seeds uniform inside the limits. */
hjcd_status hjcd_sample_seeds(hjcd_ctx* ctx, int32_t robot_id, int64_t n_cand, const int32_t* tgt,
                              const int32_t* cand, uint64_t seed, float* theta, int64_t ld, void* stream);

/* Alg. 3: PO-CCD on each candidate.  theta_in == NULL samples the seeds
 * (its seeding step); otherwise iterations k0 .. k0+n_iters-1 start from theta_in.
 * theta_out may equal theta_in.  score/perr/oerr/iters (each may be NULL)
 * receive the final score, |e_p|, |omega| and iterations executed.
 * Trace (one iteration, n_iters == 1; any pointer may be NULL):
 * dp/rp/op, dq/pq/rq and th_hat are [n][ld]: per joint the position step
 * and the |e_p| and |omega| it leaves, the orientation step and the |e_p| and
 * |omega| it leaves, and the proposed theta_hat; jp/jo the greedy joints
 * (argmin of the score (|e_p|/eps_pos)^2 + (|omega|/eps_ori)^2 over the
 * trials of each kind, a later joint winning only when lower by more than the
 * fraction cd_tie), accepted the acceptance flag. */
typedef struct hjcd_ccd_trace {
    float* dp;
    float* rp;
    float* dq;
    float* rq;
    int32_t* jp;
    int32_t* jo;
    uint8_t* accepted;
    float* th_hat;
    float* op;
    float* pq;
} hjcd_ccd_trace;
hjcd_status hjcd_po_ccd(hjcd_ctx* ctx, int32_t robot_id, int n_targets, const float* targets_pq,
                        float eps_pos, float eps_ori, uint64_t seed, const hjcd_params* params,
                        int64_t n_cand, const int32_t* tgt, const int32_t* cand,
                        const float* theta_in, float* theta_out, int64_t ld, int k0, int n_iters,
                        float* score, float* perr, float* oerr, int32_t* iters,
                        const hjcd_ccd_trace* trace, void* stream);

/* Alg. 2, top-K and duplication, for each target t: the K = max(1, floor(M_t/ratio))
 * lowest scores among its M_t = m_off[t+1]-m_off[t] seeds (ties to the lower
 * index), each copied floor(M_t/K) times with N(0, dup_sigma^2) noise, copy r
 * of kept seed i landing at b_off[t] + r*K + i.  m_off/b_off: [n_targets+1]
 * int64 device arrays (b_off must follow that layout).  src_B (may be NULL)
 * receives the source seed index inside the target. */
hjcd_status hjcd_topk_dup(hjcd_ctx* ctx, int32_t robot_id, int n_targets, const int64_t* m_off,
                          const float* score_M, const float* theta_M, int64_t ld_M,
                          const int64_t* b_off, float* theta_B, int64_t ld_B, int32_t* src_B,
                          uint64_t seed, const hjcd_params* params, void* stream);

/* Alg. 4: PJ-IK, iterations k0 .. k0+n_iters-1, theta updated in place.
 * Trace (one iteration): J [6n][ld] (row r, joint i at (r*n+i)*ld + c),
 * W [6][ld], d_lm [n][ld] the clamped LM step, branch (0 LM, 1 dogleg,
 * 2 single-coordinate, 3 perturbation), alpha the accepted line-search step
 * (0 for the dogleg and the perturbation).  For the candidates whose full LM
 * step failed (left untouched for the others): d_dog [n][ld] the dogleg step
 * of Eq. dogleg, sc_joint the joint i* of Eq. single-coord (largest |g_i| of
 * g = (WJ)^T W r, ties to the lower joint) and sc_step its clamped 1-D
 * Gauss-Newton step g_i* / |(WJ)_i*|^2. */
typedef struct hjcd_lm_trace {
    float* J;
    float* W;
    float* d_lm;
    int32_t* branch;
    float* alpha;
    float* d_dog;
    int32_t* sc_joint;
    float* sc_step;
} hjcd_lm_trace;
hjcd_status hjcd_pjik(hjcd_ctx* ctx, int32_t robot_id, int n_targets, const float* targets_pq,
                      float eps_pos, float eps_ori, uint64_t seed, const hjcd_params* params,
                      int64_t n_cand, const int32_t* tgt, const int32_t* cand,
                      float* theta, int64_t ld, int k0, int n_iters,
                      float* score, float* perr, float* oerr, int32_t* iters,
                      const hjcd_lm_trace* trace, void* stream);

/* Sec. V-C: hit[c] = 1 when candidate c overlaps itself (non-ignored body
 * pairs) or the scene (scene_id < 0: self-collision only).  Overlap of two
 * spheres: |c1-c2|^2 < (r1+r2)^2; of a sphere and a box: squared distance of
 * the centre to the box below r^2. */
hjcd_status hjcd_collide(hjcd_ctx* ctx, int32_t robot_id, int32_t scene_id, int64_t n_cand,
                         const float* theta, int64_t ld, uint8_t* hit, void* stream);

/* Sec. V-C spheres against a whole scene: touched[o] = 1 for every obstacle o
 * of scene scene_id (its spheres in the order given to hjcd_set_scene, then
 * its boxes) that overlaps a link sphere of one of the n_cand configurations
 * theta [n][ld] (device), else 0.  touched: DEVICE array of n_sph + n_box
 * bytes.  Serves to carve obstacle fields around reachable configurations. */
hjcd_status hjcd_scene_contacts(hjcd_ctx* ctx, int32_t robot_id, int32_t scene_id, int64_t n_cand,
                                const float* theta, int64_t ld, uint8_t* touched, void* stream);

/* Alg. 2, final ranking: per target, the collision-free candidates (hit may be
 * NULL) of b_off[t] .. b_off[t+1]-1, those within the tolerances
 * (perr <= eps_pos and oerr <= eps_ori) first, each group by score (ties to
 * the lower index); the first top_k written as in hjcd_solve (rows past
 * out_count NaN).  With q_ref ([n_targets][n] device, or NULL) the group within
 * the tolerances is ordered by squared joint distance to q_ref[t] instead, as
 * hjcd_solve_nearest ranks. */
hjcd_status hjcd_rank(hjcd_ctx* ctx, int32_t robot_id, int n_targets, const int64_t* b_off,
                      const float* theta_B, int64_t ld, const float* score, const float* perr,
                      const float* oerr, const uint8_t* hit, float eps_pos, float eps_ori,
                      const float* q_ref, int top_k,
                      float* out_q, float* out_err, int32_t* out_count, void* stream);

/* Philox4x32-10 (Salmon et al., SC'11), the generator of every random draw
 * of the method (seeds of Alg. 3, perturbations of Alg. 2-4): out[i] = the
 * four 32-bit words of the block at counter ctr[i] (four words) under the key
 * (key & 0xffffffff, key >> 32), computed by the kernels' own generator.
 * ctr and out: DEVICE arrays of n_blocks x 4 uint32. */
hjcd_status hjcd_philox(hjcd_ctx* ctx, int64_t n_blocks, const uint32_t* ctr, uint64_t key, uint32_t* out,
                        void* stream);

/* ---- instrumentation ------------------------------------------------------ */

/* Polls of the collision kernels' first wait for their bulk-copied obstacle
 * tables, for later launches of the context's hjcd_collide, hjcd_solve,
 * hjcd_solve_batch, graph and serving calls (polls < 0: the default 2^22, far
 * longer than any copy takes; hjcd_solve_noalloc and hjcd_solve_from_topk
 * always take the default).  0 makes that wait run out at once, which
 * exercises the timeout path (Sec. V-C has none; a bounded wait is this
 * library's): the kernel sets its error flag, waits for its copy to land with
 * the full limit, returns without verdicts, and the call reports
 * HJCD_ETIMEOUT (hjcd_collide through hjcd_counters).  For tests only. */
hjcd_status hjcd_set_wait_limit(hjcd_ctx* ctx, int64_t polls);

/* Record CUDA events around each phase of hjcd_solve (0 = off). */
hjcd_status hjcd_set_profiling(hjcd_ctx* ctx, int on);
/* Milliseconds of the phases of the last profiled hjcd_solve: [0] PO-CCD,
 * [1] top-K/dup, [2] PJ-IK, [3] collision, [4] rank, [5] whole call on the
 * device.  Synchronises with that call's events. */
hjcd_status hjcd_phase_times(hjcd_ctx* ctx, float ms[6]);
/* Work counters accumulated by the kernels since the last reset:
 * [0] PO-CCD iterations, [1] PJ-IK iterations, [2] forward-kinematics passes
 * inside PJ-IK (frames, full-step, line-search and dogleg trials, counted as
 * the sequential method takes them), [3] sphere-sphere tests executed by the
 * collision kernel (self pairs and obstacle spheres), [4] candidates checked
 * for collision, [5] PO-CCD candidates, [6] sphere-box tests, [7] PJ-IK
 * single-coordinate trials (evaluated in closed form, without a kinematics
 * pass).  Synchronises the device; ETIMEOUT when a bounded device wait ran
 * out since the context was created. */
hjcd_status hjcd_counters(hjcd_ctx* ctx, uint64_t out[8], int reset);
/* Kernel launches issued by this context since creation. */
int64_t hjcd_launch_count(const hjcd_ctx* ctx);
/* FP32 FMA throughput probe: runs a dependent-chain FFMA kernel over every SM
 * for `iters` inner iterations and returns the achieved FP32 TFLOP/s (an FMA
 * counts 2) in *tflops. */
hjcd_status hjcd_ffma_probe(hjcd_ctx* ctx, int iters, double* tflops, void* stream);

#ifdef __cplusplus
}
#endif
#endif
