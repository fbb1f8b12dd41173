/*
 * fmdp — GB300-native FastMDP first-come-first-served flight-plan scheduler.
 *
 * C ABI of libfmdp.so. Plain C types only; every pointer argument is a HOST pointer
 * owned by the caller and is copied in or out before the call returns (except where
 * a function says otherwise). Device memory is owned by the library.
 *
 * The method is the paper's (Bertram, Zambreno, Wei, "Scalable FastMDP for
 * Pre-departure Airspace Reservation and Strategic De-conflict", arXiv 2008.03518):
 *   - a request (origin, destination, departure) is planned by the FastMDP greedy
 *     rollout: at every step each action's successor state is scored with the
 *     closed-form value of Alg. 1 (goal peak minus the aggregate of risk wells of
 *     every known plan, Table 3, minus the hard-deck penalty) and the argmax action
 *     is taken (Alg. 1, Alg. 3-9);
 *   - the finished trajectory is checked for loss of separation against every known
 *     plan and for terrain collision, and is stored as a known plan only if it is
 *     conflict free (Sec. I and Sec. V, first-come-first-served).
 *
 * Conventions:
 *   - every function returns an fmdp_status; no C++ exception crosses the ABI;
 *   - a rejected plan is NOT an error: it returns FMDP_OK with verdict != ADMITTED;
 *   - on error, fmdp_last_error(ctx) returns a message (valid until the next call);
 *   - a context is used by one host thread at a time;
 *   - time is in integer steps of airspace.dt seconds; positions are metres.
 */
#ifndef FMDP_H
#define FMDP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fmdp_ctx fmdp_ctx; /* opaque, library-owned */

typedef int32_t fmdp_status;
#define FMDP_OK 0
#define FMDP_ERR_ARG (-1)     /* invalid argument (null pointer, bad size, non-finite value) */
#define FMDP_ERR_OOM (-2)     /* device or host allocation failed */
#define FMDP_ERR_CUDA (-3)    /* a CUDA call failed; the context should be destroyed */
#define FMDP_ERR_TIMEOUT (-4) /* a bounded device wait ran out; results of the call are void */
#define FMDP_ERR_FULL (-5)    /* no free plan slot */
#define FMDP_ERR_RANGE (-6)   /* time steps outside the table's sliding window */
#define FMDP_ERR_NOTFOUND (-7)
#define FMDP_ERR_IO (-8)      /* a file could not be read or written, or is not a plan file */

/* Verdicts of a planning request (Sec. V: only a collision-free trajectory is accepted). */
#define FMDP_ADMITTED 0
#define FMDP_REJ_CONFLICT 1  /* loss of separation with a known plan at some step */
#define FMDP_REJ_TERRAIN 2   /* a trajectory sample below the terrain surface */
#define FMDP_REJ_HORIZON 3   /* goal not captured within the request's horizon */
#define FMDP_REJ_NO_ACTION 4 /* every successor left the airspace box */

/* Airspace: box, step, plan-table geometry, terrain (Table 3 terrain peaks as static
 * wells and/or a heightmap with a hard-deck clearance penalty, Alg. 1). */
typedef struct {
    double x0, y0, z0, x1, y1, z1; /* box (m); successors outside it are invalid */
    double dt;                     /* step length (s) */
    int32_t n_slices_window;       /* time steps held in the device plan table (ring) */
    int32_t max_slots;             /* concurrent known plans the table can hold */
    const float* heightmap;        /* [hm_ny][hm_nx] node heights over the box, or NULL */
    int32_t hm_nx, hm_ny;
    double clearance_m;            /* clearance below which the hard-deck penalty applies */
    double deck_value;             /* penalty = deck_value - clearance (paper: 1000) */
    const double* static_wells;    /* [n][6] x, y, z, R, |r|, gamma (restricted volumes) */
    int32_t n_static_wells;        /* <= 64 */
} fmdp_airspace;

/* One action: heading change (a multiple of 15 degrees, |.| <= 180) and climb rate. */
typedef struct {
    double dpsi_deg, climb_mps;
} fmdp_action;

/* Separation minima: conflict iff horizontal distance < horiz_m AND |dz| < vert_m. */
typedef struct {
    double horiz_m, vert_m;
} fmdp_sep;

/* A risk well attached to every known plan, centred at p + tau * v (Table 3). */
typedef struct {
    double tau_s, radius_m, magnitude, gamma;
} fmdp_well;

typedef struct {
    int32_t combine;          /* 0: max over negative peaks (paper, Alg. 5-8); 1: sum */
    const fmdp_well* wells;   /* NULL: the paper's five wells (Table 3) */
    int32_t n_wells;          /* <= 8 */
    double goal_reward;       /* |r| of the goal peak (Table 3: 200) */
    int32_t lookahead_W;      /* lookahead window W (Sec. IV "Forward project", Alg. 9): each
                                 action is held for W steps of dt and valued by the largest
                                 value along them; the state advances one step. 0 or 1: the
                                 one-step rule; at most 16. With W > 1, fmdp_schedule_batch and
                                 staged batches run speculative waves of lookahead rollouts
                                 (one CTA per request), the influence test covering the W
                                 steps ahead; results equal planning one request at a time.
                                 fmdp_serve, the learned proposal, departure candidates and the
                                 autotuner require W = 1. */
    int32_t cluster_size;     /* CTAs cooperating on one rollout (0 = automatic) */
    int32_t threads_per_cta;  /* 0 = automatic; else a multiple of 32 in [128, 384] */
    int32_t batch_size;       /* fmdp_schedule_batch: requests per speculative batch
                                 (0 = 256; at most 1024) */
    int32_t full_scan;        /* 1: rollouts scan every slot of each step (no spatial index);
                                 0: they read the plans near the state from the index. Same
                                 results either way. */
    double index_vmax_mps;    /* index: plans faster than this (m/s) are scanned at every
                                 step (0 = 50) */
    double index_cell_m;      /* index: cell edge in metres (0 = automatic) */
    int32_t index_stage_items; /* index: plan samples a rollout step stages in shared memory
                                  (0 = 1536; more are read from global memory) */
    int32_t batch_mode;       /* fmdp_schedule_batch, staged batches and fmdp_serve:
                                 0 = pipelined where it applies (spatial index, W = 1, FastMDP
                                 rollouts): continuous batching without waves, see
                                 fmdp_schedule_batch; 1 = speculative waves. Same results. */
    int32_t pipe_rebuild_items; /* pipelined mode: items appended to one index row before the
                                   rows are rebuilt while no rollout runs (0 = 768). Fewer
                                   keep each step's scan of appended items short; more make
                                   rebuilds rarer. Same results. */
} fmdp_options;

/* Fills *o with the defaults (max combine, Table 3 wells, goal 200, W = 1, automatic). */
void fmdp_options_default(fmdp_options* o);

/* Creates a scheduler on the current CUDA device. gamma: MDP discount, used as the decay
 * of the goal peak (Sec. III: positive peaks share the MDP's discount). actions: up to 32,
 * index order = tie-break order (lowest index wins). Copies every input. */
fmdp_status fmdp_create(const fmdp_airspace* airspace, double gamma, const fmdp_action* actions,
                        int32_t n_actions, const fmdp_sep* sep, const fmdp_options* options,
                        fmdp_ctx** out);
void fmdp_destroy(fmdp_ctx* ctx);
const char* fmdp_last_error(fmdp_ctx* ctx);

/* Uses the caller's CUDA stream (a cudaStream_t passed as void*) for all device work; NULL
 * selects the library's own stream. Calls remain synchronous with respect to the host. */
fmdp_status fmdp_set_stream(fmdp_ctx* ctx, void* stream);

/* Stores a known plan without any conflict check (Sec. V: plans may come from an external
 * source): n fp32 (x,y,z) points, point k at step t0_step + k. The points must lie within
 * the table window. */
fmdp_status fmdp_add_plan(fmdp_ctx* ctx, int64_t t0_step, const float* xyz, int32_t n,
                          uint64_t* plan_id_out);
/* Bulk form: n_plans plans, counts[i] points each, concatenated in xyz. ids_out may be NULL. */
fmdp_status fmdp_add_plans(fmdp_ctx* ctx, int32_t n_plans, const int64_t* t0_steps,
                           const int32_t* counts, const float* xyz, uint64_t* ids_out);

typedef struct {
    uint64_t req_id;
    double ox, oy, oz;   /* origin (m) */
    double gx, gy, gz;   /* destination (m) */
    double speed_mps;    /* horizontal speed (> 0) */
    int64_t depart_step; /* time step at the origin */
    int32_t horizon;     /* maximum number of steps */
    int32_t reserved;
} fmdp_request;

typedef struct {
    int32_t verdict;             /* FMDP_ADMITTED or FMDP_REJ_* */
    int32_t n_points;            /* trajectory samples including the origin */
    uint64_t plan_id;            /* id of the stored plan if admitted, else 0 */
    int32_t first_conflict_step; /* index of the first sample in conflict, -1 if none */
    int32_t first_terrain_step;  /* index of the first sample below terrain, -1 if none */
    double min_sep_h;            /* min horizontal distance to a plan within vert_m (inf if none) */
    double min_sep_v;            /* min |dz| to a plan within horiz_m (inf if none) */
    int32_t near_ties;           /* steps whose top-2 action values differed by < 1e-4 rel. */
    int32_t replanned;           /* batch mode: times the speculative plan was redone */
    int32_t source;              /* 0: FastMDP rollout; 1: accepted learned proposal */
    int32_t reserved;
    float* xyz;                  /* caller-owned [horizon+1][3] or NULL: trajectory samples */
    uint8_t* actions;            /* caller-owned [horizon] or NULL: chosen action indices */
} fmdp_result;

/* Plans one request against every stored plan and admits it if conflict free. */
fmdp_status fmdp_schedule(fmdp_ctx* ctx, const fmdp_request* req, fmdp_result* res);
/* n requests in first-come-first-served (array) order; results identical to n calls of
 * fmdp_schedule. The whole sequence is enqueued on the device without host round trips. */
fmdp_status fmdp_schedule_many(fmdp_ctx* ctx, const fmdp_request* reqs, int32_t n,
                               fmdp_result* res);
/* Batched speculative FCFS (no counterpart in the paper, which plans requests one at a
 * time, Sec. V). Pipelined mode (options.batch_mode = 0, with the spatial index and W = 1):
 * one persistent rollout launch takes requests from a ring in host-mapped memory that the
 * host keeps filling, up to options.batch_size requests past the first unresolved one;
 * each finished plan is reported to host-mapped memory. The requests just behind the
 * first unresolved one publish their current plans in the index as tentative plans, which
 * only later requests see (the guess that they are admitted as planned). The host walks
 * the requests in array order: a request is final when no change of an earlier request's
 * contribution that its plan could not have seen (a tentative plan published or
 * withdrawn, an admission) can reach one of its successor states with a well or come
 * within the separation minima of it; an admitted request is stored at once (beside the
 * running rollouts, its index entries published only when complete), and a plan that a
 * change influences is planned again, from the first step it can alter, as soon as the
 * change is visible. Index rows whose appended lists pass options.pipe_rebuild_items are
 * rebuilt while no rollout runs. Wave mode (batch_mode = 1, or lookahead, full scan, learned
 * proposals): the requests are taken in batches of options.batch_size. Each batch is
 * planned concurrently against the table as it stands (one persistent rollout launch
 * whose clusters pull requests from a device queue, replayed as a CUDA graph), then
 * re-checked in array order: a request is final when no request admitted before it in
 * the batch can reach one of its successor states with a well or come within the
 * separation minima of it; the first request that fails the test, and every later one
 * that an admission may have changed, is planned again against the grown table. Results
 * (verdicts, trajectories, plan ids) are identical to fmdp_schedule_many.
 * On an error, requests finalised before it stay admitted. */
fmdp_status fmdp_schedule_batch(fmdp_ctx* ctx, const fmdp_request* reqs, int32_t n,
                                fmdp_result* res);

/* ---- serving (no counterpart in the paper, which plans requests one at a time) ----
 * fmdp_serve replays an arrival trace against the live table with continuous batching:
 * request i becomes visible arrival_s[i] seconds (wall clock) after the call starts
 * (array order = arrival order = first-come-first-served order; arrival_s non-decreasing).
 * Visible requests join the set of unresolved requests on the device whenever the set
 * has room (max_in_flight) and the table has free slots for all of them (memory-based
 * admission: max_active_plans); each speculative wave plans the newly joined and the
 * influenced requests together, and requests are finalised in arrival order as the
 * waves resolve them. A simulated clock (sim_start_step + time_scale x wall seconds, in
 * steps) expires plans that ended before it, never past the earliest departure still
 * pending. Results (res) equal fmdp_schedule_many over the same requests in the same
 * order; latency_ms[i] (optional) is the wall time from arrival to result. Every request
 * must fit the plan-table window at the start of the call. */
typedef struct {
    double time_scale;        /* simulated seconds per wall-clock second (0 = 1) */
    int64_t sim_start_step;   /* simulated step at the start (default: the window's first) */
    int32_t sim_start_set;    /* 1: use sim_start_step; 0: the window's first step */
    int32_t max_in_flight;    /* unresolved requests at most (0 = batch size; <= 1024) */
    int32_t max_active_plans; /* stored plans at most (0 = max_slots) */
    int32_t expire_quantum;   /* steps the clock advances between expiries (0 = 60) */
} fmdp_serve_options;

typedef struct {
    double wall_s;                 /* from the start of the call to the last result */
    double throughput_rps;         /* requests / wall_s */
    double latency_p50_ms, latency_p99_ms, latency_mean_ms, latency_max_ms;
    int64_t waves, rollouts, replans;
    int64_t expiries, plans_expired;
    int64_t final_t_base;          /* the window's first step at the end */
    int32_t admitted, rejected;
    int32_t max_in_flight_seen;    /* largest unresolved set */
    int32_t deferred_for_memory;   /* requests that waited for free plan slots */
    int32_t pipelined;             /* 1: continuous batching without waves (batch_mode 0) */
    int32_t persistent_ctas;       /* pipelined: CTAs of the persistent rollout launch */
    int64_t drains;                /* pipelined: index rebuilds that waited for the rollouts */
    double rollout_occupancy;      /* pipelined: summed rollout time / (CTAs x wall time) */
} fmdp_serve_report;

void fmdp_serve_options_default(fmdp_serve_options* o);
fmdp_status fmdp_serve(fmdp_ctx* ctx, const fmdp_request* reqs, const double* arrival_s, int32_t n,
                       const fmdp_serve_options* opt, fmdp_result* res, double* latency_ms,
                       fmdp_serve_report* report);

/* ---- learned proposal (no counterpart in the paper) ----
 * A multilayer perceptron (128 -> 256 -> 256 -> 256 -> 256 -> 25, ReLU, bf16 weights, fp32
 * accumulation) maps features of a state (own and goal terms; the nearest plan sample of
 * the next step in each of 20 sectors around the aircraft) to action logits. It is trained
 * on FastMDP's own action choices (Alg. 1), rolls out a whole trajectory by its argmax over
 * the actions that stay in the box, and the proposal is accepted when it reaches the goal,
 * passes the separation and terrain checks, and takes at most (1 + slack) times the fewest
 * steps any trajectory needs (which bounds its cost gap to FastMDP by the same factor);
 * otherwise FastMDP plans the request. Parameters: per layer W (in x out, row-major) then
 * b (out), FMDP_MLP_PARAMS floats. */
#define FMDP_MLP_PARAMS 236825
typedef struct {
    int32_t n;                      /* requests */
    int32_t accepted;               /* proposals accepted */
    int32_t proposals_captured;     /* proposals that reached the goal */
    int32_t fastmdp_captured;       /* FastMDP plans that reached the goal (evaluate) */
    double mean_gap, max_gap;       /* (proposal steps - FastMDP steps) / FastMDP steps over
                                       accepted proposals whose FastMDP plan also captured */
    int64_t proposal_steps, fastmdp_steps;
    double proposal_ms, fastmdp_ms; /* CUDA-event time of the two rollout passes (evaluate) */
} fmdp_learned_report;

/* Plans the requests with FastMDP against the table as it stands (nothing is admitted) and
 * appends one training row per rollout step: the features of the state and FastMDP's
 * action. n_rows_out: rows in the training set after the call. */
fmdp_status fmdp_learned_collect(fmdp_ctx* ctx, const fmdp_request* reqs, int32_t n, int32_t* n_rows_out);
/* Copies up to max_rows training rows out (X: [rows][128] fp32 of the stored bf16 values). */
fmdp_status fmdp_learned_rows(fmdp_ctx* ctx, float* X, uint8_t* y, int32_t max_rows, int32_t* n_out);
fmdp_status fmdp_learned_clear_rows(fmdp_ctx* ctx);
/* Seeded He-normal weights and zero biases. */
fmdp_status fmdp_learned_init(fmdp_ctx* ctx, uint64_t seed);
fmdp_status fmdp_learned_set_params(fmdp_ctx* ctx, const float* params, int32_t n);
fmdp_status fmdp_learned_get_params(fmdp_ctx* ctx, float* params, int32_t n);
/* Adam on the mean cross-entropy of the training set, shuffled with `seed` each epoch;
 * loss_per_epoch (optional, epochs floats): mean batch loss of each epoch. */
fmdp_status fmdp_learned_train(fmdp_ctx* ctx, int32_t epochs, int32_t batch, float lr, uint64_t seed,
                               float* loss_per_epoch);
/* Loss and gradient on the given rows (host X [rows][128], bf16-rounded on the device; y),
 * without changing the parameters (gradient checks). */
fmdp_status fmdp_learned_loss_grad(fmdp_ctx* ctx, const float* X, const uint8_t* y, int32_t rows, float* loss,
                                   float* grad);
/* Proposals and FastMDP plans for every request against the table as it stands (nothing is
 * admitted): acceptance and cost gap. accepted, steps_p, steps_f: optional, n entries. */
fmdp_status fmdp_learned_evaluate(fmdp_ctx* ctx, const fmdp_request* reqs, int32_t n, double slack,
                                  fmdp_learned_report* report, int32_t* accepted, int32_t* steps_p,
                                  int32_t* steps_f);
/* First-come-first-served scheduling where each request takes its accepted proposal, else
 * its FastMDP plan (res[i].source says which), through speculative batches; results equal
 * taking the requests one at a time with the same rule. */
fmdp_status fmdp_schedule_learned(fmdp_ctx* ctx, const fmdp_request* reqs, int32_t n, double slack,
                                  fmdp_result* res, fmdp_learned_report* report);

/* Departure-time candidates (the paper recommends a take-off time among several
 * candidates, Sec. I, and schedules at different departure times in parallel, Sec. IV).
 * For each request in FCFS (array) order, its n_delays variants departing delays[d] steps
 * later are planned concurrently against the table as it stands (one persistent rollout
 * launch and one separation check over all variants), and the first variant in the order
 * of delays (the preferred first) whose plan is admissible is admitted. A rejected variant
 * changes nothing, so each variant up to the chosen one has exactly the result that
 * fmdp_schedule of it alone would give, and the call equals trying the variants one after
 * another with fmdp_schedule until one is admitted.
 *   delays: n_delays entries, 1 <= n_delays <= 1024, in steps (any sign); every variant's
 *           steps must fall inside the table window (FMDP_ERR_RANGE otherwise, and nothing
 *           is planned).
 *   res[i]: the admitted variant's result (its plan_id set), else the first variant's
 *           (verdict a rejection); xyz / actions buffers as for fmdp_schedule.
 *   chosen: optional, n entries: index into delays of the admitted variant, -1 if none.
 *   verdicts: optional, [n][n_delays]: every variant's verdict. */
fmdp_status fmdp_schedule_departures(fmdp_ctx* ctx, const fmdp_request* reqs, int32_t n,
                                     const int64_t* delays, int32_t n_delays, fmdp_result* res,
                                     int32_t* chosen, int32_t* verdicts);
/* The same call through speculative batches (as fmdp_schedule_batch does for single
 * requests): the variants of many requests are planned at once against the table as it
 * stands, and a request's variants are planned again only where an admission of an earlier
 * request of the batch may have changed them. A request is final when no earlier admission
 * of the walk influences any of its variants. Results, chosen and verdicts are identical
 * to fmdp_schedule_departures; res[i].replanned counts the re-plans of the variant shown.
 * Batches hold max(1, batch_size / n_delays) requests; n * n_delays <= 2^24. */
fmdp_status fmdp_schedule_departures_batch(fmdp_ctx* ctx, const fmdp_request* reqs, int32_t n,
                                           const int64_t* delays, int32_t n_delays, fmdp_result* res,
                                           int32_t* chosen, int32_t* verdicts);

/* Batch co-simulation (the paper's batches whose aircraft see each other, Sec. V, with
 * Alg. 1 stepping every aircraft of the batch on one clock). The n requests are planned
 * together from the earliest departure on: at each step every aircraft in flight (departed,
 * not finished) values its actions against the stored plans, the static peaks and the
 * Table 3 wells of every other aircraft in flight, centred at that aircraft's position plus
 * tau times its last move over dt (zero before its first move); then all of them move. The
 * finished trajectories are then checked and admitted in array order (first come, first
 * served; each against the table including the members admitted before it). Results differ
 * from fmdp_schedule_batch, whose requests do not see each other while they plan.
 *   n: at most the number of CTAs one cooperative launch keeps resident (a few hundred;
 *   FMDP_ERR_ARG beyond) and at most the free plan slots. Honours options.lookahead_W. */
fmdp_status fmdp_schedule_cosim(fmdp_ctx* ctx, const fmdp_request* reqs, int32_t n, fmdp_result* res);

/* Failure-detection self-test (no counterpart in the paper). Every wait of the library's
 * kernels is bounded (about a second of SM cycles) and an expired wait ends the call with
 * FMDP_ERR_TIMEOUT instead of hanging the device. This call makes one such wait run out on
 * purpose without a fault: it co-simulates two requests whose grid barrier also waits for
 * a third aircraft that is never launched, so every CTA's wait expires and the kernel
 * returns. observed (optional) receives the status that call produced. Returns FMDP_OK
 * when that status was FMDP_ERR_TIMEOUT and nothing was admitted; the context stays
 * usable. Takes about one second. */
fmdp_status fmdp_selftest_wait_timeout(fmdp_ctx* ctx, int32_t* observed);

/* ---- Autotuner of the batched rollout's launch shape (no counterpart in the paper; the
 * rollout is Alg. 1 whatever the shape, and results are bit-identical across shapes).
 *
 * With the spatial index a speculative wave runs one CTA per request: a control warp, an
 * evaluator warp, an index producer warp and (threads_per_cta / 32 - 3) scanner warps that
 * share out the plan samples near the state, index_stage_items of them staged in shared
 * memory per step. Fewer scanners and less staging let two or more CTAs share a
 * multiprocessor, which pays when a wave holds more requests than there are
 * multiprocessors; more scanners shorten each step, which is what a small wave (the
 * re-plans of a speculative batch) needs. fmdp_autotune times the rollouts of the first W
 * sample requests (nothing is admitted) under every candidate shape, threads per CTA in
 * {128, 192, 256, 320, 384} x staged samples in {512, 1024, 1536, 2048} (those whose
 * staging buffers fit in shared memory), for W = min(n,
 * batch size) and its halvings down to 8, and caches the fastest shape under the key
 * (n_actions, combine, plan-count bucket, wave-size bucket). Each wave of a batched call in
 * wave mode (fmdp_schedule_batch, fmdp_serve, fmdp_schedule_learned, staged batches) then
 * launches with the cached shape of its key, or of the nearest tuned wave-size bucket. The
 * pipelined mode's persistent launch holds at most one CTA per multiprocessor and takes
 * the widest shape (384 threads, 1536 staged samples). options.threads_per_cta and
 * options.index_stage_items, when set, take precedence in both modes. */
typedef struct {
    int32_t n_actions, combine;
    int32_t plans_bucket;        /* bit length of the number of stored plans */
    int32_t wave_bucket;         /* bit length of the number of rollouts in a wave */
    int32_t threads_per_cta;     /* the chosen shape */
    int32_t index_stage_items;
    double ms;                   /* the sample's rollout time under the chosen shape */
} fmdp_tune_entry;
typedef struct {
    fmdp_tune_entry chosen;      /* the entry of the largest wave (sample requests) */
    int32_t candidates;          /* (wave size, shape) pairs timed (0 when cached) */
    int32_t entries;             /* wave-size buckets tuned by this call */
    int32_t ctas_per_sm;         /* resident rollout CTAs per multiprocessor at the choice */
    int32_t from_cache;          /* 1: the largest wave's key was cached and nothing was timed */
    int32_t sample;              /* requests in the largest timed wave */
    int32_t reserved;
    double default_ms;           /* the largest wave at 384 threads and 1536 staged samples */
} fmdp_tune_report;
/* Requires the spatial index (options.full_scan = 0). sample: host requests, at least one;
 * the largest timed wave is the first min(n, batch size). force = 1 re-times cached keys. */
fmdp_status fmdp_autotune(fmdp_ctx* ctx, const fmdp_request* sample, int32_t n, int32_t force,
                          fmdp_tune_report* report);
/* Copies up to cap cache entries out (n_out: entries in the cache), or merges n entries in
 * (a deployment can keep the cache between runs). Entries with shapes outside the candidate
 * set are rejected with FMDP_ERR_ARG. */
fmdp_status fmdp_tune_cache_get(fmdp_ctx* ctx, fmdp_tune_entry* out, int32_t cap, int32_t* n_out);
fmdp_status fmdp_tune_cache_put(fmdp_ctx* ctx, const fmdp_tune_entry* in, int32_t n);

/* Device-resident variant used for kernel-side timing: fmdp_stage_requests copies the
 * requests into library-owned device memory; fmdp_schedule_staged plans them in FCFS
 * order, like fmdp_schedule_many (batched = 0) or fmdp_schedule_batch (batched = 1), but
 * leaves trajectories on the device (only verdicts and counts come back);
 * fmdp_fetch_staged copies results of the last staged run. */
fmdp_status fmdp_stage_requests(fmdp_ctx* ctx, const fmdp_request* reqs, int32_t n);
fmdp_status fmdp_schedule_staged(fmdp_ctx* ctx, int32_t batched, int32_t* n_admitted_out);
fmdp_status fmdp_fetch_staged(fmdp_ctx* ctx, fmdp_result* res, int32_t n);

/* Ids of stored plans with at least one sample in [t_begin, t_end). */
fmdp_status fmdp_query_plans(fmdp_ctx* ctx, int64_t t_begin, int64_t t_end, uint64_t* ids,
                             int32_t cap, int32_t* n_out);
/* Samples of a stored plan (cap points of room in xyz). */
fmdp_status fmdp_get_plan(fmdp_ctx* ctx, uint64_t id, int64_t* t0_out, float* xyz, int32_t cap,
                          int32_t* n_out);

/* The plan table to a file and back (checkpoint / resume of the accepted-plan database, which
 * Sec. V keeps across scheduling runs: loaded at start, appended to by every admission).
 * fmdp_save_plans writes every stored plan's samples that are still inside the window (a
 * plan that started before the window is saved from the window's first step), in plan-id
 * order, to the file at `path` (created or replaced): a header {"FMDPPLN1", window start,
 * plans, samples}, one record {first step, count} per plan, then every sample (x, y, z as
 * float32), little-endian; n_out (optional): plans written. fmdp_load_plans adds the plans of
 * such a file as known plans, like fmdp_add_plans (new ids: ids_out, optional, receives the
 * first cap of them in file order; n_out, optional: plans in the file). A context holding no
 * plans first moves its window to the file's start; otherwise every plan must fall inside
 * the window (FMDP_ERR_RANGE). FMDP_ERR_IO: the file cannot be opened, written or read, or
 * is not a whole plan file; FMDP_ERR_FULL: not enough free slots. */
fmdp_status fmdp_save_plans(fmdp_ctx* ctx, const char* path, int64_t* n_out);
fmdp_status fmdp_load_plans(fmdp_ctx* ctx, const char* path, uint64_t* ids_out, int64_t cap, int64_t* n_out);
/* Slides the window to start at t_now_step: plans whose last sample is before it are
 * removed and their slots freed; table rows of earlier steps are cleared for reuse. */
fmdp_status fmdp_expire(fmdp_ctx* ctx, int64_t t_now_step);
/* Saves / restores the whole plan table and its bookkeeping (device copy, no host trip). */
fmdp_status fmdp_snapshot(fmdp_ctx* ctx);
fmdp_status fmdp_restore(fmdp_ctx* ctx);
/* Removes every stored plan. */
fmdp_status fmdp_clear(fmdp_ctx* ctx);

/* ---- inspection entry points (tests, tracing) ---- */

/* Rollout without separation check or admission. Optional per-step traces (NULL to skip):
 * q [horizon][n_actions] fp64 action values (-inf invalid), states [horizon+1][3] fp64,
 * headings [horizon+1] (index of 15-degree heading relative to the initial bearing),
 * tie_flags [horizon]. res->verdict is FMDP_ADMITTED when the goal was captured. */
fmdp_status fmdp_rollout_trace(fmdp_ctx* ctx, const fmdp_request* req, fmdp_result* res,
                               double* q, double* states, int32_t* headings, uint8_t* tie_flags);

typedef struct {
    int32_t first_conflict_step, first_terrain_step;
    int64_t conflicts;       /* number of (sample, plan) pairs in conflict */
    double min_sep_h, min_sep_v;
} fmdp_sep_report;
/* Separation and terrain check of n fp32 samples from step t0 against the stored plans. */
fmdp_status fmdp_sep_check(fmdp_ctx* ctx, int64_t t0_step, const float* xyz, int32_t n,
                           fmdp_sep_report* out);

/* ---- allocation-free separation check (no counterpart in the paper) ----
 * Same check and report as fmdp_sep_check, for callers that cannot allocate device memory
 * while they run: flight or ground software that must fix its memory footprint at start-up
 * (certified or real-time code that forbids allocation after initialisation), and code
 * that must not pay for, or be synchronised by, cudaMalloc/cudaFree on its path.
 * fmdp_sep_check stages the trajectory and its accumulators in device memory that the
 * library allocates and grows on demand; this variant stages them in one fixed scratch
 * array that is part of the loaded library image, and allocates nothing.
 *   - At most FMDP_NOALLOC_MAX_POINTS samples (xyz: host, 3*n fp32); a larger n returns
 *     FMDP_ERR_ARG and planning state is untouched. out: host report.
 *   - The scratch array (about 192 KiB, held by every GPU that loads the library until
 *     the process exits) is shared by every call on that device and keeps the last call's
 *     contents; each call clears the accumulators it needs. Calls whose device work
 *     overlaps (several host threads, or several contexts on one device) race on the
 *     array and must be serialised by the caller.
 *   - The first call on a context is its set-up call: it looks up the array's address on
 *     the context's device (kept in the context), and with lazy module loading that is also
 *     when the driver places the array in device memory. Make that first call during
 *     start-up, before any stream capture; later calls take no device memory.
 *   - The call runs on the context's device whichever device is current, and restores the
 *     caller's current device on return. It is counted in fmdp_stats as a separation-check
 *     launch, like fmdp_sep_check. */
#define FMDP_NOALLOC_MAX_POINTS 16384
fmdp_status fmdp_sep_check_noalloc(fmdp_ctx* ctx, int64_t t0_step, const float* xyz, int32_t n,
                                   fmdp_sep_report* out);

typedef struct {
    int64_t rollout_launches, sepcheck_launches, admit_launches;
    double rollout_ms, sepcheck_ms, admit_ms; /* summed CUDA-event durations */
    int64_t rollout_steps;                    /* rollout steps executed */
    int64_t slots_scanned;                    /* (step, slot) pairs scanned by rollouts */
    int64_t sep_pairs;                        /* (sample, slot) pairs scanned by sep_check */
    int32_t cluster_size, threads_per_cta, slots_per_cta;
    int32_t reserved;
    int64_t phase_cycles[6];  /* on = 2: summed SM cycles of rollout phases: control warp waiting
                                 at the step barrier, control per-action work, control waiting
                                 for the scanners, exchange + argmax + advance, one scanner
                                 warp's cull + wells, producer issue + wait */
    int64_t batch_waves;         /* speculative waves run by fmdp_schedule_batch */
    int64_t batch_rollouts;      /* rollouts run by those waves (first plans and re-plans) */
    int64_t batch_replans;       /* re-plans among them */
    int64_t influence_launches;  /* influence-test launches (on = 1) */
    double influence_ms;         /* their summed CUDA-event durations */
    int64_t kernel_launches;     /* every kernel launch of the library, graph nodes included */
    int64_t items_scanned;       /* indexed rollouts: plan samples read by their steps (on >= 1) */
    int64_t pipe_drains;         /* pipelined batches: index rebuilds that waited for the rollouts */
    double pipe_cta_s;           /* pipelined: summed wall time from dispatch to report of every plan */
    double pipe_slot_s;          /* pipelined: persistent CTAs x wall time of the calls */
    int32_t pipe_ctas;           /* pipelined: CTAs of the last persistent launch */
    int32_t pipe_resident;       /* pipelined: CTAs of that shape the device keeps resident */
    int64_t pipe_resumes;        /* pipelined re-plans that kept the steps before the first one an
                                    admission could change */
    int64_t pipe_rechecks;       /* pipelined re-plans that kept the whole plan and redid only its
                                    conflict check */
    int64_t qe_items;            /* indexed rollouts (on >= 1): plan samples culled by the well scan */
    int64_t qe_near;             /* ... of them inside the cull radius (their wells are masked) */
    int64_t qe_wells;            /* (sample, reachable well) pairs valued, each for every action */
    int64_t pipe_head_n[5];      /* pipelined: requests by how they waited at the head of the line:
                                    [0] plan ready and valid, [1] plan in flight, then valid, [2] in
                                    flight, then planned again, [3] ready but planned again, [4] not
                                    yet dispatched */
    double pipe_head_s[5];       /* ... and the wall seconds they waited there, per kind */
    int64_t pipe_publishes;      /* pipelined: tentative plans published for later requests */
    int64_t pipe_withdrawals;    /* pipelined: tentative plans withdrawn (superseded or rejected) */
} fmdp_stats;
/* Switches the batch mode (fmdp_options.batch_mode) of later calls: 0 pipelined, 1 waves. */
fmdp_status fmdp_set_batch_mode(fmdp_ctx* ctx, int32_t mode);
/* Completion time of each request of the last fmdp_schedule_many / _batch / _staged /
 * fmdp_schedule_learned call, in ms from the call's start (sequential calls: CUDA events
 * after each request's admission step; batched calls: when the host finalised it). Copies
 * min(cap, n) values; *n_out = n, the call's request count. Measurement support, no
 * counterpart in the paper. */
fmdp_status fmdp_last_call_times(fmdp_ctx* ctx, double* ms, int32_t cap, int32_t* n_out);
/* Measured throughput of the units the well scan uses, on the context's device: FP32 FMA
 * (2 flops each), MUFU reciprocal square root and exp2, over all SMs, with the mean SM clock
 * during the FMA probe. Takes a few milliseconds. Measurement support, no counterpart in
 * the paper. */
typedef struct {
    double fp32_tflops;
    double mufu_rsqrt_tops;
    double mufu_ex2_tops;
    double sm_mhz;
} fmdp_peaks;
fmdp_status fmdp_probe_peaks(fmdp_ctx* ctx, fmdp_peaks* out);

/* on = 1: per-kernel CUDA-event timing on the context's stream; on = 2: additionally
 * per-phase cycle counters inside the rollout kernel (diagnostic, slows it slightly);
 * 0: off (default). Resets the statistics. */
fmdp_status fmdp_set_profiling(fmdp_ctx* ctx, int32_t on);
fmdp_status fmdp_get_stats(fmdp_ctx* ctx, fmdp_stats* out);

#ifdef __cplusplus
}
#endif
#endif /* FMDP_H */
