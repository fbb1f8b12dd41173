// Internal types and device helpers of libfmdp (GB300, sm_103a).
//
// Device layout of the known-plan table (the paper's intruder peaks P^I are never
// materialised, Table 1): three fp32 planes X, Y, Z of shape [T_win][S_pad]; row
// (t mod T_win) holds every slot's position at time step t, NaN where the slot has
// no sample. A plan occupies one slot (column) for its whole life.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/fmdp.h"

namespace fmdp {

constexpr int kMaxActions = 32;  // one lane of a warp per action
constexpr int kMaxWells = 8;
constexpr int kMaxStatic = 64;
constexpr int kHeadings = 24;    // 15-degree heading table
constexpr int kRing = 4;         // slice buffers per CTA (two in use, two in flight)
constexpr int kMaxCluster = 16;
constexpr float kWellBand = 4e-5f;  // |d^2 - R^2| <= kWellBand * R^2 -> FP64 re-evaluation
constexpr float kClrBand = 0.05f;   // metres around the clearance threshold -> FP64
constexpr double kTieRel = 1e-4;    // near-tie bar on the top-2 action values
constexpr int kStatusCaptured = 0;
// SUM mode: well values are added as integers in units of 2^-kSumBits of the largest |r|
// (exact and order-independent). 48 bits resolve a well's edge value to better than 1e-6
// and leave room for 65536 full-strength terms per action and step.
constexpr int kSumBits = 48;
constexpr float kSumUnits = 281474976710656.0f;  // 2^48

// Constants of a scheduler, passed by value into every kernel.
struct Model {
    double box[6];
    double dt;
    double lg64;        // log2(gamma) of the goal peak
    double log2rg;      // log2(goal_reward)
    double goal_reward;
    double clearance, deck;
    double sep_h, sep_v;
    double sum_scale;   // 2^(sum_ref - kSumBits): value of one unit of the sum mode's fixed point
    float lg32;
    float hm_sx, hm_sy; // heightmap nodes per metre along x, y
    float reach_base;   // max_k R_k + 1 m margin (coarse cull radius without motion terms)
    float tau_absmax;   // max_k |tau_k|
    float sum_ref;      // log2 of the largest |r| (fixed-point reference of the sum mode)
    int32_t A;
    int32_t combine;
    int32_t n_wells;
    int32_t n_static;
    int32_t hm_nx, hm_ny;
    const float* hm;        // device heightmap or nullptr
    const double* statics;  // device [n_static][6] or nullptr
    int32_t dh[kMaxActions];
    double climb[kMaxActions];
    float w_tau[kMaxWells], w_R2[kMaxWells], w_band[kMaxWells], w_L[kMaxWells], w_lg[kMaxWells];
    double w_tau64[kMaxWells], w_R64[kMaxWells];
    float st_R2[kMaxStatic], st_band[kMaxStatic], st_L[kMaxStatic], st_lg[kMaxStatic];
};

struct TableView {
    float* X;
    float* Y;
    float* Z;
    int32_t T_win, S_pad;
    int64_t t_base;
};

// Spatial index of the plan table (one per ring row, rebuilt or appended as rows change).
// Row r holds one item per slot with a sample at the row's step T: the sample p(T) and the
// same slot's sample p(T+1) (NaN when there is none), 32 bytes; the first float4's w holds
// a tag (its int32 bits): the slot number (>= 0) of a stored plan; during a pipelined call
// also -(o + 2) for a sample of the tentative plan of the request with FCFS ordinal o
// (seen only by the rollouts of later requests), or -1 for a withdrawn tentative sample.
// Items are grouped by the 2-D cell of p(T) (ncx x ncy cells of `cell` metres over the airspace box, positions
// outside the box clamped to the edge cells), in cell order; after the last cell comes the
// extra list, scanned for every query: items moving faster than vmax (their wells reach
// further than the cell query covers) and items appended since the row was last rebuilt.
constexpr int32_t kTagDead = -1;
__host__ __device__ __forceinline__ int32_t tentative_tag(int32_t ord) { return -(ord + 2); }
// Is an item with this tag part of the table that the request with ordinal my_ord plans
// against? (stored plans always; tentative plans of earlier requests; never withdrawn ones)
__host__ __device__ __forceinline__ bool tag_visible(int32_t tag, int32_t my_ord) {
    return tag >= 0 || (tag <= -2 && -tag - 2 < my_ord);
}
struct IndexView {
    const int32_t* cstart;  // [T_win][ncell + 1]: first item of each cell; [ncell] = extra list start
    const int32_t* nextra;  // [T_win]: items in the extra list
    const float4* items;    // [T_win][S_pad][2]: {x, y, z, tag} at T and {x, y, z, 0} at T + 1
    int32_t ncx, ncy, ncell;
    float x0, y0, inv_cell;  // cell of x: floor((x - x0) * inv_cell), clamped
    float vmax;              // speed bound of the items outside the extra list (m/s)
};

struct RolloutOut {
    int32_t n_points;
    int32_t status;  // kStatusCaptured, FMDP_REJ_HORIZON or FMDP_REJ_NO_ACTION
    int32_t near_ties;
    int32_t steps;
};

struct SepOut {
    int32_t first_conflict;  // INT_MAX when none
    int32_t first_terrain;   // INT_MAX when none
    unsigned long long conflicts;
    uint32_t min_h_bits;     // fp32 bits, +inf when none (non-negative floats order as ints)
    uint32_t min_v_bits;
    int32_t verdict;
    int32_t pad;
};

// Pipelined speculative FCFS (continuous batching). One persistent rollout launch takes
// work items from a ring in host-mapped memory that the host appends to while the launch
// runs; each finished plan is checked for conflicts against the plans it could see, and
// its trajectory and report are written to host-mapped memory, then its completion token.
struct PipeItem {
    int32_t r;      // request number of the call
    int32_t token;  // written to done[r] when this plan has finished
    int32_t start;  // 0: plan from the origin; k > 0: keep the plan's first k steps and plan on
                    // from its state at step k; -1: keep the plan, redo only its conflict check
    int32_t pad;
    int64_t t_base;  // first step of the table window when the item was dispatched (an expiry
                     // moves it while earlier items are still in flight)
};
struct PipeRecord {
    RolloutOut ro;
    int32_t first_conflict;  // the tail check's first conflicting sample, -1 when none
    int32_t first_terrain;   // first sample below the terrain, -1 when none
    int32_t tail_pub;        // admissions published before the tail check read the index
    int32_t pad;
};
struct PipeArgs {
    int32_t on;
    int32_t qmask;            // ring entries - 1 (a power of two)
    const PipeItem* items;    // host-mapped ring
    const int32_t* tail;      // host-mapped: items written so far
    const int32_t* stop;      // host-mapped: 1 = leave once the ring is empty
    int32_t* head;            // device: items taken so far
    int32_t* done;            // host-mapped [n]: token of the last finished plan of request r
    PipeRecord* rec;          // host-mapped [n]
    float* h_traj;            // host-mapped [n][cap][3]
    SepOut* sep;              // device [n]: the tail check's report (read by the admission)
    long long idle_cycles;    // a CTA that finds no work for this many SM cycles leaves
    // Admissions of the call published so far (device; the table stream raises it after each
    // admission's index entries are visible). A rollout step records the count it read
    // before the index rows it valued (obs[r][k] for step k; copied to h_obs), so the host
    // tests an admission only against the steps that could not see it.
    const int32_t* pub_seq;
    int32_t* obs;             // device [n][cap]
    int32_t* h_obs;           // host-mapped [n][cap]
    // What a plan resumed at step k needs of step k (FastMDP's choice at a step depends on
    // the state then, not on how it was reached): per trajectory point, the exact state, its
    // double-float copy and the heading index; per decision step, its near-tie flag.
    double* st_s;             // device [n][cap][3]
    float* st_df;             // device [n][cap][6]: hi, lo of x, y, z
    uint8_t* st_h;            // device [n][cap]
    uint8_t* ties;            // device [n][cap]
    int32_t ord0;             // FCFS ordinal of the call's request 0 (request r: ord0 + r)
};

struct RolloutArgs {
    Model m;
    TableView tab;
    int32_t S_scan;   // slots scanned per step (multiple of 32)
    int32_t chunk;    // slots per CTA (multiple of 32)
    int32_t cs;       // CTAs per request (cluster size)
    int32_t ring;     // slice buffers per CTA: 4 or 8
    int32_t cap;      // trajectory capacity per request (points)
    const fmdp_request* reqs;
    int32_t n_req;
    int32_t trace;
    float* traj;      // [n_req][cap][3]
    uint8_t* acts;    // [n_req][cap]
    RolloutOut* out;  // [n_req]
    double* q_trace;  // [cap][A] (request 0 only) or nullptr
    double* st_trace; // [cap][3]
    int32_t* hd_trace;
    uint8_t* tie_trace;
    int32_t* err;     // device error word
    int32_t* queue;   // batch mode: request counter the CTAs pull from (nullptr: one cluster per request)
    const int32_t* idx;    // batch mode: request index of work item w (nullptr: identity)
    const int32_t* n_dev;  // batch mode: number of work items, read on the device (nullptr: n_req)
    unsigned long long* phase;  // [6] per-phase cycle counters (diagnostic) or nullptr
    int32_t indexed;  // 1: stage the items near the state from the spatial index (cs must be 1)
    int32_t icap;     // indexed mode: items per staging buffer in shared memory
    IndexView iv;
    unsigned long long* items_ctr;  // indexed mode: items read by the steps (statistics) or nullptr
    unsigned long long* qe_ctr;     // indexed mode (statistics) or nullptr: [0] items culled, [1] items
                                    // inside the cull radius, [2] (item, reachable well) pairs valued
    const int32_t* skip;            // batch mode: request r is not planned when skip[r] (nullptr: none)
    PipeArgs pipe;                  // pipelined mode (pipe.on): work from the host-fed ring
};

struct SepArgs {
    Model m;
    TableView tab;
    int32_t S_scan;
    int32_t cap;
    const float* traj;          // [n][cap][3]
    const RolloutOut* rout;     // n_points per request (nullptr: use n_fixed)
    const fmdp_request* reqs;   // t0 = depart_step (nullptr: use t0_fixed)
    int64_t t0_fixed;
    int32_t n_fixed;
    SepOut* out;
    const int32_t* idx;    // request index of work item z (nullptr: identity)
    const int32_t* n_dev;  // number of work items on the device (nullptr: all launched)
};

struct AdmitArgs {
    TableView tab;
    int32_t cap;
    const float* traj;
    const RolloutOut* rout;
    const fmdp_request* reqs;
    const int32_t* slots;  // slot per request
    SepOut* sep;           // verdict written here
    int32_t force;         // 1: store unconditionally (known plans)
    const int64_t* t0s;    // force mode: per plan t0
    const int32_t* counts; // force mode: per plan count
    const int64_t* offs;   // force mode: per plan offset into traj (points)
    const int32_t* idx;    // request index of work item y (nullptr: identity)
    const int32_t* n_dev;  // number of work items on the device (nullptr: all launched)
    const int32_t* err;    // device error word: nothing is stored once a wait has expired
    int32_t* slot_ord;     // if set: slot_ord[slot] = ord for an admitted trajectory
    int32_t ord;           // FCFS ordinal of the admitted request (see SepRowsArgs)
};

// Speculative batching: could request j's trajectory (as a stored plan) change request k's
// plan or verdict? out[w*n + v] for work items w (k) and v (j), j < k in arrival order.
struct InfluenceArgs {
    const float* traj;          // [n_all][cap][3]
    const RolloutOut* rout;     // n_points per request
    const fmdp_request* reqs;
    int32_t cap;
    const int32_t* idx;         // request index of work item
    const int32_t* n_dev;       // number of work items
    float reach_base;           // max_k R_k + 1 m
    float tau_absmax;
    int32_t n_wells;            // > 0: test each well centre against its own radius
    float w_tau[kMaxWells];     // well offsets along the plan's velocity (s)
    float w_R[kMaxWells];       // well radii (m)
    int32_t W;                  // lookahead sub-steps of each rollout step (1: the one-step rule)
    float feat_r;               // > 0: proposals read plan samples this close (m, + 1 m)
    const float* traj_p;        // proposals [n_all][cap][3], or null
    const RolloutOut* rout_p;   // proposals' n_points
    const int32_t* accepted;    // 1 where the stored trajectory is the accepted proposal
    float dzmax;                // largest climb * dt
    float sep_h, sep_v;
    float dt;
    uint8_t* out;               // [n][n]
    int32_t n_cap;              // row stride of out
};


// Throughput probes (probe.cu): FP32 FMA, and the MUFU reciprocal square root and exp2 the
// rollout's value terms use, over every SM; the SM clock from clock64 against event time.
cudaError_t probe_peaks(int n_sm, cudaStream_t s, fmdp_peaks* out);

// kernel launchers (rollout.cu / tables.cu)
// n_clusters > 0: persistent launch of that many clusters (work-queue mode), else one
// cluster per request.
cudaError_t launch_rollout(const RolloutArgs& a, int threads, size_t smem, cudaStream_t s, int n_clusters = 0);
size_t rollout_smem_bytes(int chunk, int depth, int icap);
cudaError_t prepare_rollout_kernel(size_t smem);
// Load the kernels of index.cu / tables.cu at context creation instead of at their first launch
// (a lazy load waits for the kernels running at the time, such as a persistent rollout launch).
cudaError_t preload_index_kernels();
cudaError_t preload_table_kernels();
// Packs the samples of n plans (slot, first step, count each; offsets into out in samples)
// from the table planes into out [sum counts][3].
cudaError_t launch_gather_plans(const float* X, const float* Y, const float* Z, int32_t S_pad, int32_t T_win,
                                const int32_t* slots, const int64_t* t0s, const int32_t* counts, const int64_t* offs,
                                float* out, int n_plans, int max_count, cudaStream_t s);
int rollout_max_active_clusters(int cs, int threads, size_t smem);
cudaError_t launch_sepcheck(const SepArgs& a, int n_req, int max_points, cudaStream_t s);
cudaError_t launch_sep_reset(SepOut* out, int n, cudaStream_t s);
cudaError_t launch_admit(const AdmitArgs& a, int n_req, int max_points, cudaStream_t s);
cudaError_t launch_fill_nan(float* p, size_t n, cudaStream_t s);

// Spatial index maintenance. Rows are named by absolute step T (ring row T mod T_win).
struct IndexArgs {
    TableView tab;
    int32_t* cstart;
    int32_t* nextra;       // [T_win]: published extra-list length (readers scan this many)
    int32_t* nres;         // [T_win]: extra-list positions handed out to appends
    int32_t* dirty;        // [T_win]: row must be rebuilt before its next use
    float4* items;
    int32_t ncx, ncy, ncell;
    float x0, y0, inv_cell, vmax, inv_dt;
    int32_t extra_limit;   // appended items beyond this mark the row dirty
};
// Rebuilds the rows of steps [T0, T0 + n) (n <= T_win); dirty_only: only rows marked dirty
// (and clears their marks).
cudaError_t launch_index_build(const IndexArgs& a, int64_t T0, int32_t n, int dirty_only, size_t smem, cudaStream_t s);
size_t index_build_smem(int ncell);
cudaError_t prepare_index_kernels(size_t smem);
// Appends the stored trajectories of the listed requests to the extra lists of their rows:
// requests idx[0 .. *n_dev) (or 0 .. n-1), admitted ones only (SepOut verdict), samples
// traj[r][0 .. rout[r].n_points) from step reqs[r].depart_step. An append takes positions
// past the published length (nres) and writes its items there; launch_index_publish then
// makes them visible, so a rollout that reads the index meanwhile never sees a partly
// written item (each item is either absent or complete).
struct IndexAppendArgs {
    IndexArgs ix;
    const int32_t* slots;  // slot of request r (force mode: of plan r), stored in each item
    int32_t tentative;     // 1: tag the items tentative_tag(tent_ord) instead of the slot, take
    int32_t tent_ord;      // the trajectory whatever its verdict, and record each sample's
    int32_t* tpos;         // position in tpos[r][k] (-1: not stored); 0: stored plans
    int32_t first;         // tentative: samples before this one keep the items (and tpos
                           // entries) an earlier append made for them; only [first, n) are added
    const float* traj;
    int32_t cap;
    const RolloutOut* rout;
    const fmdp_request* reqs;
    const SepOut* sep;
    const int32_t* idx;
    const int32_t* n_dev;
    // force mode (known plans): n plans with t0s / counts / offs into traj
    int32_t force;
    const int64_t* t0s;
    const int32_t* counts;
    const int64_t* offs;
};
cudaError_t launch_index_append(const IndexAppendArgs& a, int n_items, int max_points, cudaStream_t s);
// Publishes the appended items of every row (nextra = nres); launched after the appends.
cudaError_t launch_index_publish(const IndexArgs& a, cudaStream_t s);
// Withdraws the tentative items of one trajectory (n samples from step t0, positions
// tpos[0 .. n) as its append recorded them): their tag becomes kTagDead.
cudaError_t launch_index_withdraw(const IndexArgs& a, const int32_t* tpos, int64_t t0, int32_t n, cudaStream_t s);
// *p = v with release semantics (a counter that readers acquire), one thread
cudaError_t launch_store_release(int32_t* p, int32_t v, cudaStream_t s);
// Separation check of a batch's work items, row by row: block b takes step t_base + b, the
// samples of every work item at that step, and the row's plan samples (from the spatial
// index when there is one, else the table planes). Same results as sepcheck_kernel.
struct SepRowsArgs {
    Model m;
    TableView tab;
    int32_t S_scan;
    const float* traj;  // [n][cap][3]
    int32_t cap;
    const RolloutOut* rout;
    const fmdp_request* reqs;
    const int32_t* idx;    // work items
    const int32_t* n_dev;  // their number (<= n_max)
    int32_t n_max;
    SepOut* out;
    const float4* items;    // spatial index (nullptr: read the table planes)
    const int32_t* cstart;
    const int32_t* nextra;
    int32_t ncell;
    const int32_t* skip;    // request r is not checked when skip[r] (nullptr: none)
    // ordinal filter (pipelined FCFS, where the table may already hold plans admitted after
    // a request): request r is checked only against items whose slot's ordinal is below
    // req_ord[r]; plans that were in the table before the call carry smaller ordinals
    const int32_t* slot_ord;  // [S_pad] or nullptr (no filter)
    const int32_t* req_ord;   // [n]
    // rows checked: the steps t_base + row0 .. + nrows - 1 (nrows 0: the whole window); the
    // rows no listed trajectory reaches add nothing
    int32_t row0, nrows;
};
cudaError_t launch_sepcheck_rows(const SepRowsArgs& a, cudaStream_t s);
size_t sepcheck_rows_smem(int n_max);
cudaError_t prepare_sepcheck_rows(size_t smem);

// Batch epilogue: minimum separations to the batch's own admissions.
struct MinSepArgs {
    const float* traj;       // [n][cap][3]
    const RolloutOut* rout;
    const fmdp_request* reqs;
    int32_t cap, k0, n;      // requests k0 .. k0 + n - 1
    const int32_t* adm;      // admitted request indices, ascending
    int32_t n_adm;
    double sep_h, sep_v;
    SepOut* out;             // [n]
};
cudaError_t launch_batch_minsep(const MinSepArgs& a, cudaStream_t s);
cudaError_t launch_influence(const InfluenceArgs& a, int n_max, int max_points, cudaStream_t s);
cudaError_t launch_sep_reset_idx(SepOut* out, const int32_t* idx, const int32_t* n_dev, int n_max, cudaStream_t s);

// Rollout with a lookahead window of W sub-steps (lookahead.cu): one CTA per request,
// requests[0 .. n_req), trajectories of cap samples each; traces as for the rollout kernel.
constexpr int kMaxLookahead = 16;
struct LookArgs {
    Model m;
    TableView tab;
    int32_t S_scan;  // slots scanned per slice
    int32_t W;       // 1 .. kMaxLookahead
    int32_t cap;
    int32_t n_req;
    int32_t trace;
    const fmdp_request* reqs;
    float* traj;
    uint8_t* acts;
    RolloutOut* out;
    double* q_trace;
    double* st_trace;
    int32_t* hd_trace;
    uint8_t* tie_trace;
    int32_t* err;
    // co-simulation: the n_req CTAs (one cooperative launch) step on one clock from t_start
    // and see each other's wells; each publishes its state per step in mem
    int32_t cosim;
    int64_t t_start;
    double* mem;   // [2][n_req][8]: x, y, z, vx, vy, vz, flying, alive (by step parity)
    int32_t* bar;  // [2]: arrivals, generation of the grid barrier (zero before launch)
    int32_t absent;  // self-test only: arrivals the barrier waits for that never come
    // speculative waves (not with cosim): CTA w plans work item idx[w] while w < *n_dev
    const int32_t* idx;
    const int32_t* n_dev;
};
size_t lookahead_smem_bytes(int A, int W);
int lookahead_max_resident(int A, int W);  // CTAs of one cooperative launch that fit
cudaError_t prepare_lookahead_kernel();
cudaError_t launch_lookahead(const LookArgs& a, cudaStream_t s);

// ---------------------------------------------------------------- device helpers

__device__ __forceinline__ int float_key(float f) {
    int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float key_float(int k) {
    return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff);
}

// 2^n as a double, for n in the normal range.
__device__ __forceinline__ double pow2i(int n) {
    return __hiloint2double((n + 1023) << 20, 0);
}
// x * 2^n with gradual underflow for very negative n.
__device__ __forceinline__ double scale2(double x, int n) {
    if (n >= -1022 && n <= 1023) return x * pow2i(n);
    if (n < -1022) return (x * pow2i(-600)) * pow2i(n + 600 < -1022 ? -1022 : n + 600);
    return x * pow2i(1023);
}

// Bilinear terrain height in FP64, evaluated in exactly the order written (no FMA).
__device__ __forceinline__ double terrain64(const Model& m, double x, double y) {
    const int nx = m.hm_nx, ny = m.hm_ny;
    double fx = __dmul_rn(__ddiv_rn(__dsub_rn(x, m.box[0]), __dsub_rn(m.box[3], m.box[0])), (double)(nx - 1));
    double fy = __dmul_rn(__ddiv_rn(__dsub_rn(y, m.box[1]), __dsub_rn(m.box[4], m.box[1])), (double)(ny - 1));
    double flx = floor(fx), fly = floor(fy);
    int ix = (int)flx, iy = (int)fly;
    if (flx < 0.0) ix = 0;
    if (fly < 0.0) iy = 0;
    if (ix > nx - 2) ix = nx - 2;
    if (iy > ny - 2) iy = ny - 2;
    double ax = __dsub_rn(fx, (double)ix), ay = __dsub_rn(fy, (double)iy);
    const float* r0 = m.hm + (size_t)iy * nx + ix;
    const float* r1 = r0 + nx;
    double h00 = __ldg(r0), h10 = __ldg(r0 + 1), h01 = __ldg(r1), h11 = __ldg(r1 + 1);
    double bx = __dsub_rn(1.0, ax), by = __dsub_rn(1.0, ay);
    double lo = __dadd_rn(__dmul_rn(bx, h00), __dmul_rn(ax, h10));
    double hi = __dadd_rn(__dmul_rn(bx, h01), __dmul_rn(ax, h11));
    return __dadd_rn(__dmul_rn(by, lo), __dmul_rn(ay, hi));
}

// Bilinear terrain height in fp32 (the same grid and clamping as terrain64). Its error
// against terrain64 is below 0.05 m for heights of a few hundred metres on grids of up to a
// few thousand cells a side; callers decide in fp32 outside a band and call terrain64 inside.
__device__ __forceinline__ float terrain32(const Model& m, float x, float y) {
    const float gxf = (x - (float)m.box[0]) * m.hm_sx;
    const float gyf = (y - (float)m.box[1]) * m.hm_sy;
    int ix = (int)floorf(gxf), iy = (int)floorf(gyf);
    ix = min(max(ix, 0), m.hm_nx - 2);
    iy = min(max(iy, 0), m.hm_ny - 2);
    const float ax = gxf - (float)ix, ay = gyf - (float)iy;
    const float* r0 = m.hm + (size_t)iy * m.hm_nx + ix;
    const float h00 = __ldg(r0), h10 = __ldg(r0 + 1), h01 = __ldg(r0 + m.hm_nx), h11 = __ldg(r0 + m.hm_nx + 1);
    return (1.f - ay) * ((1.f - ax) * h00 + ax * h10) + ay * ((1.f - ax) * h01 + ax * h11);
}
constexpr float kTerrBand = 0.25f;  // metres: fp32 terrain-collision margin before an FP64 check

// cos / sin of k * 15 degrees from their surd forms (exact IEEE operations only).
__device__ __forceinline__ void unit15(int k, double& ck, double& sk) {
    const double r2 = __dsqrt_rn(2.0), r3 = __dsqrt_rn(3.0), r6 = __dsqrt_rn(6.0);
    const double c15 = __ddiv_rn(__dadd_rn(r6, r2), 4.0), s15 = __ddiv_rn(__dsub_rn(r6, r2), 4.0);
    const int m = k % 6, quad = k / 6;
    double qc, qs;
    switch (m) {
        case 0: qc = 1.0; qs = 0.0; break;
        case 1: qc = c15; qs = s15; break;
        case 2: qc = __ddiv_rn(r3, 2.0); qs = 0.5; break;
        case 3: qc = __ddiv_rn(r2, 2.0); qs = __ddiv_rn(r2, 2.0); break;
        case 4: qc = 0.5; qs = __ddiv_rn(r3, 2.0); break;
        default: qc = s15; qs = c15; break;
    }
    if (quad == 0) { ck = qc; sk = qs; }
    else if (quad == 1) { ck = -qs; sk = qc; }
    else if (quad == 2) { ck = -qc; sk = -qs; }
    else { ck = qs; sk = -qc; }
}

__device__ __forceinline__ double norm3_64(double dx, double dy, double dz) {
    return __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
}

}  // namespace fmdp
