// Host runtime and C ABI of libfmdp: scheduler context, device plan table, slot
// allocator, sliding time window and first-come-first-served sequencing.
//
// FCFS (Sec. I, Sec. V): requests are planned one after another against every stored
// plan; each admitted trajectory is stored before the next request is planned. The
// per-request chain (rollout -> separation check -> admission) is decided entirely on the
// device, so a whole sequence of requests is enqueued on one stream with no host round
// trip; the host only reads verdicts back at the end to update its bookkeeping.
#include <algorithm>
#include <chrono>
#include <thread>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <array>
#include <map>
#include <new>
#include <set>
#include <stdexcept>
#include <string>
#include <vector>

#include "learned.cuh"

using namespace fmdp;

namespace {

struct ApiError : std::runtime_error {
    fmdp_status code;
    ApiError(fmdp_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

void cuda_check(cudaError_t e, const char* what) {
    if (e != cudaSuccess) {
        const fmdp_status code = (e == cudaErrorMemoryAllocation) ? FMDP_ERR_OOM : FMDP_ERR_CUDA;
        throw ApiError(code, std::string(what) + ": " + cudaGetErrorString(e));
    }
}
#define CK(x) cuda_check((x), #x)
// a kernel launch of the library on context c (counted unless it is being captured)
#define LAUNCH(c, x)                                             \
    do {                                                         \
        cuda_check((x), #x);                                     \
        if (!(c)->capturing) (c)->stats.kernel_launches++;       \
    } while (0)

void require(bool ok, fmdp_status code, const std::string& msg) {
    if (!ok) throw ApiError(code, msg);
}

template <class T>
struct DevArray {
    T* p = nullptr;
    size_t n = 0;
    void ensure(size_t want) {
        if (want <= n) return;
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
        size_t m = std::max<size_t>(want, 16);
        CK(cudaMalloc(&p, m * sizeof(T)));
        n = m;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
};

template <class T>
struct PinnedArray {
    T* p = nullptr;
    size_t n = 0;
    void ensure(size_t want) {
        if (want <= n) return;
        if (p) cudaFreeHost(p);
        p = nullptr;
        n = 0;
        size_t m = std::max<size_t>(want, n * 2);
        CK(cudaMallocHost(&p, m * sizeof(T)));
        n = m;
    }
    void release() {
        if (p) cudaFreeHost(p);
        p = nullptr;
        n = 0;
    }
};

struct PlanMeta {
    int32_t slot;
    int64_t t0;
    int32_t n;
};

struct Book {  // host bookkeeping of the table (copied by snapshot / restore)
    std::set<int32_t> free_slots;
    std::map<uint64_t, PlanMeta> plans;
    uint64_t next_id = 1;
    int64_t t_base = 0;
    int32_t S_hw = 0;
};

int32_t round_up(int32_t x, int32_t m) { return (x + m - 1) / m * m; }

// Device buffers of one FCFS sequence run.
struct SeqBuffers {
    DevArray<fmdp_request> reqs;
    DevArray<float> traj;
    DevArray<uint8_t> acts;
    DevArray<RolloutOut> rout;
    DevArray<SepOut> sepo;
    DevArray<int32_t> slots;
    void release() {
        reqs.release(); traj.release(); acts.release(); rout.release(); sepo.release(); slots.release();
    }
};

// Device and pinned buffers of speculative batching (fmdp_schedule_batch). Per-request
// arrays cover every request of the call (rq_cap entries, trajectories of cap samples),
// so that batches of one call index them by request number. The index block holds the
// work items to plan, the unresolved requests in arrival order and the requests to store
// (n_cap entries each, one batch), then each request's slot (rq_cap entries).
struct BatchBuffers {
    int32_t n_cap = 0, rq_cap = 0, cap = 0;
    const fmdp_request* rq = nullptr;  // requests on the device (own copy or the staged ones)
    DevArray<fmdp_request> reqs;
    DevArray<float> traj;
    DevArray<uint8_t> acts;
    DevArray<RolloutOut> rout;
    DevArray<SepOut> sepo;
    DevArray<int32_t> idx;   // [3][n_cap] + [rq_cap]
    DevArray<int32_t> ctr;   // queue counter, n_todo, n_unresolved, n_store
    DevArray<uint8_t> infl;  // [n_cap][n_cap]
    DevArray<int32_t> adm;   // admissions of a run, for the minimum-separation epilogue
    PinnedArray<int32_t> h_idx, h_ctr;
    PinnedArray<uint8_t> h_infl;
    PinnedArray<RolloutOut> h_rout;
    PinnedArray<SepOut> h_sep;
    PinnedArray<float> h_traj;
    PinnedArray<uint8_t> h_acts;
    PinnedArray<int32_t> h_acc;  // learned mode: accepted proposals
    void release() {
        reqs.release(); traj.release(); acts.release(); rout.release(); sepo.release(); h_acc.release();
        idx.release(); ctr.release(); infl.release(); adm.release();
        h_idx.release(); h_ctr.release(); h_infl.release(); h_rout.release(); h_sep.release();
        h_traj.release(); h_acts.release();
    }
};

// One instantiated wave graph and the launch parameters it was captured with.
struct WaveGraph {
    std::vector<int64_t> key;
    cudaGraphExec_t exec = nullptr;
};

thread_local std::string g_create_error;

}  // namespace

struct fmdp_ctx {
    Model model{};
    fmdp_airspace air{};
    double gamma = 0.0;
    fmdp_sep sep{};
    fmdp_options opt{};
    int32_t A = 0;

    cudaStream_t own = nullptr;
    cudaStream_t stream = nullptr;
    int device = 0;
    int max_smem = 0;
    int n_sm = 1;

    // device plan table
    float* X = nullptr;
    float* Y = nullptr;
    float* Z = nullptr;
    int32_t T_win = 0, S_pad = 0, S_max = 0;
    Book book;

    float* hm = nullptr;
    double* statics = nullptr;
    int32_t* err = nullptr;

    // spatial index of the plan table (one CSR per ring row)
    bool index_on = false;
    int32_t* ix_cstart = nullptr;
    int32_t* ix_nextra = nullptr;
    int32_t* ix_dirty = nullptr;
    float4* ix_items = nullptr;
    int32_t ix_ncx = 0, ix_ncy = 0, ix_ncell = 0;
    float ix_x0 = 0.f, ix_y0 = 0.f, ix_inv = 0.f, ix_vmax = 0.f;
    size_t ix_smem = 0;
    int32_t icap_user = 0;  // options.index_stage_items (0: tuned or 1536)
    unsigned long long* items_ctr = nullptr;

    // autotuner: the batched indexed rollout's shape per workload key, and the shape a
    // tuning run is timing (0: none)
    std::map<std::array<int32_t, 4>, fmdp_tune_entry> tune;
    int32_t try_threads = 0, try_icap = 0;

    // batch co-simulation: per-step aircraft records and the grid barrier words
    DevArray<double> cs_mem;
    DevArray<int32_t> cs_bar;

    // work buffers
    SeqBuffers seq;     // fmdp_schedule / fmdp_schedule_many
    SeqBuffers stg;     // staged (device-resident) runs
    DevArray<fmdp_request> reqs;
    DevArray<float> traj;
    DevArray<uint8_t> acts;
    DevArray<RolloutOut> rout;
    DevArray<SepOut> sepo;
    DevArray<int32_t> slots;
    DevArray<int64_t> t0s, offs;
    DevArray<int32_t> counts;
    DevArray<double> q_trace, st_trace;
    DevArray<int32_t> hd_trace;
    DevArray<uint8_t> tie_trace;
    PinnedArray<float> h_traj;
    PinnedArray<uint8_t> h_acts;
    PinnedArray<RolloutOut> h_rout;
    PinnedArray<SepOut> h_sep;

    // learned proposal: fp32 parameters, gradients and Adam moments; bf16 copies (training
    // layout and the policy kernel's chunks); the training set; per-request proposal buffers
    bool mlp_ready = false;
    DevArray<float> mlp_p, mlp_g, mlp_m1, mlp_m2;
    DevArray<__nv_bfloat16> mlp_wt, mlp_wp;
    int64_t adam_t = 0;
    DevArray<__nv_bfloat16> tX;
    DevArray<uint8_t> ty;
    int64_t t_rows = 0;
    DevArray<__nv_bfloat16> trX, trH, trdZ;
    DevArray<float> trZ, trdZf, trdH, tr_loss;
    DevArray<int32_t> tr_idx;
    DevArray<uint8_t> tr_y;
    DevArray<float> p_traj;
    DevArray<uint8_t> p_acts;
    DevArray<RolloutOut> p_rout;
    DevArray<SepOut> p_sep;
    DevArray<int32_t> p_acc, p_queue, p_ident;
    DevArray<int64_t> row0;
    bool learned_mode = false;  // the batch in flight takes accepted proposals
    double slack = 0.05;

    // speculative batches
    BatchBuffers bat;
    std::vector<WaveGraph> graphs;  // most recent first
    bool use_graphs = true;
    bool capturing = false;

    // staged (device-resident) requests
    std::vector<fmdp_request> staged;
    int32_t staged_cap = 0;
    bool staged_done = false;
    bool staged_batched = false;
    std::vector<fmdp_result> staged_res;  // batched staged runs: results without points

    // snapshot
    float* sX = nullptr;
    float* sY = nullptr;
    float* sZ = nullptr;
    Book snap;
    bool has_snap = false;

    // profiling
    bool profiling = false;
    bool phase_timing = false;
    DevArray<unsigned long long> phase;
    fmdp_stats stats{};
    std::vector<cudaEvent_t> ev_pool;
    struct Pending { int kind; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    size_t ev_next = 0;

    int last_cs = 1, last_threads = 256, last_chunk = 0;
    std::string err_msg;
};

namespace {

// ------------------------------------------------------------------ model constants

void fill_model(fmdp_ctx* c, const std::vector<fmdp_well>& wells, const std::vector<fmdp_action>& actions,
                const double* host_statics) {
    Model& m = c->model;
    const fmdp_airspace& a = c->air;
    m.box[0] = a.x0; m.box[1] = a.y0; m.box[2] = a.z0;
    m.box[3] = a.x1; m.box[4] = a.y1; m.box[5] = a.z1;
    m.dt = a.dt;
    m.lg64 = std::log2(c->gamma);
    m.lg32 = (float)m.lg64;
    m.goal_reward = c->opt.goal_reward;
    m.log2rg = c->opt.goal_reward > 0.0 ? std::log2(c->opt.goal_reward) : -INFINITY;
    m.clearance = a.clearance_m;
    m.deck = a.deck_value > 0.0 ? a.deck_value : 1000.0;
    m.sep_h = c->sep.horiz_m;
    m.sep_v = c->sep.vert_m;
    m.A = (int32_t)actions.size();
    m.combine = c->opt.combine;
    for (size_t i = 0; i < actions.size(); ++i) {
        m.dh[i] = (int32_t)std::lround(actions[i].dpsi_deg / 15.0);
        m.climb[i] = actions[i].climb_mps;
    }
    m.n_wells = (int32_t)wells.size();
    double rmax = 0.0, magmax = 0.0, taumax = 0.0;
    for (size_t k = 0; k < wells.size(); ++k) {
        const fmdp_well& w = wells[k];
        m.w_tau[k] = (float)w.tau_s;
        m.w_tau64[k] = w.tau_s;
        m.w_R64[k] = w.radius_m;
        m.w_R2[k] = (float)(w.radius_m * w.radius_m);
        m.w_band[k] = kWellBand * m.w_R2[k];
        m.w_L[k] = w.magnitude > 0.0 ? (float)std::log2(w.magnitude) : -INFINITY;
        m.w_lg[k] = (float)std::log2(w.gamma);
        rmax = std::max(rmax, w.radius_m);
        magmax = std::max(magmax, w.magnitude);
        taumax = std::max(taumax, std::fabs(w.tau_s));
    }
    m.reach_base = (float)(rmax + 1.0);
    m.tau_absmax = (float)taumax;
    m.n_static = a.n_static_wells;
    for (int w = 0; w < a.n_static_wells; ++w) {
        const double* s = host_statics + 6 * w;
        m.st_R2[w] = (float)(s[3] * s[3]);
        m.st_band[w] = kWellBand * m.st_R2[w];
        m.st_L[w] = s[4] > 0.0 ? (float)std::log2(s[4]) : -INFINITY;
        m.st_lg[w] = (float)std::log2(s[5]);
        magmax = std::max(magmax, s[4]);
    }
    m.sum_ref = magmax > 0.0 ? (float)std::log2(magmax) : 0.0f;
    m.sum_scale = std::exp2((double)m.sum_ref - (double)kSumBits);
    m.hm_nx = a.heightmap ? a.hm_nx : 0;
    m.hm_ny = a.heightmap ? a.hm_ny : 0;
    m.hm_sx = a.heightmap ? (float)((a.hm_nx - 1) / (a.x1 - a.x0)) : 0.f;
    m.hm_sy = a.heightmap ? (float)((a.hm_ny - 1) / (a.y1 - a.y0)) : 0.f;
    m.hm = c->hm;
    m.statics = c->statics;
}

TableView table_view(fmdp_ctx* c) {
    TableView v;
    v.X = c->X;
    v.Y = c->Y;
    v.Z = c->Z;
    v.T_win = c->T_win;
    v.S_pad = c->S_pad;
    v.t_base = c->book.t_base;
    return v;
}

// ------------------------------------------------------------------ profiling

cudaEvent_t next_event(fmdp_ctx* c) {
    if (c->ev_next == c->ev_pool.size()) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        c->ev_pool.push_back(e);
    }
    return c->ev_pool[c->ev_next++];
}
struct KernelTimer {
    fmdp_ctx* c;
    int kind;
    cudaEvent_t a = nullptr;
    KernelTimer(fmdp_ctx* c_, int k) : c(c_), kind(k) {
        if (c->profiling && kind >= 0) {
            a = next_event(c);
            CK(cudaEventRecord(a, c->stream));
        }
    }
    void stop() {
        if (c->profiling && kind >= 0) {
            cudaEvent_t b = next_event(c);
            CK(cudaEventRecord(b, c->stream));
            c->pending.push_back({kind, a, b});
        }
    }
};
void collect_timers(fmdp_ctx* c) {
    for (auto& p : c->pending) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, p.a, p.b));
        if (p.kind == 0) { c->stats.rollout_ms += ms; c->stats.rollout_launches++; }
        else if (p.kind == 1) { c->stats.sepcheck_ms += ms; c->stats.sepcheck_launches++; }
        else if (p.kind == 2) { c->stats.admit_ms += ms; c->stats.admit_launches++; }
        else { c->stats.influence_ms += ms; c->stats.influence_launches++; }
    }
    c->pending.clear();
    c->ev_next = 0;
}

// ------------------------------------------------------------------ spatial index

constexpr int32_t kExtraLimit = 48;  // appended items per row before the row is rebuilt

IndexArgs index_args(fmdp_ctx* c) {
    IndexArgs a{};
    a.tab = table_view(c);
    a.cstart = c->ix_cstart;
    a.nextra = c->ix_nextra;
    a.dirty = c->ix_dirty;
    a.items = c->ix_items;
    a.ncx = c->ix_ncx;
    a.ncy = c->ix_ncy;
    a.ncell = c->ix_ncell;
    a.x0 = c->ix_x0;
    a.y0 = c->ix_y0;
    a.inv_cell = c->ix_inv;
    a.vmax = c->ix_vmax;
    a.inv_dt = (float)(1.0 / c->air.dt);
    a.extra_limit = kExtraLimit;
    return a;
}

IndexView index_view(fmdp_ctx* c) {
    IndexView v{};
    v.cstart = c->ix_cstart;
    v.nextra = c->ix_nextra;
    v.items = c->ix_items;
    v.ncx = c->ix_ncx;
    v.ncy = c->ix_ncy;
    v.ncell = c->ix_ncell;
    v.x0 = c->ix_x0;
    v.y0 = c->ix_y0;
    v.inv_cell = c->ix_inv;
    v.vmax = c->ix_vmax;
    return v;
}

// launch shape of a rollout
struct Geometry {
    int32_t S_scan, cs, threads, chunk, ring;
    int32_t icap = 0;  // indexed mode: plan samples staged per step
    size_t smem;
};

void set_index_args(fmdp_ctx* c, RolloutArgs& ra, const Geometry& g) {
    ra.indexed = c->index_on ? 1 : 0;
    ra.icap = g.icap;
    ra.iv = index_view(c);
    ra.items_ctr = (c->index_on && c->profiling && !c->capturing) ? c->items_ctr : nullptr;
}

// rebuilds the index rows of steps [a, b) (at most one window length)
void index_rebuild(fmdp_ctx* c, int64_t a, int64_t b, bool dirty_only) {
    if (!c->index_on || b <= a) return;
    const int32_t n = (int32_t)std::min<int64_t>(b - a, c->T_win);
    LAUNCH(c, launch_index_build(index_args(c), a, n, dirty_only ? 1 : 0, c->ix_smem, c->stream));
}
void index_rebuild_all(fmdp_ctx* c) { index_rebuild(c, c->book.t_base, c->book.t_base + c->T_win, false); }
void index_reset(fmdp_ctx* c) {
    if (!c->index_on) return;
    CK(cudaMemsetAsync(c->ix_cstart, 0, ((size_t)c->T_win * (c->ix_ncell + 1) + 16) * sizeof(int32_t), c->stream));
    CK(cudaMemsetAsync(c->ix_nextra, 0, ((size_t)c->T_win + 16) * sizeof(int32_t), c->stream));
    CK(cudaMemsetAsync(c->ix_dirty, 0, (size_t)c->T_win * sizeof(int32_t), c->stream));
}
// Appends admitted trajectories (request work items; see IndexAppendArgs) to the extra
// lists of their rows, then rebuilds the rows that grew past the limit among [a, b).
void index_append_admitted(fmdp_ctx* c, const float* traj, int32_t cap, const RolloutOut* rout,
                           const fmdp_request* reqs, const SepOut* sep, const int32_t* idx, const int32_t* n_dev,
                           int32_t n_items, int64_t a, int64_t b) {
    if (!c->index_on) return;
    IndexAppendArgs ia{};
    ia.ix = index_args(c);
    ia.traj = traj;
    ia.cap = cap;
    ia.rout = rout;
    ia.reqs = reqs;
    ia.sep = sep;
    ia.idx = idx;
    ia.n_dev = n_dev;
    LAUNCH(c, launch_index_append(ia, n_items, cap, c->stream));
    index_rebuild(c, a, b, true);
}

// ------------------------------------------------------------------ launch geometry

// Partition g.S_scan slots over clusters of cs CTAs: the deepest ring (8, else 4 slices)
// whose partition fits one CTA's shared memory. False when neither fits.
bool fit_geometry(fmdp_ctx* c, Geometry& g, int cs) {
    g.cs = cs;
    g.chunk = std::max(32, round_up((g.S_scan + cs - 1) / cs, 32));
    g.threads = c->opt.threads_per_cta > 0 ? c->opt.threads_per_cta : (g.chunk > 256 ? 384 : 256);
    for (int depth : {8, 4}) {
        g.ring = depth;
        g.smem = rollout_smem_bytes(g.chunk, depth, 0);
        if ((int)g.smem <= c->max_smem) return true;
    }
    return false;
}

// autotuner key of the current table and batch size
int32_t bit_length(int64_t v) {
    int32_t b = 0;
    while (v > 0) {
        ++b;
        v >>= 1;
    }
    return b;
}
int32_t batch_size_of(const fmdp_ctx* c) { return c->opt.batch_size > 0 ? c->opt.batch_size : 256; }
// lookahead window of the rollouts (Sec. IV "Forward project"); 1 is the one-step rule
int32_t window_of(const fmdp_ctx* c) { return c->opt.lookahead_W > 1 ? c->opt.lookahead_W : 1; }

// The lookahead rollout of one request (W > 1), written like the rollout kernel's.
void launch_window_rollout(fmdp_ctx* c, const Geometry& g, const fmdp_request* req_dev, int32_t cap, float* traj,
                           uint8_t* acts, RolloutOut* out, bool trace) {
    LookArgs la{};
    la.m = c->model;
    la.tab = table_view(c);
    la.S_scan = g.S_scan;
    la.W = window_of(c);
    la.cap = cap;
    la.n_req = 1;
    la.trace = trace ? 1 : 0;
    la.reqs = req_dev;
    la.traj = traj;
    la.acts = acts;
    la.out = out;
    if (trace) {
        la.q_trace = c->q_trace.p;
        la.st_trace = c->st_trace.p;
        la.hd_trace = c->hd_trace.p;
        la.tie_trace = c->tie_trace.p;
    }
    LAUNCH(c, launch_lookahead(la, c->stream));
}
std::array<int32_t, 4> tune_key(const fmdp_ctx* c, int32_t wave) {
    return {c->A, c->opt.combine, bit_length((int64_t)c->book.plans.size()), bit_length(wave)};
}
// the cached shape for a wave of `wave` rollouts: its own bucket, else the nearest tuned one
const fmdp_tune_entry* tune_lookup(const fmdp_ctx* c, int32_t wave) {
    const auto k = tune_key(c, wave);
    const fmdp_tune_entry* best = nullptr;
    int32_t bd = INT_MAX;
    for (const auto& kv : c->tune) {
        if (kv.first[0] != k[0] || kv.first[1] != k[1] || kv.first[2] != k[2]) continue;
        const int32_t d = std::abs(kv.first[3] - k[3]);
        if (d < bd) {
            bd = d;
            best = &kv.second;
        }
    }
    return best;
}

// Indexed geometry: one CTA per request staging only the plans near its state. A batched
// launch of `wave` rollouts takes the autotuner's shape for its key; explicit options take
// precedence.
Geometry geometry_indexed(fmdp_ctx* c, int32_t S_scan, int32_t wave = 0) {
    Geometry g;
    g.S_scan = S_scan;
    g.cs = 1;
    g.chunk = 0;
    g.ring = 4;
    g.threads = 384;
    g.icap = 1536;
    if (wave > 0) {
        if (const fmdp_tune_entry* e = tune_lookup(c, wave)) {
            g.threads = e->threads_per_cta;
            g.icap = e->index_stage_items;
        }
        if (c->try_threads > 0) {
            g.threads = c->try_threads;
            g.icap = c->try_icap;
        }
    }
    if (c->opt.threads_per_cta > 0) g.threads = c->opt.threads_per_cta;
    if (c->icap_user > 0) g.icap = c->icap_user;
    g.smem = rollout_smem_bytes(0, 0, g.icap);
    require((int)g.smem <= c->max_smem, FMDP_ERR_ARG, "index staging buffers exceed shared memory");
    c->last_cs = 1;
    c->last_threads = g.threads;
    c->last_chunk = 0;
    return g;
}

// Latency geometry (one request at a time): about 1024 slots per CTA.
Geometry geometry(fmdp_ctx* c, int32_t S_hw) {
    if (c->index_on) return geometry_indexed(c, round_up(std::max(S_hw, 0), 32));
    Geometry g;
    g.S_scan = round_up(std::max(S_hw, 0), 32);
    int cs = c->opt.cluster_size;
    if (cs <= 0) {
        const int want = (g.S_scan + 1023) / 1024;
        cs = 1;
        while (cs < want && cs < kMaxCluster) cs *= 2;
    }
    cs = std::max(1, std::min(cs, kMaxCluster));
    auto fit = [&](int cs_) { return fit_geometry(c, g, cs_); };
    while (!fit(cs) && cs < kMaxCluster) cs *= 2;  // partition too large: spread it wider
    require((int)g.smem <= c->max_smem, FMDP_ERR_ARG, "plan table partition exceeds shared memory");
    // the cluster must fit on one GPC: halve it until the hardware can place one
    while (g.cs > 1 && rollout_max_active_clusters(g.cs, g.threads, g.smem) < 1) {
        require(fit(g.cs / 2), FMDP_ERR_ARG, "plan table partition exceeds shared memory");
    }
    c->last_cs = g.cs;
    c->last_threads = g.threads;
    c->last_chunk = g.chunk;
    return g;
}

void check_request(fmdp_ctx* c, const fmdp_request& r) {
    require(std::isfinite(r.ox) && std::isfinite(r.oy) && std::isfinite(r.oz) && std::isfinite(r.gx) &&
                std::isfinite(r.gy) && std::isfinite(r.gz),
            FMDP_ERR_ARG, "request coordinates must be finite");
    require(std::isfinite(r.speed_mps) && r.speed_mps > 0.0, FMDP_ERR_ARG, "request speed must be > 0");
    require(r.horizon >= 0 && r.horizon < (1 << 24), FMDP_ERR_ARG, "request horizon out of range");
    const int64_t lo = c->book.t_base, hi = c->book.t_base + c->T_win;
    require(r.depart_step >= lo && r.depart_step + (int64_t)r.horizon < hi, FMDP_ERR_RANGE,
            "request steps fall outside the plan-table window");
}

int32_t take_slot(fmdp_ctx* c) {
    require(!c->book.free_slots.empty(), FMDP_ERR_FULL, "no free plan slot");
    const int32_t s = *c->book.free_slots.begin();
    c->book.free_slots.erase(c->book.free_slots.begin());
    return s;
}

void recompute_hw(fmdp_ctx* c) {
    int32_t hw = 0;
    for (auto& kv : c->book.plans) hw = std::max(hw, kv.second.slot + 1);
    c->book.S_hw = hw;
}

// Enqueue rollout -> sep_check -> admission for n requests (device array c->reqs, slots in
// c->slots) in FCFS order on the context's stream.
void enqueue_sequence(fmdp_ctx* c, SeqBuffers& B, const fmdp_request* host_reqs, int32_t n, int32_t cap,
                      const Geometry& g, bool plan = true) {
    const TableView tv = table_view(c);
    LAUNCH(c, launch_sep_reset(B.sepo.p, n, c->stream));
    for (int32_t i = 0; i < n; ++i) {
        RolloutArgs ra{};
        ra.m = c->model;
        ra.tab = tv;
        ra.S_scan = g.S_scan;
        ra.chunk = g.chunk;
        ra.cs = g.cs;
        ra.ring = g.ring;
        ra.cap = cap;
        ra.reqs = B.reqs.p + i;
        ra.n_req = 1;
        ra.trace = 0;
        ra.traj = B.traj.p + (size_t)i * cap * 3;
        ra.acts = B.acts.p + (size_t)i * cap;
        ra.out = B.rout.p + i;
        ra.err = c->err;
        set_index_args(c, ra, g);
        ra.phase = c->phase_timing ? c->phase.p : nullptr;
        if (plan) {
            KernelTimer t(c, 0);
            if (window_of(c) > 1)
                launch_window_rollout(c, g, ra.reqs, cap, ra.traj, ra.acts, ra.out, false);
            else
                LAUNCH(c, launch_rollout(ra, g.threads, g.smem, c->stream));
            t.stop();
        }
        SepArgs sa{};
        sa.m = c->model;
        sa.tab = tv;
        sa.S_scan = g.S_scan;
        sa.cap = cap;
        sa.traj = ra.traj;
        sa.rout = ra.out;
        sa.reqs = ra.reqs;
        sa.out = B.sepo.p + i;
        {
            KernelTimer t(c, 1);
            LAUNCH(c, launch_sepcheck(sa, 1, cap, c->stream));
            t.stop();
        }
        AdmitArgs aa{};
        aa.err = c->err;
        aa.tab = tv;
        aa.cap = cap;
        aa.traj = ra.traj;
        aa.rout = ra.out;
        aa.reqs = ra.reqs;
        aa.slots = B.slots.p + i;
        aa.sep = sa.out;
        aa.force = 0;
        {
            KernelTimer t(c, 2);
            LAUNCH(c, launch_admit(aa, 1, cap, c->stream));
            t.stop();
        }
        // an admitted trajectory joins the index before the next request plans
        const int64_t d0 = host_reqs[i].depart_step;
        index_append_admitted(c, ra.traj, cap, ra.out, ra.reqs, sa.out, nullptr, nullptr, 1, d0,
                              d0 + host_reqs[i].horizon + 1);
    }
}

int32_t read_error_word(fmdp_ctx* c) {
    int32_t e = 0;
    CK(cudaMemcpyAsync(&e, c->err, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (e != 0) {
        CK(cudaMemsetAsync(c->err, 0, sizeof(int32_t), c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return e;
}

void fill_result(const RolloutOut& ro, const SepOut& so, fmdp_result* res) {
    res->verdict = so.verdict >= 0 ? so.verdict : (ro.status == kStatusCaptured ? FMDP_ADMITTED : ro.status);
    res->n_points = ro.n_points;
    res->first_conflict_step = so.first_conflict == INT_MAX ? -1 : so.first_conflict;
    res->first_terrain_step = so.first_terrain == INT_MAX ? -1 : so.first_terrain;
    float mh, mv;
    std::memcpy(&mh, &so.min_h_bits, 4);
    std::memcpy(&mv, &so.min_v_bits, 4);
    res->min_sep_h = mh;
    res->min_sep_v = mv;
    res->near_ties = ro.near_ties;
}

// Plans n requests (already validated) in FCFS order; results and trajectories to the
// caller's buffers when res != nullptr. With staged = true the requests already sit in
// c->stg.reqs on the device and trajectories stay there. Returns the number admitted.
int32_t run_fcfs(fmdp_ctx* c, const fmdp_request* reqs, int32_t n, fmdp_result* res, bool staged,
                 bool cosim = false, int32_t absent = 0) {
    SeqBuffers& B = staged ? c->stg : c->seq;
    const bool keep_on_device = staged;
    int32_t admitted = 0;
    int32_t done = 0;
    while (done < n) {
        const int32_t m = std::min<int32_t>(n - done, (int32_t)c->book.free_slots.size());
        require(m > 0, FMDP_ERR_FULL, "no free plan slot");
        std::vector<int32_t> sl(m);
        int32_t hw = c->book.S_hw;
        int32_t cap = 1;
        for (int32_t i = 0; i < m; ++i) {
            sl[i] = take_slot(c);
            hw = std::max(hw, sl[i] + 1);
            cap = std::max(cap, reqs[done + i].horizon + 1);
        }
        try {
            const Geometry g = geometry(c, hw);
            if (staged) {
                require(m == n && done == 0, FMDP_ERR_FULL, "not enough free slots for the staged run");
            } else {
                B.reqs.ensure(m);
                B.traj.ensure((size_t)m * cap * 3);
                B.acts.ensure((size_t)m * cap);
                B.rout.ensure(m);
                B.sepo.ensure(m);
                CK(cudaMemcpyAsync(B.reqs.p, reqs + done, m * sizeof(fmdp_request), cudaMemcpyHostToDevice,
                                   c->stream));
            }
            B.slots.ensure(m);
            CK(cudaMemcpyAsync(B.slots.p, sl.data(), m * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
            if (cosim) {  // all m requests fly together first; admission below in array order
                require(m == n, FMDP_ERR_FULL, "not enough free slots for the co-simulated batch");
                c->cs_mem.ensure((size_t)2 * n * 8);
                c->cs_bar.ensure(2);
                CK(cudaMemsetAsync(c->cs_bar.p, 0, 2 * sizeof(int32_t), c->stream));
                LookArgs la{};
                la.m = c->model;
                la.tab = table_view(c);
                la.S_scan = g.S_scan;
                la.W = window_of(c);
                la.cap = cap;
                la.n_req = n;
                la.reqs = B.reqs.p;
                la.traj = B.traj.p;
                la.acts = B.acts.p;
                la.out = B.rout.p;
                la.err = c->err;
                la.cosim = 1;
                la.t_start = reqs[0].depart_step;
                for (int32_t i = 1; i < n; ++i) la.t_start = std::min(la.t_start, reqs[i].depart_step);
                la.mem = c->cs_mem.p;
                la.bar = c->cs_bar.p;
                la.absent = absent;
                KernelTimer t(c, 0);
                LAUNCH(c, launch_lookahead(la, c->stream));
                t.stop();
            }
            enqueue_sequence(c, B, reqs + done, m, cap, g, !cosim);
            c->h_rout.ensure(m);
            c->h_sep.ensure(m);
            CK(cudaMemcpyAsync(c->h_rout.p, B.rout.p, m * sizeof(RolloutOut), cudaMemcpyDeviceToHost, c->stream));
            CK(cudaMemcpyAsync(c->h_sep.p, B.sepo.p, m * sizeof(SepOut), cudaMemcpyDeviceToHost, c->stream));
            if (res && !keep_on_device) {
                c->h_traj.ensure((size_t)m * cap * 3);
                c->h_acts.ensure((size_t)m * cap);
                CK(cudaMemcpyAsync(c->h_traj.p, B.traj.p, (size_t)m * cap * 3 * sizeof(float),
                                   cudaMemcpyDeviceToHost, c->stream));
                CK(cudaMemcpyAsync(c->h_acts.p, B.acts.p, (size_t)m * cap, cudaMemcpyDeviceToHost, c->stream));
            }
            CK(cudaStreamSynchronize(c->stream));
            if (c->profiling) collect_timers(c);
            const int32_t ew = read_error_word(c);
            require(ew == 0, FMDP_ERR_TIMEOUT, "a bounded device wait expired during a rollout");
        } catch (...) {
            for (int32_t s : sl) c->book.free_slots.insert(s);
            throw;
        }
        for (int32_t i = 0; i < m; ++i) {
            const RolloutOut& ro = c->h_rout.p[i];
            const SepOut& so = c->h_sep.p[i];
            const fmdp_request& rq = reqs[done + i];
            c->stats.rollout_steps += ro.steps;
            c->stats.slots_scanned += (int64_t)ro.steps * round_up(std::max(hw, 0), 32);
            c->stats.sep_pairs += (int64_t)ro.n_points * round_up(std::max(hw, 0), 32);
            uint64_t id = 0;
            if (so.verdict == FMDP_ADMITTED) {
                id = c->book.next_id++;
                c->book.plans[id] = PlanMeta{sl[i], rq.depart_step, ro.n_points};
                c->book.S_hw = std::max(c->book.S_hw, sl[i] + 1);
                ++admitted;
            } else {
                c->book.free_slots.insert(sl[i]);
            }
            if (res) {
                fmdp_result* o = res + done + i;
                fill_result(ro, so, o);
                o->plan_id = id;
                o->replanned = 0;
                if (!keep_on_device) {
                    if (o->xyz)
                        std::memcpy(o->xyz, c->h_traj.p + (size_t)i * cap * 3, (size_t)ro.n_points * 3 * sizeof(float));
                    if (o->actions && ro.n_points > 1)
                        std::memcpy(o->actions, c->h_acts.p + (size_t)i * cap, (size_t)(ro.n_points - 1));
                }
            }
        }
        if (keep_on_device) c->staged_cap = cap;
        done += m;
    }
    return admitted;
}

// ------------------------------------------------------------------ speculative batches
//
// A batch is planned in waves. Every wave plans its work items concurrently against the
// table as it stands (one persistent rollout launch pulling items from a queue), checks
// their separation, and tests every pair of unresolved requests for influence. The host
// then walks the unresolved requests in arrival order: a request is final when no request
// admitted earlier in the same walk influences it, and the walk stops at the first one
// that is influenced. Admitted requests are stored at the start of the next wave; a
// request left unresolved is planned again only if one of them influences it, otherwise
// its plan stays exact against the grown table. Each wave finalises at least one request.

constexpr int32_t kBatchDefault = 256;
constexpr int32_t kBatchMax = 1024;
// kernels of one wave: admit, reset, rollout, sep_check, influence (+ index append, rebuild)
int wave_kernels(const fmdp_ctx* c) { return (c->index_on ? 7 : 5) + (c->learned_mode ? 4 : 0); }

// Batch geometry: the narrowest cluster whose partition fits one CTA's shared memory, so
// that as many rollouts as possible run side by side.
Geometry geometry_batch(fmdp_ctx* c, int32_t S, int32_t wave) {
    if (c->index_on) return geometry_indexed(c, std::min(round_up(std::max(S, 0), 32), c->S_pad), std::max(wave, 1));
    Geometry g;
    g.S_scan = std::min(round_up(std::max(S, 0), 32), c->S_pad);
    int cs = c->opt.cluster_size > 0 ? c->opt.cluster_size : 1;
    while (!(fit_geometry(c, g, cs) && rollout_max_active_clusters(cs, g.threads, g.smem) >= 1)) {
        require(cs < kMaxCluster, FMDP_ERR_ARG, "plan table partition exceeds shared memory");
        cs *= 2;
    }
    c->last_cs = g.cs;
    c->last_threads = g.threads;
    c->last_chunk = g.chunk;
    return g;
}

int32_t host_verdict(const RolloutOut& ro, const SepOut& so) {  // the admission kernel's rule
    if (ro.status != kStatusCaptured) return ro.status;
    if (so.first_conflict != INT_MAX) return FMDP_REJ_CONFLICT;
    if (so.first_terrain != INT_MAX) return FMDP_REJ_TERRAIN;
    return FMDP_ADMITTED;
}

// One wave on the context's stream: store the requests admitted by the previous walk,
// plan the work items, check their separation, test influence among the unresolved
// requests, and bring rollout, separation and influence results back to pinned memory.
// Every count is read on the device, so the sequence can be captured once and replayed.
size_t idx_words(const BatchBuffers& B) { return 3 * (size_t)B.n_cap + B.rq_cap; }

double climb_step(const fmdp_ctx* c) {
    double m = 0.0;
    for (int i = 0; i < c->model.A; ++i) m = std::max(m, std::fabs(c->model.climb[i] * c->model.dt));
    return m;
}

void enqueue_wave(fmdp_ctx* c, const Geometry& g, int n_clusters, BatchBuffers& B, bool timed) {
    const int32_t n_cap = B.n_cap, cap = B.cap;
    cudaStream_t s = c->stream;
    int32_t* todo = B.idx.p;
    int32_t* unres = todo + n_cap;
    int32_t* store = unres + n_cap;
    int32_t* slots = store + n_cap;
    const TableView tv = table_view(c);
    CK(cudaMemcpyAsync(B.idx.p, B.h_idx.p, idx_words(B) * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(B.ctr.p, B.h_ctr.p, 4 * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    {
        AdmitArgs aa{};
        aa.err = c->err;
        aa.tab = tv;
        aa.cap = cap;
        aa.traj = B.traj.p;
        aa.rout = B.rout.p;
        aa.reqs = B.rq;
        aa.slots = slots;
        aa.sep = B.sepo.p;
        aa.force = 0;
        aa.idx = store;
        aa.n_dev = B.ctr.p + 3;
        KernelTimer t(c, timed ? 2 : -1);
        LAUNCH(c, launch_admit(aa, n_cap, cap, s));
        t.stop();
        index_append_admitted(c, B.traj.p, cap, B.rout.p, B.rq, B.sepo.p, store, B.ctr.p + 3, n_cap,
                              c->book.t_base, c->book.t_base + c->T_win);
    }
    LAUNCH(c, launch_sep_reset_idx(B.sepo.p, todo, B.ctr.p + 1, n_cap, s));
    if (c->learned_mode) {
        // proposals for the work items, their separation check, and the judge, which copies
        // accepted proposals over the items' FastMDP buffers and marks them to skip FastMDP
        LAUNCH(c, launch_sep_reset_idx(c->p_sep.p, todo, B.ctr.p + 1, n_cap, s));
        CK(cudaMemsetAsync(c->p_queue.p, 0, sizeof(int32_t), s));
        PolicyArgs pa{};
        pa.m = c->model;
        pa.tab = tv;
        pa.iv = index_view(c);
        pa.Wp = c->mlp_wp.p;
        pa.params = c->mlp_p.p;
        pa.reqs = B.rq;
        pa.idx = todo;
        pa.n_items = n_cap;
        pa.n_dev = B.ctr.p + 1;
        pa.queue = c->p_queue.p;
        pa.cap = cap;
        pa.traj = c->p_traj.p;
        pa.acts = c->p_acts.p;
        pa.out = c->p_rout.p;
        pa.err = c->err;
        pa.rows = policy_rows_for(n_cap, c->n_sm);
        pa.step_bound = 1;  // learned FCFS: proposals beyond the judge's bound are never taken
        pa.slack = c->slack;
        pa.climb_step = climb_step(c);
        LAUNCH(c, launch_policy(pa, std::min(c->n_sm, (n_cap + pa.rows - 1) / pa.rows), s));
        SepRowsArgs sp{};
        sp.m = c->model;
        sp.tab = tv;
        sp.S_scan = g.S_scan;
        sp.traj = c->p_traj.p;
        sp.cap = cap;
        sp.rout = c->p_rout.p;
        sp.reqs = B.rq;
        sp.idx = todo;
        sp.n_dev = B.ctr.p + 1;
        sp.n_max = n_cap;
        sp.out = c->p_sep.p;
        if (c->index_on) {
            sp.items = c->ix_items;
            sp.cstart = c->ix_cstart;
            sp.nextra = c->ix_nextra;
            sp.ncell = c->ix_ncell;
        }
        LAUNCH(c, launch_sepcheck_rows(sp, s));
        JudgeArgs ja{};
        ja.reqs = B.rq;
        ja.idx = todo;
        ja.n_dev = B.ctr.p + 1;
        ja.n = n_cap;
        ja.traj_p = c->p_traj.p;
        ja.acts_p = c->p_acts.p;
        ja.rout_p = c->p_rout.p;
        ja.sep_p = c->p_sep.p;
        ja.traj = B.traj.p;
        ja.acts = B.acts.p;
        ja.rout = B.rout.p;
        ja.sep = B.sepo.p;
        ja.accepted = c->p_acc.p;
        ja.cap = cap;
        ja.dt = c->air.dt;
        ja.slack = c->slack;
        ja.climb_step = climb_step(c);
        LAUNCH(c, launch_judge(ja, cap, s));
    }
    {
        RolloutArgs ra{};
        ra.m = c->model;
        ra.tab = tv;
        ra.S_scan = g.S_scan;
        ra.chunk = g.chunk;
        ra.cs = g.cs;
        ra.ring = g.ring;
        ra.cap = cap;
        ra.reqs = B.rq;
        ra.n_req = n_cap;
        ra.traj = B.traj.p;
        ra.acts = B.acts.p;
        ra.out = B.rout.p;
        ra.err = c->err;
        set_index_args(c, ra, g);
        ra.phase = (timed && c->phase_timing) ? c->phase.p : nullptr;
        ra.queue = B.ctr.p;
        ra.idx = todo;
        ra.n_dev = B.ctr.p + 1;
        ra.skip = c->learned_mode ? c->p_acc.p : nullptr;
        KernelTimer t(c, timed ? 0 : -1);
        if (window_of(c) > 1) {  // lookahead rollouts (Sec. IV): one CTA per work item
            LookArgs la{};
            la.m = c->model;
            la.tab = tv;
            la.S_scan = g.S_scan;
            la.W = window_of(c);
            la.cap = cap;
            la.n_req = n_cap;
            la.reqs = B.rq;
            la.traj = B.traj.p;
            la.acts = B.acts.p;
            la.out = B.rout.p;
            la.err = c->err;
            la.idx = todo;
            la.n_dev = B.ctr.p + 1;
            LAUNCH(c, launch_lookahead(la, s));
        } else {
            LAUNCH(c, launch_rollout(ra, g.threads, g.smem, s, n_clusters));
        }
        t.stop();
    }
    {
        SepRowsArgs sa{};
        sa.m = c->model;
        sa.tab = tv;
        sa.S_scan = g.S_scan;
        sa.traj = B.traj.p;
        sa.cap = cap;
        sa.rout = B.rout.p;
        sa.reqs = B.rq;
        sa.idx = todo;
        sa.n_dev = B.ctr.p + 1;
        sa.n_max = n_cap;
        sa.out = B.sepo.p;
        sa.skip = c->learned_mode ? c->p_acc.p : nullptr;
        if (c->index_on) {
            sa.items = c->ix_items;
            sa.cstart = c->ix_cstart;
            sa.nextra = c->ix_nextra;
            sa.ncell = c->ix_ncell;
        }
        KernelTimer t(c, timed ? 1 : -1);
        LAUNCH(c, launch_sepcheck_rows(sa, s));
        t.stop();
    }
    {
        InfluenceArgs ia{};
        ia.traj = B.traj.p;
        ia.rout = B.rout.p;
        ia.reqs = B.rq;
        ia.cap = cap;
        ia.idx = unres;
        ia.n_dev = B.ctr.p + 2;
        ia.reach_base = c->model.reach_base;
        ia.tau_absmax = c->model.tau_absmax;
        ia.W = window_of(c);
        ia.n_wells = c->model.n_wells;
        for (int k = 0; k < c->model.n_wells; ++k) {
            ia.w_tau[k] = c->model.w_tau[k];
            ia.w_R[k] = (float)c->model.w_R64[k];
        }
        if (c->learned_mode) {  // a proposal also reads the plan samples within the feature radius
            ia.feat_r = kRF + 1.0f;
            ia.traj_p = c->p_traj.p;
            ia.rout_p = c->p_rout.p;
            ia.accepted = c->p_acc.p;
        }
        float dzmax = 0.f;
        for (int i = 0; i < c->model.A; ++i) dzmax = std::max(dzmax, (float)std::fabs(c->model.climb[i] * c->model.dt));
        ia.dzmax = dzmax;
        ia.sep_h = (float)c->sep.horiz_m;
        ia.sep_v = (float)c->sep.vert_m;
        ia.dt = (float)c->model.dt;
        ia.out = B.infl.p;
        ia.n_cap = n_cap;
        KernelTimer t(c, timed ? 3 : -1);
        LAUNCH(c, launch_influence(ia, n_cap, cap, s));
        t.stop();
    }
    CK(cudaMemcpyAsync(B.h_rout.p, B.rout.p, B.rq_cap * sizeof(RolloutOut), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(B.h_sep.p, B.sepo.p, B.rq_cap * sizeof(SepOut), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(B.h_infl.p, B.infl.p, (size_t)n_cap * n_cap, cudaMemcpyDeviceToHost, s));
    if (c->learned_mode)
        CK(cudaMemcpyAsync(B.h_acc.p, c->p_acc.p, B.rq_cap * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
}

// The wave sequence as an instantiated CUDA graph, captured on a private stream the first
// time these launch parameters occur and replayed on the context's stream afterwards.
cudaGraphExec_t wave_graph(fmdp_ctx* c, const Geometry& g, int n_clusters, BatchBuffers& B) {
    const TableView tv = table_view(c);
    const std::vector<int64_t> key = {g.S_scan, g.cs, g.threads, g.chunk, g.ring, (int64_t)g.smem, n_clusters,
                                      B.n_cap, B.rq_cap, B.cap, (int64_t)(uintptr_t)B.idx.p,
                                      (int64_t)(uintptr_t)B.traj.p, (int64_t)(uintptr_t)B.rq,
                                      (int64_t)(uintptr_t)B.rout.p, (int64_t)(uintptr_t)B.h_idx.p,
                                      (int64_t)(uintptr_t)B.h_infl.p, (int64_t)(uintptr_t)tv.X, tv.t_base,
                                      c->learned_mode ? 1 : 0, (int64_t)(uintptr_t)c->p_traj.p,
                                      (int64_t)(uintptr_t)c->p_acc.p, (int64_t)(c->slack * 1e9)};
    for (size_t i = 0; i < c->graphs.size(); ++i)
        if (c->graphs[i].key == key) {
            std::swap(c->graphs[i], c->graphs[0]);
            return c->graphs[0].exec;
        }
    cudaStream_t cap_stream = nullptr;
    CK(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));
    cudaStream_t user = c->stream;
    c->stream = cap_stream;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        c->capturing = true;
        try {
            enqueue_wave(c, g, n_clusters, B, false);
        } catch (...) {
            c->capturing = false;
            cudaStreamEndCapture(cap_stream, &graph);
            if (graph) cudaGraphDestroy(graph);
            c->stream = user;
            cudaStreamDestroy(cap_stream);
            throw;
        }
        c->capturing = false;
        e = cudaStreamEndCapture(cap_stream, &graph);
    }
    c->stream = user;
    cudaStreamDestroy(cap_stream);
    CK(e);
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(e);
    c->graphs.insert(c->graphs.begin(), WaveGraph{key, exec});
    while (c->graphs.size() > 8) {
        cudaGraphExecDestroy(c->graphs.back().exec);
        c->graphs.pop_back();
    }
    return exec;
}

// The speculative state of one call (batches or a serving run): the unresolved requests in
// arrival order (U), those to plan in the next wave (todo), the previous walk's admissions
// still to store, and each request's outcome. Request numbers are the call's (0 .. n-1).
struct Speculator {
    fmdp_ctx* c;
    BatchBuffers& B;
    const fmdp_request* reqs;  // host copies, all requests of the call
    Geometry g;
    int n_clusters = 1;
    bool graphs = false;
    std::vector<int32_t> U, todo, store, adm_all;
    std::vector<int32_t> slot_of, replans, verdict;
    std::vector<uint64_t> ids;
    std::vector<RolloutOut> fin_ro;
    std::vector<std::pair<uint64_t, int32_t>> pending;  // admitted, not yet stored: (id, slot)
    int32_t admitted = 0;
    size_t group = 1;  // work items per request (departure variants), added and resolved together

    Speculator(fmdp_ctx* c_, const fmdp_request* reqs_, int32_t n)
        : c(c_), B(c_->bat), reqs(reqs_), slot_of(n, -1), replans(n, 0), verdict(n, -1), ids(n, 0), fin_ro(n) {}

    void set_geometry(const Geometry& g_) {
        g = g_;
        n_clusters = std::max(1, std::min(B.n_cap, rollout_max_active_clusters(g.cs, g.threads, g.smem)));
        graphs = c->use_graphs && !c->profiling;
    }
    void add(int32_t r) {  // a request joins the end of the unresolved list
        U.push_back(r);
        todo.push_back(r);
    }
    void upload_lists() {
        const int32_t n_cap = B.n_cap;
        int32_t* hi = B.h_idx.p;
        std::copy(todo.begin(), todo.end(), hi);
        std::copy(U.begin(), U.end(), hi + n_cap);
        std::copy(store.begin(), store.end(), hi + 2 * n_cap);
        for (int32_t r : store) hi[3 * n_cap + r] = slot_of[r];
        B.h_ctr.p[0] = 0;
        B.h_ctr.p[1] = (int32_t)todo.size();
        B.h_ctr.p[2] = (int32_t)U.size();
        B.h_ctr.p[3] = (int32_t)store.size();
    }
    // One wave and its walk: `resolved` receives the requests finalised, in order.
    void wave(std::vector<int32_t>& resolved) {
        const int32_t n_cap = B.n_cap;
        if (c->index_on) {  // the tuned shape for this wave's size
            const Geometry gw = geometry_batch(c, c->S_pad, (int32_t)todo.size());
            if (gw.threads != g.threads || gw.icap != g.icap) set_geometry(gw);
        }
        upload_lists();
        if (graphs) {
            CK(cudaGraphLaunch(wave_graph(c, g, n_clusters, B), c->stream));
            c->stats.kernel_launches += wave_kernels(c);
        } else {
            enqueue_wave(c, g, n_clusters, B, true);
        }
        CK(cudaStreamSynchronize(c->stream));
        if (c->profiling) collect_timers(c);
        require(read_error_word(c) == 0, FMDP_ERR_TIMEOUT, "a bounded device wait expired during a rollout");
        pending.clear();  // the previous walk's admissions are now in the table
        c->stats.batch_waves++;
        for (int32_t r : todo) {
            if (c->learned_mode && B.h_acc.p[r]) continue;  // no FastMDP rollout ran
            const RolloutOut& ro = B.h_rout.p[r];
            c->stats.rollout_steps += ro.steps;
            c->stats.slots_scanned += (int64_t)ro.steps * g.S_scan;
            c->stats.sep_pairs += (int64_t)ro.n_points * g.S_scan;
            c->stats.batch_rollouts++;
        }
        // walk the unresolved requests in arrival order, a group of `group` consecutive work
        // items at a time: a group is final when no admission earlier in the walk influences
        // any of its items, and only its first admissible item is admitted
        store.clear();
        std::vector<size_t> adm_pos;  // positions in U admitted by this walk
        size_t pos = 0;
        for (; pos < U.size(); pos += group) {
            bool hit = false;
            for (size_t q = pos; q < pos + group; ++q) {
                const uint8_t* row = B.h_infl.p + q * n_cap;
                for (size_t v : adm_pos) hit = hit || row[v];
            }
            if (hit) break;
            size_t pick = SIZE_MAX;
            for (size_t q = pos; q < pos + group; ++q) {
                const int32_t k = U[q];
                fin_ro[k] = B.h_rout.p[k];
                verdict[k] = host_verdict(fin_ro[k], B.h_sep.p[k]);
                if (pick == SIZE_MAX && verdict[k] == FMDP_ADMITTED) pick = q;
            }
            for (size_t q = pos; q < pos + group; ++q) {
                const int32_t k = U[q];
                if (q == pick) {
                    const int32_t slot = take_slot(c);
                    require(slot < g.S_scan, FMDP_ERR_ARG, "internal: batch slot beyond the scanned range");
                    const uint64_t id = c->book.next_id++;
                    c->book.plans[id] = PlanMeta{slot, reqs[k].depart_step, fin_ro[k].n_points};
                    c->book.S_hw = std::max(c->book.S_hw, slot + 1);
                    pending.push_back({id, slot});
                    slot_of[k] = slot;
                    ids[k] = id;
                    store.push_back(k);
                    adm_all.push_back(k);
                    adm_pos.push_back(q);
                    ++admitted;
                }
                resolved.push_back(k);
            }
        }
        // what stays unresolved is planned again only where an admission may change it
        std::vector<int32_t> nU, ntodo;
        for (size_t w = pos; w < U.size(); ++w) {
            const uint8_t* row = B.h_infl.p + w * n_cap;
            bool hit = false;
            for (size_t v : adm_pos) hit = hit || row[v];
            nU.push_back(U[w]);
            if (hit) {
                ntodo.push_back(U[w]);
                ++replans[U[w]];
                c->stats.batch_replans++;
            }
        }
        U.swap(nU);
        todo.swap(ntodo);
    }
    // Stores the last walk's admissions, then folds the admissions of requests [k0, k0 + n)'s
    // own run into their minimum separations and brings their reports back.
    void finish(int32_t k0, int32_t n) {
        const int32_t n_cap = B.n_cap;
        std::copy(store.begin(), store.end(), B.h_idx.p + 2 * n_cap);
        for (int32_t r : store) B.h_idx.p[3 * n_cap + r] = slot_of[r];
        B.h_ctr.p[3] = (int32_t)store.size();
        CK(cudaMemcpyAsync(B.idx.p, B.h_idx.p, idx_words(B) * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(B.ctr.p, B.h_ctr.p, 4 * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
        if (!store.empty()) {
            AdmitArgs aa{};
            aa.err = c->err;
            aa.tab = table_view(c);
            aa.cap = B.cap;
            aa.traj = B.traj.p;
            aa.rout = B.rout.p;
            aa.reqs = B.rq;
            aa.slots = B.idx.p + 3 * n_cap;
            aa.sep = B.sepo.p;
            aa.idx = B.idx.p + 2 * n_cap;
            aa.n_dev = B.ctr.p + 3;
            KernelTimer t(c, 2);
            LAUNCH(c, launch_admit(aa, n_cap, B.cap, c->stream));
            t.stop();
            index_append_admitted(c, B.traj.p, B.cap, B.rout.p, B.rq, B.sepo.p, aa.idx, aa.n_dev, n_cap,
                                  c->book.t_base, c->book.t_base + c->T_win);
        }
        // the admission list may be longer than the index block's first array: own buffer
        B.adm.ensure(std::max<size_t>(adm_all.size(), 1));
        if (!adm_all.empty())
            CK(cudaMemcpyAsync(B.adm.p, adm_all.data(), adm_all.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                               c->stream));
        MinSepArgs ma{};
        ma.traj = B.traj.p;
        ma.rout = B.rout.p;
        ma.reqs = B.rq;
        ma.cap = B.cap;
        ma.k0 = k0;
        ma.n = n;
        ma.adm = B.adm.p;
        ma.n_adm = (int32_t)adm_all.size();
        ma.sep_h = c->sep.horiz_m;
        ma.sep_v = c->sep.vert_m;
        ma.out = B.sepo.p;
        LAUNCH(c, launch_batch_minsep(ma, c->stream));
        CK(cudaMemcpyAsync(B.h_sep.p + k0, B.sepo.p + k0, n * sizeof(SepOut), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));  // adm_all may be released after this
        if (c->profiling) collect_timers(c);
        pending.clear();
        store.clear();
    }
    void rollback() {  // admissions whose plans never reached the table
        for (auto& pr : pending) {
            c->book.plans.erase(pr.first);
            c->book.free_slots.insert(pr.second);
        }
        pending.clear();
        recompute_hw(c);
    }
    void results(int32_t k0, int32_t n, fmdp_result* res) {
        for (int32_t k = k0; k < k0 + n; ++k) {
            fmdp_result* o = res + k;
            SepOut so = B.h_sep.p[k];  // the final plan's report with the run's admissions folded in
            so.verdict = verdict[k];
            fill_result(fin_ro[k], so, o);
            o->plan_id = ids[k];
            o->replanned = replans[k];
        }
    }
};

// Sizes the call-wide batch buffers for n requests of trajectories up to cap_needed samples
// and puts the requests on the device (their copy in dev_reqs, or uploaded).
void batch_prepare(fmdp_ctx* c, const fmdp_request* reqs, int32_t n, int32_t n_batch, const fmdp_request* dev_reqs) {
    BatchBuffers& B = c->bat;
    int32_t cap = 1;
    for (int32_t i = 0; i < n; ++i) cap = std::max(cap, reqs[i].horizon + 1);
    // buffer shapes in buckets, so that graphs are reused from call to call
    B.n_cap = std::max(B.n_cap, round_up(std::max(n_batch, 1), 64));
    B.rq_cap = std::max(B.rq_cap, round_up(std::max(n, 1), 256));
    B.cap = std::max(B.cap, round_up(cap, 256));
    const size_t R = B.rq_cap;
    B.traj.ensure(R * B.cap * 3);
    B.acts.ensure(R * B.cap);
    B.rout.ensure(R);
    B.sepo.ensure(R);
    B.idx.ensure(idx_words(B));
    B.ctr.ensure(4);
    B.infl.ensure((size_t)B.n_cap * B.n_cap);
    B.h_idx.ensure(idx_words(B));
    B.h_ctr.ensure(4);
    B.h_infl.ensure((size_t)B.n_cap * B.n_cap);
    B.h_rout.ensure(R);
    B.h_sep.ensure(R);
    if (dev_reqs) {
        B.rq = dev_reqs;
    } else {
        B.reqs.ensure(R);
        CK(cudaMemcpyAsync(B.reqs.p, reqs, n * sizeof(fmdp_request), cudaMemcpyHostToDevice, c->stream));
        B.rq = B.reqs.p;
    }
}

// Geometry of the call: the scanned slot range covers every slot the call may fill (the
// lowest free slots) or, with the spatial index, the whole table.
Geometry batch_geometry(fmdp_ctx* c, int32_t n_new, int32_t wave) {
    if (c->index_on) return geometry_batch(c, c->S_pad, wave);
    require((size_t)n_new <= c->book.free_slots.size(), FMDP_ERR_FULL, "not enough free plan slots for the batch");
    int32_t bound = c->book.S_hw;
    auto it = c->book.free_slots.begin();
    for (int32_t i = 0; i < n_new; ++i, ++it) bound = std::max(bound, *it + 1);
    return geometry_batch(c, round_up(bound, 512), wave);
}

void copy_points_back(fmdp_ctx* c, int32_t n, fmdp_result* res) {
    BatchBuffers& B = c->bat;
    bool want_points = false;
    for (int32_t i = 0; i < n; ++i) want_points = want_points || res[i].xyz || res[i].actions;
    if (!want_points) return;
    B.h_traj.ensure((size_t)n * B.cap * 3);
    B.h_acts.ensure((size_t)n * B.cap);
    CK(cudaMemcpyAsync(B.h_traj.p, B.traj.p, (size_t)n * B.cap * 3 * sizeof(float), cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaMemcpyAsync(B.h_acts.p, B.acts.p, (size_t)n * B.cap, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int32_t i = 0; i < n; ++i) {
        const int32_t np = res[i].n_points;
        if (res[i].xyz) std::memcpy(res[i].xyz, B.h_traj.p + (size_t)i * B.cap * 3, (size_t)np * 12);
        if (res[i].actions && np > 1) std::memcpy(res[i].actions, B.h_acts.p + (size_t)i * B.cap, (size_t)(np - 1));
    }
}

// Speculative batching over n validated requests (host copies in reqs; on the device in
// dev_reqs, or copied there when it is null), in consecutive batches of the option's size.
// Results to res; sample points to the callers' buffers named in res unless keep_points,
// which leaves them in the batch buffers for fmdp_fetch_staged. Returns the number admitted.
int32_t run_batch(fmdp_ctx* c, const fmdp_request* reqs, int32_t n, fmdp_result* res,
                  const fmdp_request* dev_reqs, bool keep_points) {
    if (n <= 0) return 0;
    const int32_t bs = c->opt.batch_size > 0 ? c->opt.batch_size : kBatchDefault;
    batch_prepare(c, reqs, n, std::min(n, bs), dev_reqs);
    if (c->learned_mode) {
        const size_t R = c->bat.rq_cap;
        c->p_traj.ensure(R * c->bat.cap * 3);
        c->p_acts.ensure(R * c->bat.cap);
        c->p_rout.ensure(R);
        c->p_sep.ensure(R);
        c->p_acc.ensure(R);
        c->p_queue.ensure(1);
        c->bat.h_acc.ensure(R);
        CK(cudaMemsetAsync(c->p_acc.p, 0, R * sizeof(int32_t), c->stream));
    }
    Speculator sp(c, reqs, n);
    std::vector<int32_t> resolved;
    for (int32_t b0 = 0; b0 < n; b0 += bs) {
        const int32_t m = std::min(bs, n - b0);
        sp.set_geometry(batch_geometry(c, m, m));
        for (int32_t i = 0; i < m; ++i) sp.add(b0 + i);
        sp.adm_all.clear();
        try {
            while (!sp.U.empty()) sp.wave(resolved);
            sp.finish(b0, m);
        } catch (...) {
            sp.rollback();
            throw;
        }
    }
    sp.results(0, n, res);
    if (!keep_points) copy_points_back(c, n, res);
    return sp.admitted;
}


// ------------------------------------------------------------------ learned proposal

// platform-independent random numbers (splitmix64; Box-Muller normals)
struct SplitMix {
    uint64_t s;
    uint64_t next() {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
    double normal() {
        const double u1 = std::max(uniform(), 1e-300), u2 = uniform();
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    }
};

size_t wt_offset(int l) {
    size_t o = 0;
    for (int i = 0; i < l; ++i) o += (size_t)layer_in(i) * layer_out_pad(i);
    return o;
}

void mlp_ensure(fmdp_ctx* c) {
    const size_t P = n_params_total();
    c->mlp_p.ensure(P);
    c->mlp_g.ensure(P);
    c->mlp_m1.ensure(P);
    c->mlp_m2.ensure(P);
    c->mlp_wt.ensure(wt_offset(kLayers));
    c->mlp_wp.ensure(wp_total());
    c->tr_loss.ensure(1);
}

void mlp_upload(fmdp_ctx* c, const float* params) {
    mlp_ensure(c);
    const size_t P = n_params_total();
    CK(cudaMemcpyAsync(c->mlp_p.p, params, P * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemsetAsync(c->mlp_m1.p, 0, P * sizeof(float), c->stream));
    CK(cudaMemsetAsync(c->mlp_m2.p, 0, P * sizeof(float), c->stream));
    c->adam_t = 0;
    LAUNCH(c, launch_export_weights(c->mlp_p.p, c->mlp_wt.p, c->mlp_wp.p, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->mlp_ready = true;
}

// forward and backward of one batch (X: B rows of bf16 features on the device, y labels):
// the batch's mean loss is added to tr_loss[0], the gradient written to mlp_g
void mlp_fwd_bwd(fmdp_ctx* c, const __nv_bfloat16* X, const uint8_t* y, int B) {
    cudaStream_t s = c->stream;
    c->trH.ensure((size_t)4 * B * kHid);
    c->trZ.ensure((size_t)B * kHid);
    c->trdZ.ensure((size_t)B * kHid);
    c->trdZf.ensure((size_t)B * kHid);
    c->trdH.ensure((size_t)B * kHid);
    auto H = [&](int l) -> const __nv_bfloat16* { return l == 0 ? X : c->trH.p + (size_t)(l - 1) * B * kHid; };
    auto ldH = [&](int l) { return l == 0 ? kFeat : kHid; };
    const __nv_bfloat16* Wt = c->mlp_wt.p;
    const float* P = c->mlp_p.p;
    float* G = c->mlp_g.p;
    for (int l = 0; l < kLayers - 1; ++l) {
        LAUNCH(c, launch_gemm_bf16(B, kHid, layer_in(l), H(l), ldH(l), 1, Wt + wt_offset(l), kHid, 1, c->trZ.p, kHid, 0, s));
        LAUNCH(c, launch_bias_act(c->trZ.p, P + param_offset_b(l), c->trH.p + (size_t)l * B * kHid, B, kHid, kHid, kHid,
                                  1, s));
    }
    const int L4 = kLayers - 1;
    LAUNCH(c, launch_gemm_bf16(B, kOutPad, kHid, H(L4), kHid, 1, Wt + wt_offset(L4), kOutPad, 1, c->trZ.p, kOutPad, 0, s));
    LAUNCH(c, launch_softmax_ce(c->trZ.p, kOutPad, P + param_offset_b(L4), y, B, c->A, c->trdZ.p, kOutPad, c->trdZf.p,
                                c->tr_loss.p, s));
    for (int l = kLayers - 1; l >= 0; --l) {
        const int ld_dz = l == kLayers - 1 ? kOutPad : kHid, out = layer_out(l);
        LAUNCH(c, launch_gemm_bf16(layer_in(l), out, B, H(l), 1, ldH(l), c->trdZ.p, ld_dz, 1, G + param_offset_W(l), out,
                                   0, s));
        LAUNCH(c, launch_colsum(c->trdZf.p, B, out, ld_dz, G + param_offset_b(l), s));
        if (l > 0) {
            LAUNCH(c, launch_gemm_bf16(B, layer_in(l), out, c->trdZ.p, ld_dz, 1, Wt + wt_offset(l), 1,
                                       layer_out_pad(l), c->trdH.p, kHid, 0, s));
            LAUNCH(c, launch_relu_bwd(c->trdH.p, H(l), B, kHid, c->trdZ.p, c->trdZf.p, s));
        }
    }
}

void mlp_train(fmdp_ctx* c, int32_t epochs, int32_t batch, float lr, uint64_t seed, float* losses) {
    require(c->mlp_ready, FMDP_ERR_ARG, "the proposal network has no parameters (init or set them first)");
    require(c->t_rows > 0, FMDP_ERR_ARG, "no training rows (collect first)");
    require(epochs >= 0 && batch >= 1 && batch <= 8192 && lr > 0.f, FMDP_ERR_ARG, "training options out of range");
    const int64_t rows = c->t_rows;
    c->tr_idx.ensure(rows);
    c->trX.ensure((size_t)batch * kFeat);
    c->tr_y.ensure(batch);
    std::vector<int32_t> perm(rows);
    SplitMix rng{seed};
    for (int32_t e = 0; e < epochs; ++e) {
        for (int64_t i = 0; i < rows; ++i) perm[i] = (int32_t)i;
        for (int64_t i = rows - 1; i > 0; --i) std::swap(perm[i], perm[(int64_t)(rng.next() % (uint64_t)(i + 1))]);
        CK(cudaMemcpyAsync(c->tr_idx.p, perm.data(), rows * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemsetAsync(c->tr_loss.p, 0, sizeof(float), c->stream));
        int64_t nb = 0;
        for (int64_t b0 = 0; b0 < rows; b0 += batch, ++nb) {
            const int Bn = (int)std::min<int64_t>(batch, rows - b0);
            LAUNCH(c, launch_gather_rows(c->tX.p, c->tr_idx.p + b0, Bn, c->trX.p, c->ty.p, c->tr_y.p, c->stream));
            mlp_fwd_bwd(c, c->trX.p, c->tr_y.p, Bn);
            LAUNCH(c, launch_adam(c->mlp_p.p, c->mlp_g.p, c->mlp_m1.p, c->mlp_m2.p, n_params_total(), lr, 0.9f, 0.999f,
                                  1e-8f, (int)++c->adam_t, c->stream));
            LAUNCH(c, launch_export_weights(c->mlp_p.p, c->mlp_wt.p, c->mlp_wp.p, c->stream));
        }
        float tot = 0.f;
        CK(cudaMemcpyAsync(&tot, c->tr_loss.p, sizeof(float), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        if (losses) losses[e] = nb ? tot / (float)nb : 0.f;
    }
    CK(cudaStreamSynchronize(c->stream));
}

// grows a device array to `want` elements, keeping its first `keep` elements
template <class T>
void grow_keep(fmdp_ctx* c, DevArray<T>& a, size_t want, size_t keep) {
    if (want <= a.n) return;
    DevArray<T> b;
    b.ensure(std::max(want, a.n * 2));
    if (keep) CK(cudaMemcpyAsync(b.p, a.p, keep * sizeof(T), cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    a.release();
    a.p = b.p;
    a.n = b.n;
    b.p = nullptr;
    b.n = 0;
}

// FastMDP rollouts of every request against the table as it stands (persistent work-queue
// launch; nothing is checked or admitted); trajectories in the batch buffers
void plan_all_fastmdp(fmdp_ctx* c, int32_t n) {
    BatchBuffers& B = c->bat;
    const Geometry g = batch_geometry(c, 0, n);
    const int n_clusters = std::max(1, std::min(n, rollout_max_active_clusters(g.cs, g.threads, g.smem)));
    CK(cudaMemsetAsync(B.ctr.p, 0, sizeof(int32_t), c->stream));
    RolloutArgs ra{};
    ra.m = c->model;
    ra.tab = table_view(c);
    ra.S_scan = g.S_scan;
    ra.chunk = g.chunk;
    ra.cs = g.cs;
    ra.ring = g.ring;
    ra.cap = B.cap;
    ra.reqs = B.rq;
    ra.n_req = n;
    ra.traj = B.traj.p;
    ra.acts = B.acts.p;
    ra.out = B.rout.p;
    ra.err = c->err;
    set_index_args(c, ra, g);
    ra.queue = B.ctr.p;
    LAUNCH(c, launch_rollout(ra, g.threads, g.smem, c->stream, n_clusters));
}

// ---- departure-time candidates

// For each request in FCFS order: its variants departing delays[d] steps later, planned in
// one persistent rollout launch and separation-checked together against the table as it
// stands; the first admissible variant in the order of delays is admitted. Rejected
// variants change nothing, so every variant up to the chosen one has the result that
// fmdp_schedule of it alone would give.
void run_departures(fmdp_ctx* c, const fmdp_request* reqs, int32_t n, const int64_t* delays, int32_t D,
                    fmdp_result* res, int32_t* chosen, int32_t* verdicts) {
    std::vector<fmdp_request> cand(D);
    std::vector<int32_t> ident(D);
    for (int32_t d = 0; d < D; ++d) ident[d] = d;
    c->p_ident.ensure(D);
    CK(cudaMemcpyAsync(c->p_ident.p, ident.data(), D * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t d = 0; d < D; ++d) {
            cand[d] = reqs[i];
            cand[d].depart_step = reqs[i].depart_step + delays[d];
        }
        batch_prepare(c, cand.data(), D, D, nullptr);
        BatchBuffers& B = c->bat;
        const Geometry g = batch_geometry(c, 0, D);
        plan_all_fastmdp(c, D);
        LAUNCH(c, launch_sep_reset(B.sepo.p, D, c->stream));
        B.h_ctr.p[1] = D;
        CK(cudaMemcpyAsync(B.ctr.p + 1, &B.h_ctr.p[1], sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
        SepRowsArgs sa{};
        sa.m = c->model;
        sa.tab = table_view(c);
        sa.S_scan = g.S_scan;
        sa.traj = B.traj.p;
        sa.cap = B.cap;
        sa.rout = B.rout.p;
        sa.reqs = B.rq;
        sa.idx = c->p_ident.p;
        sa.n_dev = B.ctr.p + 1;
        sa.n_max = D;
        sa.out = B.sepo.p;
        if (c->index_on) {
            sa.items = c->ix_items;
            sa.cstart = c->ix_cstart;
            sa.nextra = c->ix_nextra;
            sa.ncell = c->ix_ncell;
        }
        LAUNCH(c, launch_sepcheck_rows(sa, c->stream));
        CK(cudaMemcpyAsync(B.h_rout.p, B.rout.p, D * sizeof(RolloutOut), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaMemcpyAsync(B.h_sep.p, B.sepo.p, D * sizeof(SepOut), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        require(read_error_word(c) == 0, FMDP_ERR_TIMEOUT, "a bounded device wait expired during a rollout");
        // the admission rule of the admit kernel, per variant
        int32_t pick = -1;
        std::vector<int32_t> vd(D);
        for (int32_t d = 0; d < D; ++d) {
            const RolloutOut& ro = B.h_rout.p[d];
            const SepOut& so = B.h_sep.p[d];
            vd[d] = ro.status != kStatusCaptured ? ro.status
                    : so.first_conflict != INT_MAX ? FMDP_REJ_CONFLICT
                    : so.first_terrain != INT_MAX ? FMDP_REJ_TERRAIN
                                                  : FMDP_ADMITTED;
            c->stats.rollout_steps += ro.steps;
            if (verdicts) verdicts[(size_t)i * D + d] = vd[d];
            if (pick < 0 && vd[d] == FMDP_ADMITTED) pick = d;
        }
        const int32_t show = pick >= 0 ? pick : 0;
        uint64_t id = 0;
        if (pick >= 0) {
            const int32_t slot = take_slot(c);
            try {
                c->slots.ensure(1);
                CK(cudaMemcpyAsync(c->slots.p, &slot, sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
                AdmitArgs aa{};
                aa.err = c->err;
                aa.tab = table_view(c);
                aa.cap = B.cap;
                aa.traj = B.traj.p + (size_t)pick * B.cap * 3;
                aa.rout = B.rout.p + pick;
                aa.reqs = B.rq + pick;
                aa.slots = c->slots.p;
                aa.sep = B.sepo.p + pick;
                aa.force = 0;
                LAUNCH(c, launch_admit(aa, 1, B.cap, c->stream));
                const int64_t d0 = cand[pick].depart_step;
                index_append_admitted(c, aa.traj, B.cap, aa.rout, aa.reqs, aa.sep, nullptr, nullptr, 1, d0,
                                      d0 + cand[pick].horizon + 1);
                CK(cudaStreamSynchronize(c->stream));
            } catch (...) {
                c->book.free_slots.insert(slot);
                throw;
            }
            id = c->book.next_id++;
            c->book.plans[id] = PlanMeta{slot, cand[pick].depart_step, B.h_rout.p[pick].n_points};
            c->book.S_hw = std::max(c->book.S_hw, slot + 1);
        }
        if (chosen) chosen[i] = pick;
        if (res) {
            fmdp_result& r = res[i];
            fill_result(B.h_rout.p[show], B.h_sep.p[show], &r);
            r.verdict = vd[show];
            r.plan_id = id;
            r.replanned = 0;
            r.source = 0;
            const int32_t np = r.n_points;
            if (r.xyz)
                CK(cudaMemcpyAsync(r.xyz, B.traj.p + (size_t)show * B.cap * 3, (size_t)np * 3 * sizeof(float),
                                   cudaMemcpyDeviceToHost, c->stream));
            if (r.actions && np > 1)
                CK(cudaMemcpyAsync(r.actions, B.acts.p + (size_t)show * B.cap, (size_t)(np - 1),
                                   cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
        }
    }
}

// Departure-time candidates through speculative batches. The variants are the work items
// (request i's variant d is item i * D + d); a request's D items are added and resolved
// together, and the walk admits its first admissible variant. An admission that influences
// no item of a request leaves all its variants' plans and verdicts exact, so the results
// equal run_departures.
void run_departures_batch(fmdp_ctx* c, const fmdp_request* reqs, int32_t n, const int64_t* delays, int32_t D,
                          fmdp_result* res, int32_t* chosen, int32_t* verdicts) {
    if (n <= 0) return;
    const int32_t N = n * D;
    std::vector<fmdp_request> cand((size_t)N);
    for (int32_t i = 0; i < n; ++i)
        for (int32_t d = 0; d < D; ++d) {
            cand[(size_t)i * D + d] = reqs[i];
            cand[(size_t)i * D + d].depart_step = reqs[i].depart_step + delays[d];
        }
    const int32_t bs = std::max(1, batch_size_of(c) / D) * D;  // whole requests per batch
    batch_prepare(c, cand.data(), N, std::min(N, bs), nullptr);
    Speculator sp(c, cand.data(), N);
    sp.group = (size_t)D;
    std::vector<int32_t> resolved;
    for (int32_t b0 = 0; b0 < N; b0 += bs) {
        const int32_t m = std::min(bs, N - b0);
        sp.set_geometry(batch_geometry(c, m / D, m));  // at most one admission per request
        for (int32_t i = 0; i < m; ++i) sp.add(b0 + i);
        sp.adm_all.clear();
        try {
            while (!sp.U.empty()) sp.wave(resolved);
            sp.finish(b0, m);
        } catch (...) {
            sp.rollback();
            throw;
        }
    }
    std::vector<fmdp_result> items((size_t)N);
    sp.results(0, N, items.data());
    BatchBuffers& B = c->bat;
    bool want_points = false;
    for (int32_t i = 0; i < n; ++i) want_points = want_points || res[i].xyz || res[i].actions;
    if (want_points) {
        B.h_traj.ensure((size_t)N * B.cap * 3);
        B.h_acts.ensure((size_t)N * B.cap);
        CK(cudaMemcpyAsync(B.h_traj.p, B.traj.p, (size_t)N * B.cap * 3 * sizeof(float), cudaMemcpyDeviceToHost,
                           c->stream));
        CK(cudaMemcpyAsync(B.h_acts.p, B.acts.p, (size_t)N * B.cap, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    for (int32_t i = 0; i < n; ++i) {
        int32_t pick = -1;
        for (int32_t d = 0; d < D; ++d) {
            const size_t k = (size_t)i * D + d;
            if (verdicts) verdicts[k] = items[k].verdict;
            if (pick < 0 && sp.ids[k] != 0) pick = d;
        }
        if (chosen) chosen[i] = pick;
        const size_t k = (size_t)i * D + (pick >= 0 ? pick : 0);
        float* xyz = res[i].xyz;
        uint8_t* acts = res[i].actions;
        res[i] = items[k];
        res[i].xyz = xyz;
        res[i].actions = acts;
        res[i].source = 0;
        const int32_t np = res[i].n_points;
        if (xyz) std::memcpy(xyz, B.h_traj.p + k * B.cap * 3, (size_t)np * 12);
        if (acts && np > 1) std::memcpy(acts, B.h_acts.p + k * B.cap, (size_t)(np - 1));
    }
}

// ---- autotuner of the batched indexed rollout (results do not depend on the shape)

constexpr int32_t kTuneThreads[] = {128, 192, 256, 320, 384};
constexpr int32_t kTuneStage[] = {512, 1024, 1536, 2048};

bool tune_shape_ok(int32_t threads, int32_t icap) {
    bool t = false, i = false;
    for (int32_t v : kTuneThreads) t |= v == threads;
    for (int32_t v : kTuneStage) i |= v == icap;
    return t && i;
}

// Times the rollouts of the first W sample requests (one wave, nothing admitted) under each
// candidate shape, for W = min(n, batch size) and its halvings down to 8, and caches the
// fastest shape of each wave-size bucket. The report describes the largest wave.
void autotune(fmdp_ctx* c, const fmdp_request* sample, int32_t n, bool force, fmdp_tune_report* rep) {
    require(c->index_on, FMDP_ERR_ARG, "the autotuner covers the indexed rollout (full_scan must be 0)");
    require(n >= 1 && sample, FMDP_ERR_ARG, "the autotuner needs at least one sample request");
    fmdp_tune_report r{};
    const int32_t m = std::min(n, batch_size_of(c));
    r.sample = m;
    const auto key = tune_key(c, m);
    const auto hit = c->tune.find(key);
    auto describe = [&](const fmdp_tune_entry& e) {
        r.chosen = e;
        c->try_threads = e.threads_per_cta;
        c->try_icap = e.index_stage_items;
        const Geometry g = batch_geometry(c, 0, m);
        c->try_threads = c->try_icap = 0;
        r.ctas_per_sm = rollout_max_active_clusters(1, g.threads, g.smem) / std::max(1, c->n_sm);
    };
    if (hit != c->tune.end() && !force) {
        describe(hit->second);
        r.from_cache = 1;
        r.default_ms = -1.0;
        if (rep) *rep = r;
        return;
    }
    std::vector<int32_t> sizes;
    for (int32_t w = m; w >= 1; w /= 2) {
        sizes.push_back(w);
        if (w <= 8) break;
    }
    batch_prepare(c, sample, m, m, nullptr);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    try {
        for (int32_t w : sizes) {
            double best = 1e300;
            int32_t bt = 384, bi = 1536;
            for (int32_t th : kTuneThreads)
                for (int32_t ic : kTuneStage) {
                    if (rollout_smem_bytes(0, 0, ic) > (size_t)c->max_smem) continue;
                    c->try_threads = th;
                    c->try_icap = ic;
                    plan_all_fastmdp(c, w);  // warm-up
                    double t_min = 1e300;
                    for (int rep_i = 0; rep_i < 2; ++rep_i) {
                        CK(cudaEventRecord(e0, c->stream));
                        plan_all_fastmdp(c, w);
                        CK(cudaEventRecord(e1, c->stream));
                        CK(cudaEventSynchronize(e1));
                        float ms = 0.f;
                        CK(cudaEventElapsedTime(&ms, e0, e1));
                        t_min = std::min(t_min, (double)ms);
                    }
                    require(read_error_word(c) == 0, FMDP_ERR_TIMEOUT,
                            "a bounded device wait expired during a rollout");
                    ++r.candidates;
                    if (w == m && th == 384 && ic == 1536) r.default_ms = t_min;
                    if (t_min < best) {
                        best = t_min;
                        bt = th;
                        bi = ic;
                    }
                }
            c->try_threads = c->try_icap = 0;
            const auto k = tune_key(c, w);
            fmdp_tune_entry en{};
            en.n_actions = k[0];
            en.combine = k[1];
            en.plans_bucket = k[2];
            en.wave_bucket = k[3];
            en.threads_per_cta = bt;
            en.index_stage_items = bi;
            en.ms = best;
            c->tune[k] = en;
            ++r.entries;
        }
    } catch (...) {
        c->try_threads = c->try_icap = 0;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    describe(c->tune[key]);
    if (rep) *rep = r;
}

void learned_collect(fmdp_ctx* c, const fmdp_request* reqs, int32_t n) {
    require(c->index_on, FMDP_ERR_ARG, "the learned proposal reads the spatial index (full_scan must be 0)");
    if (n <= 0) return;
    batch_prepare(c, reqs, n, 64, nullptr);
    BatchBuffers& B = c->bat;
    plan_all_fastmdp(c, n);
    CK(cudaMemcpyAsync(B.h_rout.p, B.rout.p, n * sizeof(RolloutOut), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    require(read_error_word(c) == 0, FMDP_ERR_TIMEOUT, "a bounded device wait expired during a rollout");
    std::vector<int64_t> row0(n);
    int64_t rows = c->t_rows;
    for (int32_t i = 0; i < n; ++i) {
        row0[i] = rows;
        rows += std::max(B.h_rout.p[i].n_points - 1, 0);
    }
    grow_keep(c, c->tX, (size_t)rows * kFeat, (size_t)c->t_rows * kFeat);
    grow_keep(c, c->ty, (size_t)rows, (size_t)c->t_rows);
    c->row0.ensure(n);
    CK(cudaMemcpyAsync(c->row0.p, row0.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
    CollectArgs ca{};
    ca.m = c->model;
    ca.tab = table_view(c);
    ca.iv = index_view(c);
    ca.traj = B.traj.p;
    ca.acts = B.acts.p;
    ca.cap = B.cap;
    ca.rout = B.rout.p;
    ca.reqs = B.rq;
    ca.row0 = c->row0.p;
    ca.X = c->tX.p;
    ca.y = c->ty.p;
    ca.n = n;
    LAUNCH(c, launch_collect(ca, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->t_rows = rows;
}

void learned_evaluate(fmdp_ctx* c, const fmdp_request* reqs, int32_t n, double slack, fmdp_learned_report* rep,
                      int32_t* accepted, int32_t* steps_p, int32_t* steps_f) {
    require(c->index_on, FMDP_ERR_ARG, "the learned proposal reads the spatial index (full_scan must be 0)");
    require(c->mlp_ready, FMDP_ERR_ARG, "the proposal network has no parameters (init or set them first)");
    require(slack >= 0.0, FMDP_ERR_ARG, "slack must be >= 0");
    fmdp_learned_report r{};
    r.n = n;
    if (n <= 0) {
        if (rep) *rep = r;
        return;
    }
    batch_prepare(c, reqs, n, 64, nullptr);
    BatchBuffers& B = c->bat;
    const size_t R = B.rq_cap;
    c->p_traj.ensure(R * B.cap * 3);
    c->p_acts.ensure(R * B.cap);
    c->p_rout.ensure(R);
    c->p_sep.ensure(R);
    c->p_acc.ensure(R);
    c->p_queue.ensure(1);
    c->p_ident.ensure(R);
    std::vector<int32_t> ident(n);
    for (int32_t i = 0; i < n; ++i) ident[i] = i;
    CK(cudaMemcpyAsync(c->p_ident.p, ident.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
    cudaEvent_t e[4];
    for (auto& ev : e) CK(cudaEventCreate(&ev));
    // proposals for every request
    CK(cudaMemsetAsync(c->p_queue.p, 0, sizeof(int32_t), c->stream));
    PolicyArgs pa{};
    pa.m = c->model;
    pa.tab = table_view(c);
    pa.iv = index_view(c);
    pa.Wp = c->mlp_wp.p;
    pa.params = c->mlp_p.p;
    pa.reqs = B.rq;
    pa.n_items = n;
    pa.queue = c->p_queue.p;
    pa.cap = B.cap;
    pa.traj = c->p_traj.p;
    pa.acts = c->p_acts.p;
    pa.out = c->p_rout.p;
    pa.err = c->err;
    pa.rows = policy_rows_for(n, c->n_sm);
    CK(cudaEventRecord(e[0], c->stream));
    LAUNCH(c, launch_policy(pa, std::min(c->n_sm, (n + pa.rows - 1) / pa.rows), c->stream));
    CK(cudaEventRecord(e[1], c->stream));
    // their separation checks and the judge (decisions only), in chunks of the row kernel's size
    LAUNCH(c, launch_sep_reset(c->p_sep.p, n, c->stream));
    for (int32_t o = 0; o < n; o += kBatchMax) {
        const int32_t m = std::min<int32_t>(kBatchMax, n - o);
        B.h_ctr.p[1] = m;
        CK(cudaMemcpyAsync(B.ctr.p + 1, &B.h_ctr.p[1], sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
        SepRowsArgs sp{};
        sp.m = c->model;
        sp.tab = table_view(c);
        sp.S_scan = c->S_pad;
        sp.traj = c->p_traj.p;
        sp.cap = B.cap;
        sp.rout = c->p_rout.p;
        sp.reqs = B.rq;
        sp.idx = c->p_ident.p + o;
        sp.n_dev = B.ctr.p + 1;
        sp.n_max = m;
        sp.out = c->p_sep.p;
        sp.items = c->ix_items;
        sp.cstart = c->ix_cstart;
        sp.nextra = c->ix_nextra;
        sp.ncell = c->ix_ncell;
        LAUNCH(c, launch_sepcheck_rows(sp, c->stream));
        CK(cudaStreamSynchronize(c->stream));  // the count word is reused by the next chunk
    }
    JudgeArgs ja{};
    ja.reqs = B.rq;
    ja.n = n;
    ja.traj_p = c->p_traj.p;
    ja.acts_p = c->p_acts.p;
    ja.rout_p = c->p_rout.p;
    ja.sep_p = c->p_sep.p;
    ja.accepted = c->p_acc.p;
    ja.cap = B.cap;
    ja.dt = c->air.dt;
    ja.slack = slack;
    ja.climb_step = climb_step(c);
    LAUNCH(c, launch_judge(ja, B.cap, c->stream));
    // FastMDP plans of every request
    CK(cudaEventRecord(e[2], c->stream));
    plan_all_fastmdp(c, n);
    CK(cudaEventRecord(e[3], c->stream));
    std::vector<RolloutOut> rp(n), rf(n);
    std::vector<int32_t> acc(n);
    CK(cudaMemcpyAsync(rp.data(), c->p_rout.p, n * sizeof(RolloutOut), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(rf.data(), B.rout.p, n * sizeof(RolloutOut), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(acc.data(), c->p_acc.p, n * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    float ms1 = 0.f, ms2 = 0.f;
    CK(cudaEventElapsedTime(&ms1, e[0], e[1]));
    CK(cudaEventElapsedTime(&ms2, e[2], e[3]));
    for (auto& ev : e) cudaEventDestroy(ev);
    require(read_error_word(c) == 0, FMDP_ERR_TIMEOUT, "a bounded device wait expired during a rollout");
    double gap_sum = 0.0;
    int32_t gap_n = 0;
    for (int32_t i = 0; i < n; ++i) {
        r.accepted += acc[i];
        r.proposals_captured += rp[i].status == kStatusCaptured;
        r.fastmdp_captured += rf[i].status == kStatusCaptured;
        r.proposal_steps += rp[i].steps;
        r.fastmdp_steps += rf[i].steps;
        if (acc[i] && rf[i].status == kStatusCaptured && rf[i].steps > 0) {
            const double gap = (double)(rp[i].steps - rf[i].steps) / rf[i].steps;
            gap_sum += gap;
            r.max_gap = gap_n ? std::max(r.max_gap, gap) : gap;
            ++gap_n;
        }
        if (accepted) accepted[i] = acc[i];
        if (steps_p) steps_p[i] = rp[i].steps;
        if (steps_f) steps_f[i] = rf[i].steps;
    }
    r.mean_gap = gap_n ? gap_sum / gap_n : 0.0;
    r.proposal_ms = ms1;
    r.fastmdp_ms = ms2;
    if (rep) *rep = r;
}

// ------------------------------------------------------------------ serving loop

void expire_to(fmdp_ctx* c, int64_t t_now, int64_t* n_expired);  // below

// Continuous batching over an arrival trace (see fmdp_serve in the header).
void run_serve(fmdp_ctx* c, const fmdp_request* reqs, const double* arrival_s, int32_t n,
               const fmdp_serve_options& o, fmdp_result* res, double* latency_ms, fmdp_serve_report* rep) {
    using clk = std::chrono::steady_clock;
    const int32_t bs = c->opt.batch_size > 0 ? c->opt.batch_size : kBatchDefault;
    const int32_t in_flight = std::max(1, std::min(o.max_in_flight > 0 ? o.max_in_flight : bs, kBatchMax));
    const int32_t max_active = o.max_active_plans > 0 ? std::min(o.max_active_plans, c->S_max) : c->S_max;
    const double scale = o.time_scale > 0.0 ? o.time_scale : 1.0;
    const int64_t quantum = o.expire_quantum > 0 ? o.expire_quantum : 60;
    const int64_t sim0 = o.sim_start_set ? o.sim_start_step : c->book.t_base;
    batch_prepare(c, reqs, n, in_flight, nullptr);
    Speculator sp(c, reqs, n);
    sp.set_geometry(batch_geometry(c, 0, 1));
    // earliest departure among requests i .. n-1 (the clock never expires past it)
    std::vector<int64_t> dep_suffix(n + 1, INT64_MAX);
    for (int32_t i = n - 1; i >= 0; --i) dep_suffix[i] = std::min(dep_suffix[i + 1], reqs[i].depart_step);
    std::vector<double> done_at(n, -1.0);
    std::vector<int32_t> resolved;
    std::vector<uint8_t> deferred(n, 0);
    int32_t next = 0, completed = 0;
    int64_t expiries = 0, expired = 0;
    int32_t max_seen = 0;
    const fmdp_stats st0 = c->stats;
    const auto t0 = clk::now();
    auto elapsed = [&]() { return std::chrono::duration<double>(clk::now() - t0).count(); };
    try {
        while (completed < n) {
            const double now = elapsed();
            // expiry: up to the clock, never past a departure still to plan or to store
            int64_t first_open = sp.U.empty() ? next : sp.U.front();
            int64_t limit = sim0 + (int64_t)std::floor(now * scale / c->air.dt);
            limit = std::min(limit, dep_suffix[std::min<int64_t>(first_open, n)]);
            for (int32_t r : sp.store) limit = std::min(limit, reqs[r].depart_step);
            if (limit >= c->book.t_base + quantum) {
                expire_to(c, limit, &expired);
                ++expiries;
                sp.set_geometry(batch_geometry(c, 0, 1));
            }
            // admission: arrived requests join while the set has room and slots remain for all
            bool blocked = false;
            while (next < n && arrival_s[next] <= now && (int32_t)sp.U.size() < in_flight) {
                const int64_t active = (int64_t)c->book.plans.size();
                const int64_t room = std::min<int64_t>((int64_t)c->book.free_slots.size(), max_active - active);
                if ((int64_t)sp.U.size() + 1 > room) {
                    blocked = true;
                    if (!deferred[next]) deferred[next] = 1;
                    break;
                }
                sp.add(next++);
            }
            max_seen = std::max(max_seen, (int32_t)sp.U.size());
            if (!sp.U.empty()) {
                resolved.clear();
                sp.wave(resolved);
                const double t = elapsed();
                for (int32_t k : resolved) done_at[k] = t;
                completed += (int32_t)resolved.size();
                continue;
            }
            if (next >= n) break;
            if (blocked) {
                // nothing in flight and no room: only the clock can free slots, by expiring a
                // plan that ends before the next departure
                int64_t first_end = INT64_MAX;
                for (auto& kv : c->book.plans) first_end = std::min(first_end, kv.second.t0 + kv.second.n);
                require(first_end <= dep_suffix[next], FMDP_ERR_FULL, "plan table full and no plan can expire");
                std::this_thread::sleep_for(std::chrono::microseconds(200));
                continue;
            }
            const double wait = arrival_s[next] - elapsed();
            if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(std::min(wait, 0.01)));
        }
        sp.finish(0, n);
    } catch (...) {
        sp.rollback();
        throw;
    }
    sp.results(0, n, res);
    copy_points_back(c, n, res);
    // report
    std::vector<double> lat(n);
    double mx = 0.0, sum = 0.0, last = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        lat[i] = 1e3 * std::max(0.0, done_at[i] - arrival_s[i]);
        if (latency_ms) latency_ms[i] = lat[i];
        mx = std::max(mx, lat[i]);
        sum += lat[i];
        last = std::max(last, done_at[i]);
    }
    if (rep) {
        std::vector<double> sorted = lat;
        std::sort(sorted.begin(), sorted.end());
        auto pct = [&](double q) {
            if (sorted.empty()) return 0.0;
            const size_t i = (size_t)std::min<double>((double)sorted.size() - 1, std::ceil(q * sorted.size()) - 1);
            return sorted[i];
        };
        *rep = fmdp_serve_report{};
        rep->wall_s = last;
        rep->throughput_rps = last > 0.0 ? n / last : 0.0;
        rep->latency_p50_ms = pct(0.50);
        rep->latency_p99_ms = pct(0.99);
        rep->latency_mean_ms = n ? sum / n : 0.0;
        rep->latency_max_ms = mx;
        rep->waves = c->stats.batch_waves - st0.batch_waves;
        rep->rollouts = c->stats.batch_rollouts - st0.batch_rollouts;
        rep->replans = c->stats.batch_replans - st0.batch_replans;
        rep->expiries = expiries;
        rep->plans_expired = expired;
        rep->final_t_base = c->book.t_base;
        rep->admitted = sp.admitted;
        rep->rejected = n - sp.admitted;
        rep->max_in_flight_seen = max_seen;
        int32_t nd = 0;
        for (uint8_t d : deferred) nd += d;
        rep->deferred_for_memory = nd;
    }
}

void store_plans(fmdp_ctx* c, int32_t n_plans, const int64_t* t0s, const int32_t* counts, const float* xyz,
                 uint64_t* ids_out) {
    require(n_plans >= 0, FMDP_ERR_ARG, "n_plans < 0");
    if (n_plans == 0) return;
    require(t0s && counts && xyz, FMDP_ERR_ARG, "null plan arrays");
    require((size_t)n_plans <= c->book.free_slots.size(), FMDP_ERR_FULL, "not enough free plan slots");
    std::vector<int64_t> offs(n_plans);
    int64_t total = 0;
    int32_t maxc = 0;
    const int64_t lo = c->book.t_base, hi = c->book.t_base + c->T_win;
    for (int32_t i = 0; i < n_plans; ++i) {
        require(counts[i] >= 1, FMDP_ERR_ARG, "a plan needs at least one point");
        require(t0s[i] >= lo && t0s[i] + counts[i] <= hi, FMDP_ERR_RANGE, "plan steps fall outside the window");
        offs[i] = total;
        total += counts[i];
        maxc = std::max(maxc, counts[i]);
    }
    bool finite = true;  // one pass without early exit (vectorises)
    for (int64_t i = 0; i < 3 * total; ++i) finite &= std::isfinite(xyz[i]);
    require(finite, FMDP_ERR_ARG, "plan points must be finite");
    std::vector<int32_t> sl(n_plans);
    for (int32_t i = 0; i < n_plans; ++i) sl[i] = take_slot(c);
    try {
        c->traj.ensure((size_t)total * 3);
        c->t0s.ensure(n_plans);
        c->offs.ensure(n_plans);
        c->counts.ensure(n_plans);
        c->slots.ensure(n_plans);
        CK(cudaMemcpyAsync(c->traj.p, xyz, (size_t)total * 3 * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(c->t0s.p, t0s, n_plans * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(c->offs.p, offs.data(), n_plans * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(c->counts.p, counts, n_plans * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(c->slots.p, sl.data(), n_plans * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
        AdmitArgs aa{};
        aa.err = c->err;
        aa.tab = table_view(c);
        aa.cap = 0;
        aa.traj = c->traj.p;
        aa.slots = c->slots.p;
        aa.force = 1;
        aa.t0s = c->t0s.p;
        aa.counts = c->counts.p;
        aa.offs = c->offs.p;
        LAUNCH(c, launch_admit(aa, n_plans, maxc, c->stream));
        if (c->index_on) {
            int64_t tlo = t0s[0], thi = t0s[0];
            for (int32_t i = 0; i < n_plans; ++i) {
                tlo = std::min(tlo, t0s[i]);
                thi = std::max(thi, t0s[i] + counts[i]);
            }
            if (n_plans <= 8) {  // a few plans: append them to their rows' extra lists
                IndexAppendArgs ia{};
                ia.ix = index_args(c);
                ia.traj = c->traj.p;
                ia.force = 1;
                ia.t0s = c->t0s.p;
                ia.counts = c->counts.p;
                ia.offs = c->offs.p;
                LAUNCH(c, launch_index_append(ia, n_plans, maxc, c->stream));
                index_rebuild(c, tlo, thi, true);
            } else {
                index_rebuild(c, tlo, thi, false);
            }
        }
        CK(cudaStreamSynchronize(c->stream));
    } catch (...) {
        for (int32_t s : sl) c->book.free_slots.insert(s);
        throw;
    }
    for (int32_t i = 0; i < n_plans; ++i) {
        const uint64_t id = c->book.next_id++;
        c->book.plans[id] = PlanMeta{sl[i], t0s[i], counts[i]};
        c->book.S_hw = std::max(c->book.S_hw, sl[i] + 1);
        if (ids_out) ids_out[i] = id;
    }
}

// clears table rows for steps [a, b) (clipped to one window length), index rows with them
void clear_rows(fmdp_ctx* c, int64_t a, int64_t b) {
    if (b <= a) return;
    if (b - a >= c->T_win) {
        const size_t n = (size_t)c->T_win * c->S_pad;
        LAUNCH(c, launch_fill_nan(c->X, n, c->stream));
        LAUNCH(c, launch_fill_nan(c->Y, n, c->stream));
        LAUNCH(c, launch_fill_nan(c->Z, n, c->stream));
        index_reset(c);
        return;
    }
    int64_t ra = a % c->T_win;
    if (ra < 0) ra += c->T_win;
    int64_t len = b - a;
    while (len > 0) {
        const int64_t run = std::min<int64_t>(len, c->T_win - ra);
        const size_t off = (size_t)ra * c->S_pad, n = (size_t)run * c->S_pad;
        LAUNCH(c, launch_fill_nan(c->X + off, n, c->stream));
        LAUNCH(c, launch_fill_nan(c->Y + off, n, c->stream));
        LAUNCH(c, launch_fill_nan(c->Z + off, n, c->stream));
        len -= run;
        ra = 0;
    }
    index_rebuild(c, a, b, false);  // the cleared rows hold no items
}

void expire_to(fmdp_ctx* c, int64_t t_now, int64_t* n_expired) {
    if (t_now <= c->book.t_base) return;
    int64_t n = 0;
    for (auto it = c->book.plans.begin(); it != c->book.plans.end();) {
        if (it->second.t0 + it->second.n - 1 < t_now) {
            c->book.free_slots.insert(it->second.slot);
            it = c->book.plans.erase(it);
            ++n;
        } else {
            ++it;
        }
    }
    clear_rows(c, c->book.t_base, t_now);
    c->book.t_base = t_now;
    recompute_hw(c);
    CK(cudaStreamSynchronize(c->stream));
    if (n_expired) *n_expired += n;
}

void destroy_ctx(fmdp_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (float* p : {c->X, c->Y, c->Z, c->sX, c->sY, c->sZ})
        if (p) cudaFree(p);
    if (c->hm) cudaFree(c->hm);
    if (c->statics) cudaFree(c->statics);
    if (c->err) cudaFree(c->err);
    for (void* p : {(void*)c->ix_cstart, (void*)c->ix_nextra, (void*)c->ix_dirty, (void*)c->ix_items,
                    (void*)c->items_ctr})
        if (p) cudaFree(p);
    c->seq.release(); c->stg.release(); c->bat.release();
    c->mlp_p.release(); c->mlp_g.release(); c->mlp_m1.release(); c->mlp_m2.release(); c->mlp_wt.release();
    c->mlp_wp.release(); c->tX.release(); c->ty.release(); c->trX.release(); c->trH.release(); c->trdZ.release();
    c->trZ.release(); c->trdZf.release(); c->trdH.release(); c->tr_loss.release(); c->tr_idx.release();
    c->tr_y.release(); c->p_traj.release(); c->p_acts.release(); c->p_rout.release(); c->p_sep.release();
    c->p_acc.release(); c->p_queue.release(); c->p_ident.release(); c->row0.release();
    for (auto& g : c->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    c->reqs.release(); c->traj.release(); c->acts.release(); c->rout.release(); c->sepo.release();
    c->slots.release(); c->t0s.release(); c->offs.release(); c->counts.release();
    c->q_trace.release(); c->st_trace.release(); c->hd_trace.release(); c->tie_trace.release();
    c->phase.release();
    c->h_traj.release(); c->h_acts.release(); c->h_rout.release(); c->h_sep.release();
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    if (c->own) cudaStreamDestroy(c->own);
    delete c;
}

template <class F>
fmdp_status guard(fmdp_ctx* c, F&& f) {
    try {
        f();
        if (c) c->err_msg.clear();
        return FMDP_OK;
    } catch (const ApiError& e) {
        if (c) c->err_msg = e.what();
        return e.code;
    } catch (const std::bad_alloc&) {
        if (c) c->err_msg = "host allocation failed";
        return FMDP_ERR_OOM;
    } catch (const std::exception& e) {
        if (c) c->err_msg = e.what();
        return FMDP_ERR_ARG;
    } catch (...) {
        if (c) c->err_msg = "unknown error";
        return FMDP_ERR_ARG;
    }
}

}  // namespace

// Accessors for the allocation-free entry point (noalloc.cu).
namespace fmdp {
void ctx_sep_view(fmdp_ctx* c, SepView* v) {
    v->m = c->model;
    v->tab = table_view(c);
    v->S_scan = round_up(c->book.S_hw, 32);
    v->stream = c->stream;
}
void ctx_set_error(fmdp_ctx* c, const char* msg) { c->err_msg = msg ? msg : ""; }
}  // namespace fmdp

// ====================================================================== C ABI

extern "C" {

void fmdp_options_default(fmdp_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->combine = 0;
    o->wells = nullptr;
    o->n_wells = 0;
    o->goal_reward = 200.0;
    o->lookahead_W = 1;
}

fmdp_status fmdp_create(const fmdp_airspace* air, double gamma, const fmdp_action* actions, int32_t n_actions,
                        const fmdp_sep* sep, const fmdp_options* options, fmdp_ctx** out) {
    if (!out) return FMDP_ERR_ARG;
    *out = nullptr;
    fmdp_ctx* c = nullptr;
    try {
        c = new fmdp_ctx();
    } catch (...) {
        return FMDP_ERR_OOM;
    }
    fmdp_status st = guard(c, [&] {
        require(air && actions && sep, FMDP_ERR_ARG, "null airspace, actions or separation");
        const fmdp_airspace& a = *air;
        require(std::isfinite(a.x0) && std::isfinite(a.x1) && a.x1 > a.x0 && std::isfinite(a.y0) &&
                    std::isfinite(a.y1) && a.y1 > a.y0 && std::isfinite(a.z0) && std::isfinite(a.z1) && a.z1 > a.z0,
                FMDP_ERR_ARG, "airspace box must be finite with x1>x0, y1>y0, z1>z0");
        require(std::isfinite(a.dt) && a.dt > 0.0, FMDP_ERR_ARG, "dt must be > 0");
        require(gamma > 0.0 && gamma < 1.0, FMDP_ERR_ARG, "gamma must lie in (0, 1)");
        require(n_actions >= 1 && n_actions <= kMaxActions, FMDP_ERR_ARG, "1 to 32 actions");
        require(a.n_slices_window >= 4 && a.n_slices_window <= (1 << 24), FMDP_ERR_ARG, "window must hold >= 4 steps");
        require(a.max_slots >= 1 && a.max_slots <= (1 << 24), FMDP_ERR_ARG, "max_slots out of range");
        require(sep->horiz_m > 0.0 && sep->vert_m > 0.0, FMDP_ERR_ARG, "separation minima must be > 0");
        require(a.n_static_wells >= 0 && a.n_static_wells <= kMaxStatic, FMDP_ERR_ARG, "at most 64 static wells");
        require(a.n_static_wells == 0 || a.static_wells, FMDP_ERR_ARG, "null static wells");
        require(!a.heightmap || (a.hm_nx >= 2 && a.hm_ny >= 2), FMDP_ERR_ARG, "heightmap needs >= 2x2 nodes");
        std::vector<fmdp_action> acts(actions, actions + n_actions);
        for (auto& ac : acts) {
            const double q = ac.dpsi_deg / 15.0;
            require(std::isfinite(q) && std::fabs(q - std::round(q)) < 1e-9 && std::fabs(ac.dpsi_deg) <= 180.0,
                    FMDP_ERR_ARG, "heading changes must be multiples of 15 degrees within +-180");
            require(std::isfinite(ac.climb_mps), FMDP_ERR_ARG, "climb rate must be finite");
        }
        fmdp_options o;
        if (options) o = *options; else fmdp_options_default(&o);
        require(o.combine == 0 || o.combine == 1, FMDP_ERR_ARG, "combine must be 0 (max) or 1 (sum)");
        require(o.lookahead_W >= 0 && o.lookahead_W <= kMaxLookahead, FMDP_ERR_ARG, "lookahead_W must be 0 .. 16");
        require(o.goal_reward >= 0.0 && std::isfinite(o.goal_reward), FMDP_ERR_ARG, "goal reward must be >= 0");
        require(o.cluster_size >= 0 && o.cluster_size <= kMaxCluster, FMDP_ERR_ARG, "cluster size 0..16");
        require(o.threads_per_cta == 0 || (o.threads_per_cta >= 128 && o.threads_per_cta <= 384 &&
                                           o.threads_per_cta % 32 == 0),
                FMDP_ERR_ARG, "threads per CTA: 0 or a multiple of 32 in [128, 384]");
        require(o.batch_size >= 0 && o.batch_size <= kBatchMax, FMDP_ERR_ARG, "batch size 0..1024");
        require(o.index_stage_items >= 0 && o.index_stage_items <= 3000, FMDP_ERR_ARG,
                "index stage items 0..3000");
        require(o.index_vmax_mps >= 0.0 && o.index_cell_m >= 0.0, FMDP_ERR_ARG, "index bounds must be >= 0");
        std::vector<fmdp_well> wells;
        if (o.wells && o.n_wells > 0) {
            wells.assign(o.wells, o.wells + o.n_wells);
        } else {
            for (double t : {-5.0, 0.0, 5.0, 10.0, 15.0}) wells.push_back({t, 300.0 + 10.0 * t, 1000.0, 0.97});
        }
        require(wells.size() <= (size_t)kMaxWells, FMDP_ERR_ARG, "at most 8 wells per plan");
        for (auto& w : wells)
            require(w.radius_m > 0.0 && w.magnitude >= 0.0 && w.gamma > 0.0 && w.gamma < 1.0 &&
                        std::isfinite(w.tau_s),
                    FMDP_ERR_ARG, "well needs radius > 0, magnitude >= 0, gamma in (0,1)");
        for (int w = 0; w < a.n_static_wells; ++w) {
            const double* s = a.static_wells + 6 * w;
            require(std::isfinite(s[0]) && std::isfinite(s[1]) && std::isfinite(s[2]) && s[3] > 0.0 && s[4] >= 0.0 &&
                        s[5] > 0.0 && s[5] < 1.0,
                    FMDP_ERR_ARG, "static well needs finite centre, R > 0, |r| >= 0, gamma in (0,1)");
        }
        c->air = a;
        c->air.heightmap = nullptr;
        c->air.static_wells = nullptr;
        c->gamma = gamma;
        c->sep = *sep;
        c->opt = o;
        c->opt.wells = nullptr;
        c->A = n_actions;

        CK(cudaGetDevice(&c->device));
        CK(cudaDeviceGetAttribute(&c->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
        CK(cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device));
        CK(cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking));
        c->stream = c->own;
        CK(prepare_rollout_kernel((size_t)c->max_smem));
        CK(prepare_sepcheck_rows(sepcheck_rows_smem(kBatchMax)));
        CK(prepare_policy_kernel());
        CK(prepare_lookahead_kernel());

        c->T_win = a.n_slices_window;
        c->S_max = a.max_slots;
        c->S_pad = round_up(a.max_slots, 32);
        const size_t plane = (size_t)c->T_win * c->S_pad;
        CK(cudaMalloc(&c->X, plane * sizeof(float)));
        CK(cudaMalloc(&c->Y, plane * sizeof(float)));
        CK(cudaMalloc(&c->Z, plane * sizeof(float)));
        LAUNCH(c, launch_fill_nan(c->X, plane, c->stream));
        LAUNCH(c, launch_fill_nan(c->Y, plane, c->stream));
        LAUNCH(c, launch_fill_nan(c->Z, plane, c->stream));
        if (a.heightmap) {
            const size_t nh = (size_t)a.hm_nx * a.hm_ny;
            CK(cudaMalloc(&c->hm, nh * sizeof(float)));
            CK(cudaMemcpyAsync(c->hm, a.heightmap, nh * sizeof(float), cudaMemcpyHostToDevice, c->stream));
            c->air.heightmap = c->hm;
        }
        if (a.n_static_wells > 0) {
            CK(cudaMalloc(&c->statics, (size_t)a.n_static_wells * 6 * sizeof(double)));
            CK(cudaMemcpyAsync(c->statics, a.static_wells, (size_t)a.n_static_wells * 6 * sizeof(double),
                               cudaMemcpyHostToDevice, c->stream));
            c->air.static_wells = c->statics;
        }
        CK(cudaMalloc(&c->err, sizeof(int32_t)));
        CK(cudaMemsetAsync(c->err, 0, sizeof(int32_t), c->stream));
        for (int32_t s = 0; s < c->S_max; ++s) c->book.free_slots.insert(c->book.free_slots.end(), s);
        fill_model(c, wells, acts, a.static_wells);
        c->index_on = o.full_scan == 0;
        if (c->index_on) {
            c->icap_user = o.index_stage_items > 0 ? o.index_stage_items : 0;
            // cells of about 0.6 query radii (a query then spans 3 to 5 cell rows); at most 16384
            const double vmax = o.index_vmax_mps > 0.0 ? o.index_vmax_mps : 50.0;
            const double W = a.x1 - a.x0, H = a.y1 - a.y0;
            double cell = o.index_cell_m;
            if (!(cell > 0.0)) {
                const double rq = (double)c->model.reach_base + (double)c->model.tau_absmax * vmax + 80.0 * a.dt + 10.0;
                cell = std::max(0.6 * rq, std::max(W, H) / 256.0);
            }
            while (std::ceil(W / cell) * std::ceil(H / cell) > 16384.0) cell *= 1.25;
            c->ix_ncx = std::max(1, (int)std::ceil(W / cell));
            c->ix_ncy = std::max(1, (int)std::ceil(H / cell));
            c->ix_ncell = c->ix_ncx * c->ix_ncy;
            c->ix_x0 = (float)a.x0;
            c->ix_y0 = (float)a.y0;
            c->ix_inv = (float)(1.0 / cell);
            c->ix_vmax = (float)vmax;
            // 16 words of padding: rollouts stage aligned 16-byte blocks around the words they need
            CK(cudaMalloc(&c->ix_cstart, ((size_t)c->T_win * (c->ix_ncell + 1) + 16) * sizeof(int32_t)));
            CK(cudaMalloc(&c->ix_nextra, ((size_t)c->T_win + 16) * sizeof(int32_t)));
            CK(cudaMalloc(&c->ix_dirty, (size_t)c->T_win * sizeof(int32_t)));
            CK(cudaMalloc(&c->ix_items, plane * 2 * sizeof(float4)));
            CK(cudaMalloc(&c->items_ctr, sizeof(unsigned long long)));
            CK(cudaMemsetAsync(c->items_ctr, 0, sizeof(unsigned long long), c->stream));
            c->ix_smem = index_build_smem(c->ix_ncell);
            CK(prepare_index_kernels(c->ix_smem));
            index_reset(c);
        }
        CK(cudaStreamSynchronize(c->stream));
    });
    if (st != FMDP_OK) {
        g_create_error = c->err_msg;  // fmdp_last_error(NULL) reports it
        destroy_ctx(c);
        return st;
    }
    *out = c;
    return FMDP_OK;
}

void fmdp_destroy(fmdp_ctx* ctx) { destroy_ctx(ctx); }

const char* fmdp_last_error(fmdp_ctx* ctx) { return ctx ? ctx->err_msg.c_str() : g_create_error.c_str(); }

fmdp_status fmdp_set_stream(fmdp_ctx* c, void* stream) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        CK(cudaStreamSynchronize(c->stream));
        c->stream = stream ? reinterpret_cast<cudaStream_t>(stream) : c->own;
    });
}

fmdp_status fmdp_add_plan(fmdp_ctx* c, int64_t t0, const float* xyz, int32_t n, uint64_t* id_out) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] { store_plans(c, 1, &t0, &n, xyz, id_out); });
}

fmdp_status fmdp_add_plans(fmdp_ctx* c, int32_t n_plans, const int64_t* t0s, const int32_t* counts, const float* xyz,
                           uint64_t* ids_out) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] { store_plans(c, n_plans, t0s, counts, xyz, ids_out); });
}

fmdp_status fmdp_schedule(fmdp_ctx* c, const fmdp_request* req, fmdp_result* res) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        require(req && res, FMDP_ERR_ARG, "null request or result");
        check_request(c, *req);
        run_fcfs(c, req, 1, res, false);
    });
}

fmdp_status fmdp_schedule_many(fmdp_ctx* c, const fmdp_request* reqs, int32_t n, fmdp_result* res) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        require(n >= 0 && (n == 0 || (reqs && res)), FMDP_ERR_ARG, "null requests or results");
        for (int32_t i = 0; i < n; ++i) check_request(c, reqs[i]);
        run_fcfs(c, reqs, n, res, false);
    });
}

fmdp_status fmdp_stage_requests(fmdp_ctx* c, const fmdp_request* reqs, int32_t n) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        require(n >= 0 && (n == 0 || reqs), FMDP_ERR_ARG, "null requests");
        int32_t cap = 1;
        for (int32_t i = 0; i < n; ++i) {
            check_request(c, reqs[i]);
            cap = std::max(cap, reqs[i].horizon + 1);
        }
        c->staged.assign(reqs, reqs + n);
        c->staged_done = false;
        // requests go to device memory now; buffers are sized so the timed run allocates nothing
        c->stg.reqs.ensure(n);
        c->stg.slots.ensure(n);
        c->stg.traj.ensure((size_t)n * cap * 3);
        c->stg.acts.ensure((size_t)n * cap);
        c->stg.rout.ensure(n);
        c->stg.sepo.ensure(n);
        c->h_rout.ensure(n);
        c->h_sep.ensure(n);
        if (n > 0)
            CK(cudaMemcpyAsync(c->stg.reqs.p, reqs, n * sizeof(fmdp_request), cudaMemcpyHostToDevice, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    });
}

fmdp_status fmdp_schedule_staged(fmdp_ctx* c, int32_t batched, int32_t* n_admitted) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        const int32_t n = (int32_t)c->staged.size();
        require(n > 0, FMDP_ERR_ARG, "no staged requests");
        require((size_t)n <= c->book.free_slots.size(), FMDP_ERR_FULL, "not enough free slots for the staged run");
        c->staged_done = false;
        int32_t adm;
        if (batched) {
            c->staged_res.assign(n, fmdp_result{});
            adm = run_batch(c, c->staged.data(), n, c->staged_res.data(), c->stg.reqs.p, true);
        } else {
            adm = run_fcfs(c, c->staged.data(), n, nullptr, true);
        }
        c->staged_batched = batched != 0;
        c->staged_done = true;
        if (n_admitted) *n_admitted = adm;
    });
}

fmdp_status fmdp_fetch_staged(fmdp_ctx* c, fmdp_result* res, int32_t n) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        require(c->staged_done, FMDP_ERR_ARG, "no finished staged run");
        require(res && n == (int32_t)c->staged.size(), FMDP_ERR_ARG, "result count must equal the staged count");
        if (c->staged_batched) {
            const BatchBuffers& B = c->bat;
            c->h_traj.ensure((size_t)n * B.cap * 3);
            c->h_acts.ensure((size_t)n * B.cap);
            CK(cudaMemcpyAsync(c->h_traj.p, B.traj.p, (size_t)n * B.cap * 3 * sizeof(float), cudaMemcpyDeviceToHost,
                               c->stream));
            CK(cudaMemcpyAsync(c->h_acts.p, B.acts.p, (size_t)n * B.cap, cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
            for (int32_t i = 0; i < n; ++i) {
                float* xyz = res[i].xyz;
                uint8_t* acts = res[i].actions;
                res[i] = c->staged_res[i];
                res[i].xyz = xyz;
                res[i].actions = acts;
                const int32_t np = res[i].n_points;
                if (xyz) std::memcpy(xyz, c->h_traj.p + (size_t)i * B.cap * 3, (size_t)np * 12);
                if (acts && np > 1) std::memcpy(acts, c->h_acts.p + (size_t)i * B.cap, (size_t)np - 1);
            }
            return;
        }
        const int32_t cap = c->staged_cap;
        c->h_traj.ensure((size_t)n * cap * 3);
        c->h_acts.ensure((size_t)n * cap);
        CK(cudaMemcpyAsync(c->h_traj.p, c->stg.traj.p, (size_t)n * cap * 3 * sizeof(float), cudaMemcpyDeviceToHost,
                           c->stream));
        CK(cudaMemcpyAsync(c->h_acts.p, c->stg.acts.p, (size_t)n * cap, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaMemcpyAsync(c->h_rout.p, c->stg.rout.p, n * sizeof(RolloutOut), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaMemcpyAsync(c->h_sep.p, c->stg.sepo.p, n * sizeof(SepOut), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        for (int32_t i = 0; i < n; ++i) {
            const RolloutOut& ro = c->h_rout.p[i];
            fill_result(ro, c->h_sep.p[i], res + i);
            res[i].plan_id = 0;
            res[i].replanned = 0;
            if (res[i].xyz) std::memcpy(res[i].xyz, c->h_traj.p + (size_t)i * cap * 3, (size_t)ro.n_points * 12);
            if (res[i].actions && ro.n_points > 1)
                std::memcpy(res[i].actions, c->h_acts.p + (size_t)i * cap, (size_t)ro.n_points - 1);
        }
    });
}

fmdp_status fmdp_schedule_batch(fmdp_ctx* c, const fmdp_request* reqs, int32_t n, fmdp_result* res) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        require(n >= 0 && (n == 0 || (reqs && res)), FMDP_ERR_ARG, "null requests or results");
        for (int32_t i = 0; i < n; ++i) check_request(c, reqs[i]);
        run_batch(c, reqs, n, res, nullptr, false);
    });
}

fmdp_status fmdp_query_plans(fmdp_ctx* c, int64_t t_begin, int64_t t_end, uint64_t* ids, int32_t cap,
                             int32_t* n_out) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        require(n_out && (cap == 0 || ids) && cap >= 0, FMDP_ERR_ARG, "null output");
        int32_t n = 0;
        for (auto& kv : c->book.plans) {
            const PlanMeta& p = kv.second;
            if (p.t0 < t_end && p.t0 + p.n > t_begin) {
                if (n < cap) ids[n] = kv.first;
                ++n;
            }
        }
        *n_out = n;
    });
}

fmdp_status fmdp_get_plan(fmdp_ctx* c, uint64_t id, int64_t* t0_out, float* xyz, int32_t cap, int32_t* n_out) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        auto it = c->book.plans.find(id);
        require(it != c->book.plans.end(), FMDP_ERR_NOTFOUND, "no such plan");
        const PlanMeta& p = it->second;
        if (t0_out) *t0_out = p.t0;
        if (n_out) *n_out = p.n;
        if (!xyz) return;
        require(cap >= p.n, FMDP_ERR_ARG, "xyz capacity too small");
        require(p.t0 >= c->book.t_base, FMDP_ERR_RANGE, "plan start has left the window");
        c->h_traj.ensure((size_t)p.n * 3);
        float* planes[3] = {c->X, c->Y, c->Z};
        int64_t r0 = p.t0 % c->T_win;
        int64_t left = p.n, k0 = 0;
        while (left > 0) {
            const int64_t run = std::min<int64_t>(left, c->T_win - r0);
            for (int q = 0; q < 3; ++q) {
                CK(cudaMemcpy2DAsync(c->h_traj.p + (size_t)q * p.n + k0, sizeof(float),
                                     planes[q] + (size_t)r0 * c->S_pad + p.slot, (size_t)c->S_pad * sizeof(float),
                                     sizeof(float), (size_t)run, cudaMemcpyDeviceToHost, c->stream));
            }
            left -= run;
            k0 += run;
            r0 = 0;
        }
        CK(cudaStreamSynchronize(c->stream));
        for (int32_t k = 0; k < p.n; ++k)
            for (int q = 0; q < 3; ++q) xyz[3 * k + q] = c->h_traj.p[(size_t)q * p.n + k];
    });
}

fmdp_status fmdp_expire(fmdp_ctx* c, int64_t t_now) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] { expire_to(c, t_now, nullptr); });
}

fmdp_status fmdp_serve(fmdp_ctx* c, const fmdp_request* reqs, const double* arrival_s, int32_t n,
                       const fmdp_serve_options* opt, fmdp_result* res, double* latency_ms,
                       fmdp_serve_report* report) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        require(window_of(c) == 1, FMDP_ERR_ARG, "this entry point plans with lookahead_W = 1");
        require(n >= 0 && (n == 0 || (reqs && arrival_s && res)), FMDP_ERR_ARG, "null requests, arrivals or results");
        fmdp_serve_options o;
        if (opt) o = *opt; else fmdp_serve_options_default(&o);
        require(o.time_scale >= 0.0 && o.max_in_flight >= 0 && o.max_in_flight <= kBatchMax &&
                    o.max_active_plans >= 0 && o.expire_quantum >= 0,
                FMDP_ERR_ARG, "serve options out of range");
        for (int32_t i = 0; i < n; ++i) {
            check_request(c, reqs[i]);
            require(std::isfinite(arrival_s[i]) && arrival_s[i] >= 0.0 && (i == 0 || arrival_s[i] >= arrival_s[i - 1]),
                    FMDP_ERR_ARG, "arrival times must be finite, >= 0 and non-decreasing");
        }
        run_serve(c, reqs, arrival_s, n, o, res, latency_ms, report);
    });
}

fmdp_status fmdp_learned_collect(fmdp_ctx* c, const fmdp_request* reqs, int32_t n, int32_t* n_rows_out) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        require(window_of(c) == 1, FMDP_ERR_ARG, "this entry point plans with lookahead_W = 1");
        require(n >= 0 && (n == 0 || reqs), FMDP_ERR_ARG, "null requests");
        for (int32_t i = 0; i < n; ++i) check_request(c, reqs[i]);
        learned_collect(c, reqs, n);
        require(c->t_rows < INT32_MAX, FMDP_ERR_FULL, "training set too large");
        if (n_rows_out) *n_rows_out = (int32_t)c->t_rows;
    });
}

fmdp_status fmdp_learned_rows(fmdp_ctx* c, float* X, uint8_t* y, int32_t max_rows, int32_t* n_out) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        require(max_rows >= 0 && n_out, FMDP_ERR_ARG, "null output");
        const int64_t m = std::min<int64_t>(max_rows, c->t_rows);
        if (m > 0 && X) {
            std::vector<__nv_bfloat16> h((size_t)m * kFeat);
            CK(cudaMemcpyAsync(h.data(), c->tX.p, h.size() * sizeof(__nv_bfloat16), cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
            for (size_t i = 0; i < h.size(); ++i) X[i] = __bfloat162float(h[i]);
        }
        if (m > 0 && y) {
            CK(cudaMemcpyAsync(y, c->ty.p, (size_t)m, cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
        }
        *n_out = (int32_t)m;
    });
}

fmdp_status fmdp_learned_clear_rows(fmdp_ctx* c) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] { c->t_rows = 0; });
}

fmdp_status fmdp_learned_init(fmdp_ctx* c, uint64_t seed) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        std::vector<float> prm(n_params_total(), 0.f);
        SplitMix rng{seed};
        for (int l = 0; l < kLayers; ++l) {
            const double sd = std::sqrt(2.0 / layer_in(l));
            float* W = prm.data() + param_offset_W(l);
            for (size_t i = 0; i < (size_t)layer_in(l) * layer_out(l); ++i) W[i] = (float)(sd * rng.normal());
        }
        mlp_upload(c, prm.data());
    });
}

fmdp_status fmdp_learned_set_params(fmdp_ctx* c, const float* params, int32_t n) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        require(params && n == (int32_t)n_params_total(), FMDP_ERR_ARG, "expected FMDP_MLP_PARAMS parameters");
        for (int32_t i = 0; i < n; ++i) require(std::isfinite(params[i]), FMDP_ERR_ARG, "parameters must be finite");
        mlp_upload(c, params);
    });
}

fmdp_status fmdp_learned_get_params(fmdp_ctx* c, float* params, int32_t n) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        require(params && n == (int32_t)n_params_total(), FMDP_ERR_ARG, "expected FMDP_MLP_PARAMS parameters");
        require(c->mlp_ready, FMDP_ERR_ARG, "the proposal network has no parameters");
        CK(cudaMemcpyAsync(params, c->mlp_p.p, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    });
}

fmdp_status fmdp_learned_train(fmdp_ctx* c, int32_t epochs, int32_t batch, float lr, uint64_t seed,
                               float* loss_per_epoch) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] { mlp_train(c, epochs, batch, lr, seed, loss_per_epoch); });
}

fmdp_status fmdp_learned_loss_grad(fmdp_ctx* c, const float* X, const uint8_t* y, int32_t rows, float* loss,
                                   float* grad) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        require(X && y && loss && grad && rows >= 1 && rows <= 8192, FMDP_ERR_ARG, "null arrays or rows out of range");
        require(c->mlp_ready, FMDP_ERR_ARG, "the proposal network has no parameters");
        for (int32_t i = 0; i < rows; ++i) require(y[i] < c->A, FMDP_ERR_ARG, "label beyond the action set");
        std::vector<__nv_bfloat16> h((size_t)rows * kFeat);
        for (size_t i = 0; i < h.size(); ++i) h[i] = __float2bfloat16_rn(X[i]);
        c->trX.ensure((size_t)rows * kFeat);
        c->tr_y.ensure(rows);
        CK(cudaMemcpyAsync(c->trX.p, h.data(), h.size() * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(c->tr_y.p, y, rows, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemsetAsync(c->tr_loss.p, 0, sizeof(float), c->stream));
        mlp_fwd_bwd(c, c->trX.p, c->tr_y.p, rows);
        CK(cudaMemcpyAsync(loss, c->tr_loss.p, sizeof(float), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaMemcpyAsync(grad, c->mlp_g.p, n_params_total() * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    });
}

fmdp_status fmdp_learned_evaluate(fmdp_ctx* c, const fmdp_request* reqs, int32_t n, double slack,
                                  fmdp_learned_report* report, int32_t* accepted, int32_t* steps_p,
                                  int32_t* steps_f) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        require(window_of(c) == 1, FMDP_ERR_ARG, "this entry point plans with lookahead_W = 1");
        require(n >= 0 && (n == 0 || reqs), FMDP_ERR_ARG, "null requests");
        for (int32_t i = 0; i < n; ++i) check_request(c, reqs[i]);
        learned_evaluate(c, reqs, n, slack, report, accepted, steps_p, steps_f);
    });
}

fmdp_status fmdp_schedule_departures(fmdp_ctx* c, const fmdp_request* reqs, int32_t n, const int64_t* delays,
                                     int32_t n_delays, fmdp_result* res, int32_t* chosen, int32_t* verdicts) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        require(window_of(c) == 1, FMDP_ERR_ARG, "this entry point plans with lookahead_W = 1");
        require(n >= 0 && (n == 0 || (reqs && res)), FMDP_ERR_ARG, "null requests or results");
        require(n_delays >= 1 && n_delays <= kBatchMax && delays, FMDP_ERR_ARG,
                "between 1 and 1024 departure delays are required");
        for (int32_t i = 0; i < n; ++i)
            for (int32_t d = 0; d < n_delays; ++d) {
                require(std::llabs(delays[d]) < (1ll << 40), FMDP_ERR_ARG, "departure delay out of range");
                fmdp_request v = reqs[i];
                v.depart_step += delays[d];
                check_request(c, v);
            }
        run_departures(c, reqs, n, delays, n_delays, res, chosen, verdicts);
    });
}

fmdp_status fmdp_schedule_departures_batch(fmdp_ctx* c, const fmdp_request* reqs, int32_t n, const int64_t* delays,
                                           int32_t n_delays, fmdp_result* res, int32_t* chosen, int32_t* verdicts) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        require(window_of(c) == 1, FMDP_ERR_ARG, "this entry point plans with lookahead_W = 1");
        require(n >= 0 && (n == 0 || (reqs && res)), FMDP_ERR_ARG, "null requests or results");
        require(n_delays >= 1 && n_delays <= kBatchMax && delays, FMDP_ERR_ARG,
                "between 1 and 1024 departure delays are required");
        require((int64_t)n * n_delays <= (1 << 24), FMDP_ERR_ARG, "at most 2^24 variants per call");
        for (int32_t i = 0; i < n; ++i)
            for (int32_t d = 0; d < n_delays; ++d) {
                require(std::llabs(delays[d]) < (1ll << 40), FMDP_ERR_ARG, "departure delay out of range");
                fmdp_request v = reqs[i];
                v.depart_step += delays[d];
                check_request(c, v);
            }
        run_departures_batch(c, reqs, n, delays, n_delays, res, chosen, verdicts);
    });
}

fmdp_status fmdp_schedule_cosim(fmdp_ctx* c, const fmdp_request* reqs, int32_t n, fmdp_result* res) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        require(n >= 0 && (n == 0 || (reqs && res)), FMDP_ERR_ARG, "null requests or results");
        for (int32_t i = 0; i < n; ++i) check_request(c, reqs[i]);
        if (n == 0) return;
        const int32_t fit = lookahead_max_resident(c->A, window_of(c));
        require(n <= fit, FMDP_ERR_ARG, "co-simulated batch larger than the CTAs one launch keeps resident");
        require((size_t)n <= c->book.free_slots.size(), FMDP_ERR_FULL, "not enough free slots for the co-simulated batch");
        run_fcfs(c, reqs, n, res, false, true);
    });
}

fmdp_status fmdp_selftest_wait_timeout(fmdp_ctx* c, int32_t* observed) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        // two requests far from everything, co-simulated with a barrier that also waits for
        // a third aircraft that is never launched: every wait must run out and report
        fmdp_request r[2] = {};
        const double cx = 0.5 * (c->air.x0 + c->air.x1), cy = 0.5 * (c->air.y0 + c->air.y1);
        const double cz = 0.5 * (c->air.z0 + c->air.z1);
        for (int i = 0; i < 2; ++i) {
            r[i].req_id = (uint64_t)(i + 1);
            r[i].ox = cx;
            r[i].oy = cy + (i ? 1.0 : -1.0);
            r[i].oz = cz;
            r[i].gx = cx + 1.0;
            r[i].gy = r[i].oy;
            r[i].gz = cz;
            r[i].speed_mps = 1.0;
            r[i].depart_step = c->book.t_base;
            r[i].horizon = 4;
            check_request(c, r[i]);
        }
        const size_t plans_before = c->book.plans.size();
        int32_t st = FMDP_OK;
        try {
            run_fcfs(c, r, 2, nullptr, false, true, 1);
        } catch (const ApiError& f) {
            st = f.code;
        }
        if (observed) *observed = st;
        require(st == FMDP_ERR_TIMEOUT, FMDP_ERR_CUDA, "the self-test wait did not report a timeout");
        require(c->book.plans.size() == plans_before, FMDP_ERR_CUDA, "the self-test admitted a plan");
    });
}

fmdp_status fmdp_autotune(fmdp_ctx* c, const fmdp_request* sample, int32_t n, int32_t force,
                          fmdp_tune_report* report) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        require(window_of(c) == 1, FMDP_ERR_ARG, "this entry point plans with lookahead_W = 1");
        require(n >= 1 && sample, FMDP_ERR_ARG, "the autotuner needs at least one sample request");
        for (int32_t i = 0; i < n; ++i) check_request(c, sample[i]);
        autotune(c, sample, n, force != 0, report);
    });
}

fmdp_status fmdp_tune_cache_get(fmdp_ctx* c, fmdp_tune_entry* out, int32_t cap, int32_t* n_out) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        require(cap >= 0 && (cap == 0 || out), FMDP_ERR_ARG, "null output");
        int32_t i = 0;
        for (const auto& kv : c->tune) {
            if (i < cap) out[i] = kv.second;
            ++i;
        }
        if (n_out) *n_out = i;
    });
}

fmdp_status fmdp_tune_cache_put(fmdp_ctx* c, const fmdp_tune_entry* in, int32_t n) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        require(n >= 0 && (n == 0 || in), FMDP_ERR_ARG, "null entries");
        for (int32_t i = 0; i < n; ++i)
            require(tune_shape_ok(in[i].threads_per_cta, in[i].index_stage_items) &&
                        rollout_smem_bytes(0, 0, in[i].index_stage_items) <= (size_t)c->max_smem,
                    FMDP_ERR_ARG, "tune entry outside the candidate shapes");
        for (int32_t i = 0; i < n; ++i)
            c->tune[{in[i].n_actions, in[i].combine, in[i].plans_bucket, in[i].wave_bucket}] = in[i];
    });
}

fmdp_status fmdp_schedule_learned(fmdp_ctx* c, const fmdp_request* reqs, int32_t n, double slack, fmdp_result* res,
                                  fmdp_learned_report* report) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        require(window_of(c) == 1, FMDP_ERR_ARG, "this entry point plans with lookahead_W = 1");
        require(n >= 0 && (n == 0 || (reqs && res)), FMDP_ERR_ARG, "null requests or results");
        require(c->index_on, FMDP_ERR_ARG, "the learned proposal reads the spatial index (full_scan must be 0)");
        require(c->mlp_ready, FMDP_ERR_ARG, "the proposal network has no parameters (init or set them first)");
        require(slack >= 0.0 && std::isfinite(slack), FMDP_ERR_ARG, "slack must be >= 0");
        for (int32_t i = 0; i < n; ++i) check_request(c, reqs[i]);
        c->learned_mode = true;
        c->slack = slack;
        try {
            run_batch(c, reqs, n, res, nullptr, false);
        } catch (...) {
            c->learned_mode = false;
            throw;
        }
        c->learned_mode = false;
        std::vector<int32_t> acc(std::max(n, 1));
        if (n > 0) {
            CK(cudaMemcpyAsync(acc.data(), c->p_acc.p, n * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
        }
        fmdp_learned_report r{};
        r.n = n;
        for (int32_t i = 0; i < n; ++i) {
            res[i].source = acc[i] ? 1 : 0;
            r.accepted += acc[i] ? 1 : 0;
        }
        if (report) *report = r;
    });
}

void fmdp_serve_options_default(fmdp_serve_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->time_scale = 1.0;
}

fmdp_status fmdp_snapshot(fmdp_ctx* c) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        const size_t plane = (size_t)c->T_win * c->S_pad * sizeof(float);
        if (!c->sX) {
            CK(cudaMalloc(&c->sX, plane));
            CK(cudaMalloc(&c->sY, plane));
            CK(cudaMalloc(&c->sZ, plane));
        }
        CK(cudaMemcpyAsync(c->sX, c->X, plane, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(c->sY, c->Y, plane, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(c->sZ, c->Z, plane, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        c->snap = c->book;
        c->has_snap = true;
    });
}

fmdp_status fmdp_restore(fmdp_ctx* c) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        require(c->has_snap, FMDP_ERR_ARG, "no snapshot");
        const size_t plane = (size_t)c->T_win * c->S_pad * sizeof(float);
        CK(cudaMemcpyAsync(c->X, c->sX, plane, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(c->Y, c->sY, plane, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(c->Z, c->sZ, plane, cudaMemcpyDeviceToDevice, c->stream));
        c->book = c->snap;
        index_rebuild_all(c);
        CK(cudaStreamSynchronize(c->stream));
    });
}

fmdp_status fmdp_clear(fmdp_ctx* c) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        const size_t plane = (size_t)c->T_win * c->S_pad;
        LAUNCH(c, launch_fill_nan(c->X, plane, c->stream));
        LAUNCH(c, launch_fill_nan(c->Y, plane, c->stream));
        LAUNCH(c, launch_fill_nan(c->Z, plane, c->stream));
        index_reset(c);
        CK(cudaStreamSynchronize(c->stream));
        const int64_t tb = c->book.t_base;
        c->book = Book();
        c->book.t_base = tb;
        for (int32_t s = 0; s < c->S_max; ++s) c->book.free_slots.insert(c->book.free_slots.end(), s);
    });
}

fmdp_status fmdp_rollout_trace(fmdp_ctx* c, const fmdp_request* req, fmdp_result* res, double* q, double* states,
                               int32_t* headings, uint8_t* tie_flags) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        require(req && res, FMDP_ERR_ARG, "null request or result");
        check_request(c, *req);
        const int32_t cap = req->horizon + 1;
        const Geometry g = geometry(c, c->book.S_hw);
        c->reqs.ensure(1);
        c->traj.ensure((size_t)cap * 3);
        c->acts.ensure((size_t)cap);
        c->rout.ensure(1);
        c->q_trace.ensure((size_t)cap * c->A);
        c->st_trace.ensure((size_t)cap * 3);
        c->hd_trace.ensure((size_t)cap);
        c->tie_trace.ensure((size_t)cap);
        CK(cudaMemcpyAsync(c->reqs.p, req, sizeof(fmdp_request), cudaMemcpyHostToDevice, c->stream));
        RolloutArgs ra{};
        ra.m = c->model;
        ra.tab = table_view(c);
        ra.S_scan = g.S_scan;
        ra.chunk = g.chunk;
        ra.cs = g.cs;
        ra.ring = g.ring;
        ra.cap = cap;
        ra.reqs = c->reqs.p;
        ra.n_req = 1;
        ra.trace = 1;
        ra.traj = c->traj.p;
        ra.acts = c->acts.p;
        ra.out = c->rout.p;
        ra.q_trace = c->q_trace.p;
        ra.st_trace = c->st_trace.p;
        ra.hd_trace = c->hd_trace.p;
        ra.tie_trace = c->tie_trace.p;
        ra.err = c->err;
        set_index_args(c, ra, g);
        if (window_of(c) > 1)
            launch_window_rollout(c, g, c->reqs.p, cap, c->traj.p, c->acts.p, c->rout.p, true);
        else
            LAUNCH(c, launch_rollout(ra, g.threads, g.smem, c->stream));
        RolloutOut ro;
        CK(cudaMemcpyAsync(&ro, c->rout.p, sizeof(ro), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        require(read_error_word(c) == 0, FMDP_ERR_TIMEOUT, "a bounded device wait expired during a rollout");
        const int32_t np = ro.n_points, ns = np - 1;
        if (res->xyz) CK(cudaMemcpy(res->xyz, c->traj.p, (size_t)np * 12, cudaMemcpyDeviceToHost));
        if (res->actions && ns > 0) CK(cudaMemcpy(res->actions, c->acts.p, (size_t)ns, cudaMemcpyDeviceToHost));
        const int32_t qrows = ro.status == FMDP_REJ_NO_ACTION ? ns + 1 : ns;
        if (q && qrows > 0) CK(cudaMemcpy(q, c->q_trace.p, (size_t)qrows * c->A * sizeof(double), cudaMemcpyDeviceToHost));
        if (states) CK(cudaMemcpy(states, c->st_trace.p, (size_t)np * 3 * sizeof(double), cudaMemcpyDeviceToHost));
        if (headings) CK(cudaMemcpy(headings, c->hd_trace.p, (size_t)np * sizeof(int32_t), cudaMemcpyDeviceToHost));
        if (tie_flags && ns > 0) CK(cudaMemcpy(tie_flags, c->tie_trace.p, (size_t)ns, cudaMemcpyDeviceToHost));
        res->verdict = ro.status == kStatusCaptured ? FMDP_ADMITTED : ro.status;
        res->n_points = np;
        res->plan_id = 0;
        res->first_conflict_step = -1;
        res->first_terrain_step = -1;
        res->min_sep_h = INFINITY;
        res->min_sep_v = INFINITY;
        res->near_ties = ro.near_ties;
        res->replanned = 0;
    });
}

fmdp_status fmdp_sep_check(fmdp_ctx* c, int64_t t0, const float* xyz, int32_t n, fmdp_sep_report* out) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        require(xyz && out && n >= 1, FMDP_ERR_ARG, "null trajectory or output");
        const int32_t S_scan = round_up(c->book.S_hw, 32);
        c->traj.ensure((size_t)n * 3);
        c->sepo.ensure(1);
        CK(cudaMemcpyAsync(c->traj.p, xyz, (size_t)n * 12, cudaMemcpyHostToDevice, c->stream));
        LAUNCH(c, launch_sep_reset(c->sepo.p, 1, c->stream));
        SepArgs sa{};
        sa.m = c->model;
        sa.tab = table_view(c);
        sa.S_scan = S_scan;
        sa.cap = n;
        sa.traj = c->traj.p;
        sa.rout = nullptr;
        sa.reqs = nullptr;
        sa.t0_fixed = t0;
        sa.n_fixed = n;
        sa.out = c->sepo.p;
        {
            KernelTimer t(c, 1);
            LAUNCH(c, launch_sepcheck(sa, 1, n, c->stream));
            t.stop();
        }
        SepOut so;
        CK(cudaMemcpyAsync(&so, c->sepo.p, sizeof(so), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        if (c->profiling) collect_timers(c);
        c->stats.sep_pairs += (int64_t)n * S_scan;
        out->first_conflict_step = so.first_conflict == INT_MAX ? -1 : so.first_conflict;
        out->first_terrain_step = so.first_terrain == INT_MAX ? -1 : so.first_terrain;
        out->conflicts = (int64_t)so.conflicts;
        float mh, mv;
        std::memcpy(&mh, &so.min_h_bits, 4);
        std::memcpy(&mv, &so.min_v_bits, 4);
        out->min_sep_h = mh;
        out->min_sep_v = mv;
    });
}

fmdp_status fmdp_set_profiling(fmdp_ctx* c, int32_t on) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        c->profiling = on != 0;
        c->phase_timing = on == 2;
        c->stats = fmdp_stats{};
        c->pending.clear();
        c->ev_next = 0;
        if (c->items_ctr) CK(cudaMemsetAsync(c->items_ctr, 0, sizeof(unsigned long long), c->stream));
        if (c->phase_timing) {
            c->phase.ensure(6);
            CK(cudaMemsetAsync(c->phase.p, 0, 6 * sizeof(unsigned long long), c->stream));
            CK(cudaStreamSynchronize(c->stream));
        }
    });
}

fmdp_status fmdp_get_stats(fmdp_ctx* c, fmdp_stats* out) {
    if (!c || !out) return FMDP_ERR_ARG;
    return guard(c, [&] {
        *out = c->stats;
        if (c->phase_timing) {
            unsigned long long ph[6];
            CK(cudaMemcpyAsync(ph, c->phase.p, sizeof(ph), cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
            for (int i = 0; i < 6; ++i) out->phase_cycles[i] = (int64_t)ph[i];
        }
        if (c->items_ctr) {
            unsigned long long n = 0;
            CK(cudaMemcpyAsync(&n, c->items_ctr, sizeof(n), cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
            out->items_scanned = (int64_t)n;
        }
        out->cluster_size = c->last_cs;
        out->threads_per_cta = c->last_threads;
        out->slots_per_cta = c->last_chunk;
    });
}

}  // extern "C"
