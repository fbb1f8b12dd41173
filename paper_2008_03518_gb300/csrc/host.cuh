// Host runtime internals of libfmdp: error handling, device and pinned arrays, the
// scheduler context (fmdp_ctx) and the functions the host sources share.
#pragma once

#include <algorithm>
#include <chrono>
#include <thread>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <array>
#include <atomic>
#include <map>
#include <new>
#include <set>
#include <functional>
#include <stdexcept>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "learned.cuh"
#include "plan_book.h"

namespace fmdp {

struct ApiError : std::runtime_error {
    fmdp_status code;
    ApiError(fmdp_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

inline void cuda_check(cudaError_t e, const char* what) {
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

inline void require(bool ok, fmdp_status code, const std::string& msg) {
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

inline int32_t round_up(int32_t x, int32_t m) { return (x + m - 1) / m * m; }

constexpr int32_t kExtraLimit = 48;  // appended items per index row before the row is rebuilt

struct PipeState;  // pipelined FCFS (host_pipeline.cu)

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

}  // namespace fmdp

// The opaque context of the C ABI (global, as include/fmdp.h declares it).
using namespace fmdp;

struct fmdp_ctx {
    Model model{};
    fmdp_airspace air{};
    double gamma = 0.0;
    fmdp_sep sep{};
    fmdp_options opt{};
    int32_t A = 0;

    cudaStream_t own = nullptr;
    cudaStream_t stream = nullptr;
    int device = -1;  // recorded by fmdp_create (the device current at creation)
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
    int32_t* ix_nres = nullptr;
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

    // per-request completion times of the last scheduling call (ms from its start); the
    // sequential path records an event after each request (req_ev, from req_ev_base)
    std::vector<double> call_ms;
    std::vector<cudaEvent_t> req_ev;
    int32_t req_ev_base = -1;  // -1: no recording

    // pipelined FCFS: streams, host-mapped ring and reports, ordinals (host_pipeline.cu)
    PipeState* pipe = nullptr;
    int32_t extra_limit = kExtraLimit;  // appended items per index row before it is marked dirty

    // allocation-free separation check: device address of the library's static scratch
    // array on this context's device (looked up by the context's first such call)
    void* noalloc_scratch = nullptr;
};

namespace fmdp {

cudaEvent_t next_event(fmdp_ctx* c);
struct Geometry;

// Names a coarse host phase on timeline tools (an NVTX range; nothing happens unless a tool
// is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
struct KernelTimer {
    fmdp_ctx* c;
    int kind;
    cudaStream_t s;  // the stream the timed kernels run on
    cudaEvent_t a = nullptr;
    KernelTimer(fmdp_ctx* c_, int k, cudaStream_t st = nullptr) : c(c_), kind(k), s(st ? st : c_->stream) {
        if (c->profiling && kind >= 0) {
            a = next_event(c);
            CK(cudaEventRecord(a, s));
        }
    }
    void stop() {
        if (c->profiling && kind >= 0) {
            cudaEvent_t b = next_event(c);
            CK(cudaEventRecord(b, s));
            c->pending.push_back({kind, a, b});
        }
    }
};
// launch shape of a rollout
struct Geometry {
    int32_t S_scan, cs, threads, chunk, ring;
    int32_t icap = 0;  // indexed mode: plan samples staged per step
    size_t smem;
};
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
// ------------------------------------------------------------------ shared constants

constexpr int32_t kBatchDefault = 256;
constexpr int32_t kBatchMax = 1024;

// ------------------------------------------------------------------ host runtime (host_table.cu)

void fill_model(fmdp_ctx* c, const std::vector<fmdp_well>& wells, const std::vector<fmdp_action>& actions,
                const double* host_statics);
TableView table_view(fmdp_ctx* c);
cudaEvent_t next_event(fmdp_ctx* c);
void collect_timers(fmdp_ctx* c);
IndexArgs index_args(fmdp_ctx* c);
IndexView index_view(fmdp_ctx* c);
void set_index_args(fmdp_ctx* c, RolloutArgs& ra, const Geometry& g);
void index_rebuild(fmdp_ctx* c, int64_t a, int64_t b, bool dirty_only);
void index_rebuild_all(fmdp_ctx* c);
void index_reset(fmdp_ctx* c);
void index_append_admitted(fmdp_ctx* c, const float* traj, int32_t cap, const RolloutOut* rout,
                           const fmdp_request* reqs, const SepOut* sep, const int32_t* slots, const int32_t* idx,
                           const int32_t* n_dev, int32_t n_items, int64_t t_lo, int64_t t_hi,
                           bool rebuild_dirty = true);
bool fit_geometry(fmdp_ctx* c, Geometry& g, int cs);
int32_t bit_length(int64_t v);
int32_t batch_size_of(const fmdp_ctx* c);
int32_t window_of(const fmdp_ctx* c);
void launch_window_rollout(fmdp_ctx* c, const Geometry& g, const fmdp_request* req_dev, int32_t cap, float* traj,
                           uint8_t* acts, RolloutOut* out, bool trace);
std::array<int32_t, 4> tune_key(const fmdp_ctx* c, int32_t wave);
const fmdp_tune_entry* tune_lookup(const fmdp_ctx* c, int32_t wave);
Geometry geometry_indexed(fmdp_ctx* c, int32_t S_scan, int32_t wave = 0);
Geometry geometry(fmdp_ctx* c, int32_t S_hw);
void check_request(fmdp_ctx* c, const fmdp_request& r);
int32_t take_slot(fmdp_ctx* c);
void recompute_hw(fmdp_ctx* c);
void enqueue_sequence(fmdp_ctx* c, SeqBuffers& B, const fmdp_request* host_reqs, int32_t n, int32_t cap,
                      const Geometry& g, bool plan = true);
int32_t read_error_word(fmdp_ctx* c);
void fill_result(const RolloutOut& ro, const SepOut& so, fmdp_result* res);
void store_plans(fmdp_ctx* c, int32_t n_plans, const int64_t* t0s, const int32_t* counts, const float* xyz,
                 uint64_t* ids_out);
void clear_rows(fmdp_ctx* c, int64_t a, int64_t b);
// Expires the plans that ended before t_now and moves the window to start there (device
// work on the context's stream; sync: wait for it).
void expire_to(fmdp_ctx* c, int64_t t_now, int64_t* n_expired, bool sync = true);
void destroy_ctx(fmdp_ctx* c);

// ------------------------------------------------------------------ FCFS (host_fcfs.cu)

int32_t run_fcfs(fmdp_ctx* c, const fmdp_request* reqs, int32_t n, fmdp_result* res, bool staged,
                 bool cosim = false, int32_t absent = 0);

// ------------------------------------------------------------------ speculative batches (host_batch.cu)

int wave_kernels(const fmdp_ctx* c);
Geometry geometry_batch(fmdp_ctx* c, int32_t S, int32_t wave);
int32_t host_verdict(const RolloutOut& ro, const SepOut& so);
size_t idx_words(const BatchBuffers& B);
double climb_step(const fmdp_ctx* c);
void enqueue_wave(fmdp_ctx* c, const Geometry& g, int n_clusters, BatchBuffers& B, bool timed);
cudaGraphExec_t wave_graph(fmdp_ctx* c, const Geometry& g, int n_clusters, BatchBuffers& B);
void batch_prepare(fmdp_ctx* c, const fmdp_request* reqs, int32_t n, int32_t n_batch, const fmdp_request* dev_reqs);
Geometry batch_geometry(fmdp_ctx* c, int32_t n_new, int32_t wave);
void copy_points_back(fmdp_ctx* c, int32_t n, fmdp_result* res);
int32_t run_batch(fmdp_ctx* c, const fmdp_request* reqs, int32_t n, fmdp_result* res,
                  const fmdp_request* dev_reqs, bool keep_points);
void plan_all_fastmdp(fmdp_ctx* c, int32_t n);
void run_departures(fmdp_ctx* c, const fmdp_request* reqs, int32_t n, const int64_t* delays, int32_t D,
                    fmdp_result* res, int32_t* chosen, int32_t* verdicts);
void run_departures_batch(fmdp_ctx* c, const fmdp_request* reqs, int32_t n, const int64_t* delays, int32_t D,
                          fmdp_result* res, int32_t* chosen, int32_t* verdicts);
bool tune_shape_ok(int32_t threads, int32_t icap);
void autotune(fmdp_ctx* c, const fmdp_request* sample, int32_t n, bool force, fmdp_tune_report* rep);

// ------------------------------------------------------------------ learned proposal (host_learned.cu)

size_t wt_offset(int l);
void mlp_ensure(fmdp_ctx* c);
void mlp_upload(fmdp_ctx* c, const float* params);
void mlp_fwd_bwd(fmdp_ctx* c, const __nv_bfloat16* X, const uint8_t* y, int B);
void mlp_train(fmdp_ctx* c, int32_t epochs, int32_t batch, float lr, uint64_t seed, float* losses);
void learned_collect(fmdp_ctx* c, const fmdp_request* reqs, int32_t n);
void learned_evaluate(fmdp_ctx* c, const fmdp_request* reqs, int32_t n, double slack, fmdp_learned_report* rep,
                      int32_t* accepted, int32_t* steps_p, int32_t* steps_f);

// ------------------------------------------------------------------ pipelined FCFS (host_pipeline.cu)

// The arrival trace and options of a serving call.
struct PipeServe {
    const double* arrival_s;
    fmdp_serve_options o;
    double* latency_ms;
    fmdp_serve_report* rep;
};
bool pipeline_eligible(const fmdp_ctx* c);
struct PipeServe;
bool pipeline_fits(fmdp_ctx* c, int32_t n, const PipeServe* serve);
int32_t run_pipeline(fmdp_ctx* c, const fmdp_request* reqs, int32_t n, fmdp_result* res,
                     const fmdp_request* dev_reqs, bool keep_points, const PipeServe* serve);
void pipe_release(fmdp_ctx* c);

// ------------------------------------------------------------------ serving (host_serve.cu)

void run_serve(fmdp_ctx* c, const fmdp_request* reqs, const double* arrival_s, int32_t n,
               const fmdp_serve_options& o, fmdp_result* res, double* latency_ms, fmdp_serve_report* rep);

// Makes `dev` the current device for its lifetime and restores the caller's device after,
// so that a call runs on its context's device whichever device the caller has current.
struct DeviceScope {
    int prev = -1;
    explicit DeviceScope(int dev) {
        int cur = -1;
        if (dev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != dev && cudaSetDevice(dev) == cudaSuccess)
            prev = cur;
    }
    ~DeviceScope() {
        if (prev >= 0) cudaSetDevice(prev);
    }
    DeviceScope(const DeviceScope&) = delete;
    DeviceScope& operator=(const DeviceScope&) = delete;
};

// Runs f on the context's device, translating exceptions into a status and the context's
// error message.
template <class F>
fmdp_status guard(fmdp_ctx* c, F&& f) {
    DeviceScope on_device(c ? c->device : -1);
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

}  // namespace fmdp
