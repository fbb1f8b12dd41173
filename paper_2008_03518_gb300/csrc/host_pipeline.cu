// Pipelined speculative FCFS: continuous batching without waves.
//
// First-come-first-served planning (Sec. I, Sec. V) admits request k against every plan
// admitted before it. Speculative batching plans many requests at once and keeps a plan
// only when nothing it did not see could have changed it (the influence test). Here the
// planning never stops at a wave boundary:
//   - one persistent rollout launch (one CTA per work item) takes work items from a ring
//     in host-mapped memory that the host appends to while the launch runs;
//   - each finished plan is checked for conflicts against the plans its request's table
//     holds at that moment and reported, with its trajectory, to host-mapped memory;
//   - the requests just behind the head of the line publish their current plans as
//     tentative plans in the index: a tentative plan of request j is part of the table of
//     every later request (the guess that j will be admitted as planned), so a later
//     request plans against it at once instead of after j's admission. A superseded or
//     rejected tentative plan is withdrawn;
//   - the host walks the requests in arrival order: a request is final once every change of
//     an earlier request's contribution (a tentative plan published or withdrawn) has been
//     tested against its plan and none influences it; an admitted request is stored on a
//     high-priority table stream, beside the running rollouts, and its tentative plan stays;
//   - a plan that a change influences is planned again as soon as the change is visible,
//     from the first step it can alter (the steps before it keep their decisions).
// Exactness. FastMDP's choice at a step depends only on the state and the table at the next
// step, and a plan whose wells cannot reach the successors adds an exact zero. Every table
// change (an index append then its publication, or a withdrawal) is a numbered operation
// that raises a device counter when it completes; each rollout step records the counter it
// read before the index rows it valued, so the host knows, step by step, which items of an
// earlier request's plans the step saw for certain (those of every operation up to the
// counter) and which it may have seen (any later operation). A step is exact if the earlier
// requests' final contributions were visible to it and nothing else of theirs was, or if
// the difference has no influence at that step; the walk tests exactly the differences. An
// appended item becomes visible only when complete, and a withdrawal only flips its tag, so
// each item is read either whole or not at all. A plan resumed from a later step keeps the
// items of its unchanged first samples in place (only the items past them are withdrawn and
// appended), so no read misses those. Row rebuilds, which move items, happen only while no
// rollout runs; the tentative plans are published again after them. The exact
// separation report of each request (minimum separations to every earlier plan) comes from
// the row-major check with an ordinal filter: it skips plans of later requests.
#include "host.cuh"
#include "pipe_influence.cuh"

namespace fmdp {

namespace {

// Pinned host memory mapped into the device address space.
template <class T>
struct MappedArray {
    T* p = nullptr;  // host pointer
    T* d = nullptr;  // device pointer of the same memory
    size_t n = 0;
    void ensure(size_t want) {
        if (want <= n) return;
        release();
        const size_t m = std::max<size_t>(want, 16);
        CK(cudaHostAlloc((void**)&p, m * sizeof(T), cudaHostAllocMapped | cudaHostAllocPortable));
        n = m;
        CK(cudaHostGetDevicePointer((void**)&d, p, 0));
    }
    void release() {
        if (p) cudaFreeHost(p);
        p = d = nullptr;
        n = 0;
    }
};

constexpr int kQueueCap = 4096;           // ring entries (a power of two)
constexpr int kRepSlots = 8;              // staging slots of the asynchronous separation reports
constexpr int kRepChunk = 64;             // finished requests per report while the launch runs
constexpr int32_t kPipeExtraLimit = 768;  // appended items per row before the rows are rebuilt (default)
constexpr int32_t kPublishAhead = 128;    // requests past the head whose plans are published
constexpr int32_t kOrdLimit = 1 << 30;    // ordinals are rebased before they reach this

}  // namespace

struct PipeState {
    cudaStream_t pstream = nullptr;  // the persistent rollout launch
    cudaStream_t tstream = nullptr;  // table operations (admission, index, expiry), high priority
    cudaEvent_t kern_ev = nullptr;   // recorded after each persistent launch
    cudaEvent_t sync_ev = nullptr;
    MappedArray<PipeItem> ring;
    MappedArray<int32_t> ctl;  // [0] tail, [1] stop
    MappedArray<int32_t> done;
    MappedArray<PipeRecord> rec;
    MappedArray<float> h_traj;
    MappedArray<int32_t> h_slot;  // slot of an admitted request (read by its admission)
    MappedArray<int32_t> h_obs;   // per plan step: table operations done when its rows were read
    DevArray<int32_t> head, pub_seq, obs, tpos;
    DevArray<double> st_s;  // per trajectory point: what a resumed plan starts from
    DevArray<float> st_df;
    DevArray<uint8_t> st_h, ties;
    DevArray<SepOut> sep;
    DevArray<int32_t> slot_ord, req_ord, list, nlist;
    PinnedArray<int32_t> h_list;
    cudaEvent_t rep_ev[kRepSlots] = {};  // separation reports: a staging slot is free again after its event
    bool rep_used[kRepSlots] = {};
    int rep_next = 0;
    std::vector<cudaEvent_t> ev_free;
    int32_t ord_base = 0;
    bool ord_init = false;
    ~PipeState() {
        if (pstream) cudaStreamSynchronize(pstream);
        if (tstream) cudaStreamSynchronize(tstream);
        ring.release(); ctl.release(); done.release(); rec.release(); h_traj.release(); h_slot.release();
        h_obs.release(); pub_seq.release(); obs.release(); tpos.release(); st_s.release(); st_df.release();
        st_h.release(); ties.release();
        head.release(); sep.release(); slot_ord.release(); req_ord.release(); list.release(); nlist.release();
        h_list.release();
        for (cudaEvent_t e : rep_ev)
            if (e) cudaEventDestroy(e);
        for (cudaEvent_t e : ev_free) cudaEventDestroy(e);
        if (kern_ev) cudaEventDestroy(kern_ev);
        if (sync_ev) cudaEventDestroy(sync_ev);
        if (pstream) cudaStreamDestroy(pstream);
        if (tstream) cudaStreamDestroy(tstream);
    }
};

void pipe_release(fmdp_ctx* c) {
    delete c->pipe;
    c->pipe = nullptr;
}

bool pipeline_eligible(const fmdp_ctx* c) {
    return c->index_on && window_of(c) == 1 && !c->learned_mode && c->opt.batch_mode == 0 && c->model.A <= 32;
}

namespace {

int32_t pipeline_window(const fmdp_ctx* c, const PipeServe* serve) {
    const int32_t bs = c->opt.batch_size > 0 ? c->opt.batch_size : kBatchDefault;
    int32_t window = std::max(1, std::min(bs, kBatchMax));
    if (serve && serve->o.max_in_flight > 0) window = std::min(serve->o.max_in_flight, kBatchMax);
    return window;
}

// Items each index row holds now (built items + appended ones), from the device.
std::vector<int32_t> row_fill(fmdp_ctx* c) {
    const int32_t W = c->T_win;
    std::vector<int32_t> built(W), extra(W);
    CK(cudaMemcpy2DAsync(built.data(), sizeof(int32_t), c->ix_cstart + c->ix_ncell,
                         (size_t)(c->ix_ncell + 1) * sizeof(int32_t), sizeof(int32_t), W, cudaMemcpyDeviceToHost,
                         c->stream));
    CK(cudaMemcpyAsync(extra.data(), c->ix_nres, (size_t)W * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int32_t r = 0; r < W; ++r) built[r] += extra[r];
    return built;
}

// Appends a row can still receive after the pipeline decided to rebuild the rows: dispatch
// stops at that moment, so each request of the window appends at most its latest plan.
int32_t append_margin(int32_t window, int32_t n) { return std::min(window, n) + 2; }

}  // namespace

// Room for the pipelined mode's appends in every index row (an item that finds its row full
// would be lost, so the mode runs only where the rows have room for the appends a rebuild
// margin allows, and a few more); otherwise the caller batches in waves.
bool pipeline_fits(fmdp_ctx* c, int32_t n, const PipeServe* serve) {
    const std::vector<int32_t> fill = row_fill(c);
    const int32_t mx = fill.empty() ? 0 : *std::max_element(fill.begin(), fill.end());
    return (int64_t)mx + append_margin(pipeline_window(c, serve), n) + 32 <= c->S_pad;
}

namespace {

static_assert(kInflWells == kMaxWells, "the influence rule holds every well of a plan");

enum Phase : uint8_t { kAbsent = 0, kWait = 1, kFlight = 2, kDone = 3, kFinal = 4 };

// A published tentative plan of one request. A read that acquired the table-operation count q
// sees the work of every operation up to q and may see any part of a later one: an item
// appended by operation a and withdrawn by operation w is seen by the reads with
// a <= q < w and may be seen by any read with q < w. q_pub: the operation that appended this
// version's items past the ones it kept from the version before it; q_kill: the one that
// withdrew its items past the ones the next version kept; q_from: the one that appended the
// oldest item it holds (the first version of the chain whose versions kept items from one
// another).
struct Version {
    int32_t j;
    int32_t n;
    int32_t q_pub, q_kill;
    int32_t q_from;
    std::vector<float> xyz;
    TrajBoxes boxes;
};

// A change of request j's contribution to the tables of later requests.
struct Change {
    int32_t j;
    int32_t v_old, v_new;  // versions withdrawn and published (-1: none)
    int32_t q_last;        // the last table operation of the change
    int32_t keep;          // items [0, keep) of both versions are the same ones, left in place
};

}  // namespace

// One pipelined call (see the top of this file). serve == nullptr: every request is there
// from the start (fmdp_schedule_batch); else the arrival trace and options of fmdp_serve.
int32_t run_pipeline(fmdp_ctx* c, const fmdp_request* reqs, int32_t n, fmdp_result* res,
                     const fmdp_request* dev_reqs, bool keep_points, const PipeServe* serve) {
    using clk = std::chrono::steady_clock;
    if (n <= 0) return 0;
    const NvtxRange range("fmdp pipelined FCFS");
    require(pipeline_eligible(c), FMDP_ERR_ARG, "internal: pipelined FCFS needs the index and W = 1");
    const int32_t window = pipeline_window(c, serve);
    batch_prepare(c, reqs, n, window, dev_reqs);
    BatchBuffers& B = c->bat;
    const int32_t cap = B.cap;
    if (!c->pipe) c->pipe = new PipeState();
    PipeState& P = *c->pipe;
    if (!P.tstream) {
        int lo = 0, hi = 0;
        CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        CK(cudaStreamCreateWithPriority(&P.tstream, cudaStreamNonBlocking, hi));
        CK(cudaStreamCreateWithPriority(&P.pstream, cudaStreamNonBlocking, lo));
        CK(cudaEventCreateWithFlags(&P.kern_ev, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&P.sync_ev, cudaEventDisableTiming));
    }
    const size_t R = B.rq_cap;
    P.ring.ensure(kQueueCap);
    P.ctl.ensure(2);
    P.done.ensure(R);
    P.rec.ensure(R);
    P.h_traj.ensure(R * (size_t)cap * 3);
    P.h_slot.ensure(R);
    P.h_obs.ensure(R * (size_t)cap);
    P.obs.ensure(R * (size_t)cap);
    P.tpos.ensure(R * (size_t)cap);
    P.pub_seq.ensure(1);
    P.st_s.ensure(R * (size_t)cap * 3);
    P.st_df.ensure(R * (size_t)cap * 6);
    P.st_h.ensure(R * (size_t)cap);
    P.ties.ensure(R * (size_t)cap);
    P.head.ensure(1);
    P.sep.ensure(R);
    P.req_ord.ensure(R);
    P.list.ensure((size_t)kRepSlots * kBatchMax);
    P.nlist.ensure(kRepSlots);
    P.h_list.ensure((size_t)kRepSlots * (kBatchMax + 1));
    for (cudaEvent_t& e : P.rep_ev)
        if (!e) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    if (!P.ord_init || P.ord_base + n >= kOrdLimit) {  // every stored plan counts as earlier
        P.slot_ord.ensure(c->S_pad);
        CK(cudaMemsetAsync(P.slot_ord.p, 0x80, (size_t)c->S_pad * sizeof(int32_t), c->stream));  // INT_MIN-ish
        P.ord_base = 0;
        P.ord_init = true;
    }
    const int32_t ord0 = P.ord_base;
    P.ord_base += n;

    // streams: the call's table operations go to the table stream (c->stream is swapped for
    // the call), after the work already on the caller's stream
    cudaStream_t user = c->stream;
    CK(cudaEventRecord(P.sync_ev, user));
    CK(cudaStreamWaitEvent(P.tstream, P.sync_ev, 0));
    CK(cudaStreamWaitEvent(P.pstream, P.sync_ev, 0));
    c->stream = P.tstream;
    const int32_t saved_limit = c->extra_limit;
    c->extra_limit = INT32_MAX;  // rows are rebuilt only by the pipeline's own drains

    // per-request state
    std::vector<uint8_t> phase(n, serve ? kAbsent : kWait);  // a batch's requests are all there
    std::vector<int32_t> chk(n, 0), gate(n, 0), tok(n, 0), slot_of(n, -1), verdict(n, -1), replans(n, 0),
        tail_obs(n, 0), start(n, 0), cur(n, -1), contrib_tok(n, 0);
    std::vector<uint64_t> ids(n, 0);
    std::vector<RolloutOut> fin_ro(n);
    std::vector<TrajBoxes> boxes(n);
    std::vector<double> t_disp(n, 0.0), done_at(n, -1.0);
    std::vector<Version> V;
    std::vector<Change> E;      // contribution changes, in table-operation order
    size_t e_done = 0;          // E[0 .. e_done) have completed all their operations
    int32_t ops = 0;            // table operations enqueued (numbered 1 .. ops)
    int32_t ops_done = 0;       // ... and known complete
    struct OpEv {
        int32_t q;
        cudaEvent_t ev;
    };
    std::vector<OpEv> op_ev;    // completion events of enqueued operations, in order
    size_t op_head = 0;
    std::vector<int32_t> inflight;
    std::vector<int32_t> xcnt(c->T_win, 0);
    int32_t xmax = 0;
    // rows rebuilt before any of them could fill up: the appends since the rows were last
    // measured (acnt) reaching room[row] start a drain
    const int32_t margin = append_margin(window, n);
    const int32_t rebuild_mark = c->opt.pipe_rebuild_items > 0 ? c->opt.pipe_rebuild_items : kPipeExtraLimit;
    std::vector<int32_t> room(c->T_win, 0), acnt(c->T_win, 0);
    bool overfull = false;
    auto measure_rows = [&]() {
        const std::vector<int32_t> fill = row_fill(c);
        for (int32_t r = 0; r < c->T_win; ++r) {
            room[r] = c->S_pad - margin - fill[r];
            require(room[r] >= 1, FMDP_ERR_FULL, "an index row has no room left for pipelined batching");
        }
        std::fill(acnt.begin(), acnt.end(), 0);
        overfull = false;
    };
    bool draining = false;
    int32_t dispatch_gate = 0;  // after a drain: operations that must be complete first
    bool tentative_used = false;
    std::vector<int32_t> unreported;
    for (int32_t k = 0; k < n; ++k) P.done.p[k] = 0;
    // ordinals of the call's requests, for the exact separation report
    {
        std::vector<int32_t> ho(n);
        for (int32_t k = 0; k < n; ++k) ho[k] = ord0 + k;
        CK(cudaMemcpyAsync(P.req_ord.p, ho.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, P.tstream));
        CK(cudaStreamSynchronize(P.tstream));
    }

    InflRule rule{};
    rule.dt = c->model.dt;
    rule.H = c->sep.horiz_m + 1.0;
    rule.V = c->sep.vert_m + 1.0;
    rule.dzmax = climb_step(c);
    rule.n_wells = c->model.n_wells;
    for (int w = 0; w < rule.n_wells; ++w) {
        rule.tau[w] = c->model.w_tau64[w];
        rule.R[w] = c->model.w_R64[w];
    }

    // launch shape: the widest indexed shape (384 threads, unless the options set one). The
    // persistent launch holds at most one CTA per SM, where more scanner warps give the
    // shortest step; the autotuner's shapes are chosen for waves of full rollouts side by
    // side, two CTAs per SM when a wave holds more rollouts than there are SMs. Persistent
    // CTAs leave room on a few SMs for the table stream's kernels
    Geometry g = geometry_indexed(c, c->S_pad, 0);
    const int resident = rollout_max_active_clusters(1, g.threads, g.smem);
    require(resident >= 1, FMDP_ERR_ARG, "the rollout shape does not fit an SM");
    const int per_sm = std::max(1, resident / std::max(1, c->n_sm));
    const int reserve = per_sm * std::max(4, c->n_sm / 16);
    // persistent CTAs: serving, at most two thirds of the SM count (its reports and expiry
    // clearing run beside the launch and must find room, or every table operation behind them
    // waits until the launch idles out); a batch call, at most the SM count (it reports at its
    // end). Measured on 152 SMs: serving C4 with 100 CTAs held 32k req/s at p99 11 ms where
    // 144 fell to 7.6k/s and 256 to 4.5k/s; batches: C2 0.101 / 0.103 / 0.110 s per call with
    // 100 / 144 / 256 CTAs, the 20k-plan batch of 512 27.2k / 26.3k / 26.0k plans/s with
    // 100 / 152 / 256, the 100k-plan batch of 512 23.6k / 26.0k / 27.1k
    const int cta_cap = serve ? c->n_sm * 2 / 3 : c->n_sm;
    const int n_ctas = std::max(1, std::min(std::min(resident - reserve, window), cta_cap));

    RolloutArgs ra{};
    ra.m = c->model;
    ra.S_scan = g.S_scan;
    ra.chunk = g.chunk;
    ra.cs = 1;
    ra.ring = g.ring;
    ra.cap = cap;
    ra.reqs = B.rq;
    ra.n_req = n;
    ra.traj = B.traj.p;
    ra.acts = B.acts.p;
    ra.out = B.rout.p;
    ra.err = c->err;
    ra.pipe.on = 1;
    ra.pipe.qmask = kQueueCap - 1;
    ra.pipe.items = P.ring.d;
    ra.pipe.tail = P.ctl.d;
    ra.pipe.stop = P.ctl.d + 1;
    ra.pipe.head = P.head.p;
    ra.pipe.done = P.done.d;
    ra.pipe.rec = P.rec.d;
    ra.pipe.h_traj = P.h_traj.d;
    ra.pipe.sep = P.sep.p;
    ra.pipe.idle_cycles = 1ll << 31;  // about a second without work
    ra.pipe.pub_seq = P.pub_seq.p;
    ra.pipe.obs = P.obs.p;
    ra.pipe.h_obs = P.h_obs.d;
    ra.pipe.st_s = P.st_s.p;
    ra.pipe.st_df = P.st_df.p;
    ra.pipe.st_h = P.st_h.p;
    ra.pipe.ties = P.ties.p;
    ra.pipe.ord0 = ord0;
    CK(cudaMemsetAsync(P.pub_seq.p, 0, sizeof(int32_t), P.tstream));
    int32_t tail = 0;
    P.ctl.p[0] = 0;
    P.ctl.p[1] = 0;
    CK(cudaMemsetAsync(P.head.p, 0, sizeof(int32_t), P.pstream));
    bool launched = false;
    auto launch = [&]() {
        ra.tab = table_view(c);
        set_index_args(c, ra, g);
        std::atomic_thread_fence(std::memory_order_seq_cst);
        cudaEvent_t ka = nullptr;
        if (c->profiling) {  // the persistent launch's duration (kernel kind 0: rollout)
            ka = next_event(c);
            CK(cudaEventRecord(ka, P.pstream));
        }
        LAUNCH(c, launch_rollout(ra, g.threads, g.smem, P.pstream, n_ctas));
        CK(cudaEventRecord(P.kern_ev, P.pstream));
        if (ka) {
            cudaEvent_t kb = next_event(c);
            CK(cudaEventRecord(kb, P.pstream));
            c->pending.push_back({0, ka, kb});
        }
        launched = true;
    };
    auto kernel_running = [&]() {
        if (!launched) return false;
        const cudaError_t e = cudaEventQuery(P.kern_ev);
        if (e == cudaErrorNotReady) return true;
        CK(e);
        return false;
    };
    auto stop_kernel = [&]() {  // every CTA leaves once the ring is empty
        if (!launched) return;
        std::atomic_thread_fence(std::memory_order_seq_cst);
        *reinterpret_cast<volatile int32_t*>(P.ctl.p + 1) = 1;
        CK(cudaEventSynchronize(P.kern_ev));
        launched = false;
        *reinterpret_cast<volatile int32_t*>(P.ctl.p + 1) = 0;
    };

    const auto t0 = clk::now();
    auto elapsed = [&]() { return std::chrono::duration<double>(clk::now() - t0).count(); };
    double cta_time = 0.0, last_progress = 0.0;
    int64_t n_dispatch = 0, n_replans = 0, n_drains = 0, steps_sum = 0, n_resumes = 0, n_rechecks = 0;
    int64_t n_publish = 0, n_withdraw = 0;
    int32_t head = 0, joined = serve ? 0 : n, finalized = 0, admitted = 0, max_seen = 0;
    // how each head of line waited (statistics): its phase and re-plans when it became head
    int32_t head_mark = -1, head_replans = 0;
    uint8_t head_phase = kAbsent;
    double head_since = 0.0;
    int64_t expiries = 0, expired = 0;
    int32_t deferred = 0;
    std::vector<uint8_t> deferred_flag(serve ? n : 0, 0);
    std::vector<int64_t> dep_suffix;
    int64_t sim0 = 0, quantum = 60;
    double scale = 1.0;
    int32_t max_active = c->S_max;
    if (serve) {
        dep_suffix.assign(n + 1, INT64_MAX);
        for (int32_t i = n - 1; i >= 0; --i) dep_suffix[i] = std::min(dep_suffix[i + 1], reqs[i].depart_step);
        sim0 = serve->o.sim_start_set ? serve->o.sim_start_step : c->book.t_base;
        quantum = serve->o.expire_quantum > 0 ? serve->o.expire_quantum : 60;
        scale = serve->o.time_scale > 0.0 ? serve->o.time_scale : 1.0;
        max_active = serve->o.max_active_plans > 0 ? std::min(serve->o.max_active_plans, c->S_max) : c->S_max;
    }

    // the exact separation report (row-major check with the ordinal filter) of the listed
    // requests, on the table stream, into B.sepo: the rows their trajectories reach only, and
    // without waiting (a staging slot is reused once the report that last used it is done)
    auto report = [&](std::vector<int32_t>& L) {
        const NvtxRange range("fmdp separation report");
        for (size_t o = 0; o < L.size(); o += kBatchMax) {
            const int32_t m = (int32_t)std::min<size_t>(kBatchMax, L.size() - o);
            const int q = P.rep_next;
            P.rep_next = (P.rep_next + 1) % kRepSlots;
            if (P.rep_used[q]) CK(cudaEventSynchronize(P.rep_ev[q]));
            int32_t* hl = P.h_list.p + (size_t)q * (kBatchMax + 1);
            int32_t* dl = P.list.p + (size_t)q * kBatchMax;
            int32_t* dn = P.nlist.p + q;
            std::copy(L.begin() + o, L.begin() + o + m, hl);
            hl[kBatchMax] = m;
            int64_t t_lo = INT64_MAX, t_hi = INT64_MIN;
            for (int32_t i = 0; i < m; ++i) {
                const int32_t k = L[o + i];
                t_lo = std::min<int64_t>(t_lo, reqs[k].depart_step);
                t_hi = std::max<int64_t>(t_hi, reqs[k].depart_step + fin_ro[k].n_points);
            }
            const int64_t w0 = c->book.t_base, w1 = c->book.t_base + c->T_win;
            t_lo = std::max(t_lo, w0);
            t_hi = std::min(t_hi, w1);
            CK(cudaMemcpyAsync(dl, hl, m * sizeof(int32_t), cudaMemcpyHostToDevice, P.tstream));
            CK(cudaMemcpyAsync(dn, hl + kBatchMax, sizeof(int32_t), cudaMemcpyHostToDevice, P.tstream));
            LAUNCH(c, launch_sep_reset_idx(B.sepo.p, dl, dn, m, P.tstream));
            SepRowsArgs sp{};
            sp.m = c->model;
            sp.tab = table_view(c);
            sp.S_scan = c->S_pad;
            sp.traj = B.traj.p;
            sp.cap = cap;
            sp.rout = B.rout.p;
            sp.reqs = B.rq;
            sp.idx = dl;
            sp.n_dev = dn;
            sp.n_max = m;
            sp.out = B.sepo.p;
            sp.items = c->ix_items;
            sp.cstart = c->ix_cstart;
            sp.nextra = c->ix_nextra;
            sp.ncell = c->ix_ncell;
            sp.slot_ord = P.slot_ord.p;
            sp.req_ord = P.req_ord.p;
            if (t_hi > t_lo) {
                sp.row0 = (int32_t)(t_lo - w0);
                sp.nrows = (int32_t)(t_hi - t_lo);
                KernelTimer t(c, 1, P.tstream);
                LAUNCH(c, launch_sepcheck_rows(sp, P.tstream));
                t.stop();
            }
            CK(cudaEventRecord(P.rep_ev[q], P.tstream));
            P.rep_used[q] = true;
            for (int32_t i = 0; i < m; ++i) c->stats.sep_pairs += (int64_t)fin_ro[L[o + i]].n_points * c->S_pad;
        }
        L.clear();
    };
    // a table operation was just enqueued: number it, raise the device counter after it, and
    // keep an event to learn when it is complete
    auto close_op = [&]() {
        ++ops;
        LAUNCH(c, launch_store_release(P.pub_seq.p, ops, P.tstream));
        cudaEvent_t ev;
        if (P.ev_free.empty()) {
            CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        } else {
            ev = P.ev_free.back();
            P.ev_free.pop_back();
        }
        CK(cudaEventRecord(ev, P.tstream));
        op_ev.push_back({ops, ev});
        return ops;
    };
    auto count_rows = [&](int32_t k, int32_t first, int32_t np) {  // rows that items [first, np) went to
        const int64_t d = reqs[k].depart_step;
        for (int32_t i = first; i < np; ++i) {
            const int64_t T = d + i;
            if (T < c->book.t_base || T >= c->book.t_base + c->T_win) continue;
            int64_t row = T % c->T_win;
            if (row < 0) row += c->T_win;
            xmax = std::max(xmax, ++xcnt[row]);
            if (++acnt[row] >= room[row]) overfull = true;
        }
    };
    // appends request k's latest plan (as planned on the device) to the index as its
    // tentative plan and publishes it
    auto append_tentative = [&](int32_t k, int32_t np, int32_t first) {
        IndexAppendArgs ia{};
        ia.ix = index_args(c);
        ia.tentative = 1;
        ia.first = first;
        ia.tent_ord = ord0 + k;
        ia.tpos = P.tpos.p + (size_t)k * cap;
        ia.traj = B.traj.p + (size_t)k * cap * 3;
        ia.cap = cap;
        ia.rout = B.rout.p + k;
        ia.reqs = B.rq + k;
        ia.sep = P.sep.p + k;
        LAUNCH(c, launch_index_append(ia, 1, np, P.tstream));
        LAUNCH(c, launch_index_publish(ia.ix, P.tstream));
        count_rows(k, first, np);
        tentative_used = true;
    };
    // request k's contribution becomes its latest plan (published when admissible) or nothing.
    // A plan resumed from a later step keeps its first samples: the items of those (sample i
    // and sample i + 1 each) stay in the index as they are, so that no read ever misses them,
    // and only the items past them are withdrawn and appended.
    auto set_contribution = [&](int32_t k) {
        const int32_t v_old = cur[k];
        const bool admissible = verdict[k] == FMDP_ADMITTED;
        const int32_t n_new = admissible ? fin_ro[k].n_points : 0;
        const float* xyz = P.h_traj.p + (size_t)k * cap * 3;
        int32_t keep = 0;  // items kept
        if (v_old >= 0 && admissible) {
            const Version& a = V[v_old];
            const int32_t m = std::min(a.n, n_new);
            int32_t same = 0;  // samples equal in both
            while (same < m && a.xyz[3 * same] == xyz[3 * same] && a.xyz[3 * same + 1] == xyz[3 * same + 1] &&
                   a.xyz[3 * same + 2] == xyz[3 * same + 2])
                ++same;
            keep = std::max(same - 1, 0);
        }
        int32_t v_new = -1;
        if (v_old >= 0) {
            const Version& x = V[v_old];
            LAUNCH(c, launch_index_withdraw(index_args(c), P.tpos.p + (size_t)k * cap + keep,
                                            reqs[k].depart_step + keep, x.n - keep, P.tstream));
            V[v_old].q_kill = close_op();
            ++n_withdraw;
        }
        if (admissible) {
            Version x;
            x.j = k;
            x.n = n_new;
            x.xyz.assign(xyz, xyz + 3 * (size_t)n_new);
            x.boxes = boxes[k];
            append_tentative(k, n_new, keep);
            x.q_pub = close_op();
            x.q_kill = INT32_MAX;
            x.q_from = keep > 0 ? V[v_old].q_from : x.q_pub;
            v_new = (int32_t)V.size();
            V.push_back(std::move(x));
            ++n_publish;
        }
        cur[k] = v_new;
        contrib_tok[k] = tok[k];
        if (v_old >= 0 || v_new >= 0) E.push_back({k, v_old, v_new, ops, keep});
    };
    // stores an admitted request: scatter into the plan table on the table stream (its index
    // items are its tentative plan's, already published)
    auto admit = [&](int32_t k) {
        const int32_t slot = take_slot(c);
        const uint64_t id = c->book.next_id++;
        c->book.add(id, PlanMeta{slot, reqs[k].depart_step, fin_ro[k].n_points});
        c->book.S_hw = std::max(c->book.S_hw, slot + 1);
        slot_of[k] = slot;
        ids[k] = id;
        P.h_slot.p[k] = slot;
        std::atomic_thread_fence(std::memory_order_seq_cst);
        AdmitArgs aa{};
        aa.err = c->err;
        aa.tab = table_view(c);
        aa.cap = cap;
        aa.traj = B.traj.p + (size_t)k * cap * 3;
        aa.rout = B.rout.p + k;
        aa.reqs = B.rq + k;
        aa.slots = P.h_slot.d + k;
        aa.sep = P.sep.p + k;
        aa.force = 0;
        aa.slot_ord = P.slot_ord.p;
        aa.ord = ord0 + k;
        KernelTimer t(c, 2, P.tstream);
        LAUNCH(c, launch_admit(aa, 1, fin_ro[k].n_points, P.tstream));
        t.stop();
        ++admitted;
    };
    // brings request k's completed plan up to date with the contribution changes of earlier
    // requests; false (and k waits for a new plan) when one of them influences it. The new
    // plan keeps the steps before the first one any of them could change, and only the
    // conflict check runs again when none changes a step but one may change the verdict.
    auto check_plan = [&](int32_t k) {
        const int32_t nk = fin_ro[k].n_points;
        const float* pk = P.h_traj.p + (size_t)k * cap * 3;
        const int32_t* ok = P.h_obs.p + (size_t)k * cap;
        int first = INT32_MAX;
        bool sep_any = false;
        for (; chk[k] < (int32_t)E.size(); ++chk[k]) {
            const Change& ch = E[chk[k]];
            if (ch.j >= k) continue;  // later requests are not part of k's table
            const int64_t tj = reqs[ch.j].depart_step;
            bool sep = false;
            auto test = [&](const Version& x, int32_t q_lo, int32_t q_hi, int32_t floor_) {
                const int f = first_influenced(rule, x.xyz.data(), x.n, tj, x.boxes, q_lo, q_hi, pk, nk,
                                               reqs[k].depart_step, reqs[k].speed_mps, boxes[k], ok, tail_obs[k], &sep,
                                               floor_);
                if (f >= 0) first = std::min(first, f);
                sep_any = sep_any || sep;
            };
            // only the items past the kept ones changed: the withdrawn ones where a read could
            // still see them (from the first append of the chain of versions they belong to),
            // the appended ones where a read could still miss them
            if (ch.v_old >= 0) test(V[ch.v_old], V[ch.v_old].q_from, V[ch.v_old].q_kill, ch.keep);
            if (ch.v_new >= 0) test(V[ch.v_new], INT32_MIN, V[ch.v_new].q_pub, ch.keep);
        }
        if (first == INT32_MAX && !sep_any) return true;
        phase[k] = kWait;
        gate[k] = ops;  // every operation so far visible to the next plan
        start[k] = first == INT32_MAX ? -1 : first;
        ++replans[k];
        ++n_replans;
        if (start[k] > 0) ++n_resumes;
        if (start[k] < 0) ++n_rechecks;
        return false;
    };
    auto dispatch = [&](int32_t k) {
        tok[k] += 1;
        // a plan from the origin reads every completed change; a resumed plan's kept steps
        // were checked up to chk[k] and keep their observations
        if (start[k] == 0) chk[k] = (int32_t)e_done;
        PipeItem& it = P.ring.p[tail & (kQueueCap - 1)];
        it.r = k;
        it.token = tok[k];
        it.start = start[k];
        it.pad = 0;
        it.t_base = c->book.t_base;
        start[k] = 0;
        std::atomic_thread_fence(std::memory_order_release);
        *reinterpret_cast<volatile int32_t*>(P.ctl.p) = ++tail;
        inflight.push_back(k);
        phase[k] = kFlight;
        t_disp[k] = elapsed();
        ++n_dispatch;
    };

    measure_rows();
    size_t e_seen = SIZE_MAX;
    int32_t head_seen = -1;
    try {
        launch();
        while (finalized < n) {
            const double now = elapsed();
            bool progress = false;
            // table operations that are complete, and the changes they close
            while (op_head < op_ev.size()) {
                const cudaError_t e = cudaEventQuery(op_ev[op_head].ev);
                if (e == cudaErrorNotReady) break;
                CK(e);
                ops_done = op_ev[op_head].q;
                P.ev_free.push_back(op_ev[op_head].ev);
                ++op_head;
                progress = true;
            }
            while (e_done < E.size() && E[e_done].q_last <= ops_done) ++e_done;
            // finished plans
            for (size_t q = 0; q < inflight.size();) {
                const int32_t k = inflight[q];
                if (*reinterpret_cast<volatile int32_t*>(P.done.p + k) != tok[k]) {
                    ++q;
                    continue;
                }
                std::atomic_thread_fence(std::memory_order_acquire);
                inflight[q] = inflight.back();
                inflight.pop_back();
                const PipeRecord rc = P.rec.p[k];
                fin_ro[k] = rc.ro;
                steps_sum += rc.ro.steps;
                c->stats.slots_scanned += (int64_t)rc.ro.steps * g.S_scan;
                cta_time += now - t_disp[k];
                verdict[k] = rc.ro.status != kStatusCaptured ? rc.ro.status
                             : rc.first_conflict >= 0       ? FMDP_REJ_CONFLICT
                             : rc.first_terrain >= 0        ? FMDP_REJ_TERRAIN
                                                            : FMDP_ADMITTED;
                boxes[k].build(P.h_traj.p + (size_t)k * cap * 3, rc.ro.n_points, c->model.dt,
                               P.h_obs.p + (size_t)k * cap);
                tail_obs[k] = rc.tail_pub;
                phase[k] = kDone;
                progress = true;
            }
            // plans near the head: up to date with every change, published when they are new
            // (only when a change was logged, a plan finished or the head moved since the last
            // pass: otherwise nothing here can differ)
            if (progress || E.size() != e_seen || head != head_seen) {
                const int32_t lim = std::min(joined, head + window);
                for (int32_t k = head; k < lim; ++k) {
                    if (phase[k] != kDone) continue;
                    if (chk[k] < (int32_t)E.size() && !check_plan(k)) continue;
                    if (k < head + kPublishAhead && contrib_tok[k] != tok[k]) set_contribution(k);
                }
                e_seen = E.size();
                head_seen = head;
            }
            if (head < joined && head_mark != head) {  // a new head of line: how it waits
                head_mark = head;
                head_since = now;
                head_phase = phase[head];
                head_replans = replans[head];
            }
            // the walk: a head whose plan is up to date is final
            while (head < joined && phase[head] == kDone && check_plan(head)) {
                const int32_t k = head;
                if (contrib_tok[k] != tok[k]) set_contribution(k);
                if (verdict[k] == FMDP_ADMITTED) admit(k);
                phase[k] = kFinal;
                done_at[k] = elapsed();
                unreported.push_back(k);
                if (head_mark == k) {
                    const bool again = replans[k] > head_replans;
                    const int cls = head_phase == kWait ? 4 : head_phase == kFlight ? (again ? 2 : 1) : (again ? 3 : 0);
                    ++c->stats.pipe_head_n[cls];
                    c->stats.pipe_head_s[cls] += done_at[k] - head_since;
                }
                ++head;
                ++finalized;
                progress = true;
                if (head < joined) {
                    head_mark = head;
                    head_since = done_at[k];
                    head_phase = phase[head];
                    head_replans = replans[head];
                }
                // the request that joins the published range
                const int32_t q = head + kPublishAhead - 1;
                if (q < joined && phase[q] == kDone && check_plan(q) && contrib_tok[q] != tok[q]) set_contribution(q);
            }
            // serving: reports as requests finish, so that an expiry (which must report the
            // finished requests before it clears their rows) finds few waiting. A batch call
            // reports at its end: a report kernel beside a busy persistent launch could hold
            // up the table stream behind it until the launch idled out
            if (serve && unreported.size() >= (size_t)kRepChunk) report(unreported);
            if (progress) last_progress = now;
            if (finalized >= n) break;

            // serving: expiry (a drain: the persistent launch holds the window's first step)
            bool want_expiry = false;
            int64_t limit = INT64_MIN;
            if (serve) {
                limit = sim0 + (int64_t)std::floor(now * scale / c->air.dt);
                limit = std::min(limit, dep_suffix[joined]);
                for (int32_t k = head; k < joined; ++k) limit = std::min(limit, reqs[k].depart_step);
                want_expiry = limit >= c->book.t_base + quantum;
            }
            // an expiry moves the window's first step without stopping the launch: a plan in
            // flight keeps the window its item was dispatched with, and none of them reads the
            // rows the expiry clears (every unresolved request departs at or after the new
            // first step); the clearing is a table operation that later dispatches wait for
            if (want_expiry && !draining) {
                report(unreported);  // before the rows of finished requests can be cleared
                {
                    cudaStream_t own = c->stream;
                    c->stream = P.tstream;  // in order with the other table operations
                    try {
                        expire_to(c, limit, &expired, false);
                    } catch (...) {
                        c->stream = own;
                        throw;
                    }
                    c->stream = own;
                }
                close_op();
                dispatch_gate = ops;
                ++expiries;
                // (the rows' room stays as measured: clearing rows only lowers their fill)
            }
            if (!draining && (xmax > rebuild_mark || overfull)) draining = true;
            if (draining && inflight.empty()) {
                stop_kernel();  // the idle CTAs give their SMs to the rebuild
                if (xmax > rebuild_mark || overfull) {  // rows whose extra lists grew long: rebuilt now
                    const NvtxRange range("fmdp drain: index rows rebuilt");
                    CK(cudaStreamSynchronize(P.tstream));  // no report still reads the rows
                    index_rebuild_all(c);
                    std::fill(xcnt.begin(), xcnt.end(), 0);
                    xmax = 0;
                    measure_rows();
                    ++n_drains;
                    // the rebuild keeps only stored plans. A tentative plan that is still its
                    // request's latest plan goes back in (the same version: visible to every
                    // read after the drain as before it); one whose request has planned again
                    // since (the device holds the newer plan) is withdrawn
                    const int32_t q_rebuild = close_op();
                    for (int32_t k = head; k < joined; ++k) {
                        if (cur[k] < 0) continue;
                        if (contrib_tok[k] == tok[k]) {  // (nothing is in flight: the device holds it)
                            append_tentative(k, V[cur[k]].n, 0);
                            close_op();
                        } else {
                            V[cur[k]].q_kill = q_rebuild;
                            E.push_back({k, cur[k], -1, q_rebuild, 0});
                            cur[k] = -1;
                            contrib_tok[k] = -1;
                            ++n_withdraw;
                        }
                    }
                }
                dispatch_gate = ops;
                draining = false;
            }
            // serving: arrivals join while the set has room and the table has slots for all
            if (serve) {
                while (joined < n && serve->arrival_s[joined] <= now && joined - head < window) {
                    const int64_t active = (int64_t)c->book.size();
                    const int64_t room = std::min<int64_t>((int64_t)c->book.free_slots.size(), max_active - active);
                    if ((int64_t)(joined - head) + 1 > room) {
                        if (!deferred_flag[joined]) {
                            deferred_flag[joined] = 1;
                            ++deferred;
                        }
                        break;
                    }
                    phase[joined] = kWait;
                    ++joined;
                }
                max_seen = std::max(max_seen, joined - head);
            }
            // dispatch the waiting requests nearest the head, the changes they wait for visible
            if (!draining && ops_done >= dispatch_gate) {
                const int32_t end = std::min(joined, head + window);
                for (int32_t k = head; k < end && (int32_t)inflight.size() < n_ctas; ++k)
                    if (phase[k] == kWait && gate[k] <= ops_done) dispatch(k);
            }
            if (!inflight.empty() && !kernel_running()) {
                require(read_error_word(c) == 0, FMDP_ERR_TIMEOUT, "a bounded device wait expired during a rollout");
                launch();  // the launch left while idle; the ring keeps its position
            }
            if (serve && inflight.empty() && head == joined && joined < n) {
                if (deferred_flag[joined]) {  // nothing unresolved and no room: only expiry frees slots
                    int64_t first_end = INT64_MAX;
                    c->book.for_each([&](uint64_t, const PlanMeta& p) { first_end = std::min(first_end, p.t0 + p.n); });
                    require(first_end <= dep_suffix[joined], FMDP_ERR_FULL, "plan table full and no plan can expire");
                    std::this_thread::sleep_for(std::chrono::microseconds(200));
                } else {
                    const double wait = serve->arrival_s[joined] - elapsed();
                    if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(std::min(wait, 0.002)));
                }
                last_progress = elapsed();
            }
            require(elapsed() - last_progress < 30.0, FMDP_ERR_TIMEOUT, "pipelined FCFS made no progress for 30 s");
        }
        stop_kernel();
        // the index again holds only stored plans (tentative and withdrawn items go), then
        // the exact separation reports
        CK(cudaStreamSynchronize(P.tstream));  // no report still reads the rows
        if (tentative_used) index_rebuild_all(c);
        report(unreported);
        CK(cudaStreamSynchronize(P.tstream));
        require(read_error_word(c) == 0, FMDP_ERR_TIMEOUT, "a bounded device wait expired during a rollout");
    } catch (...) {
        // leave nothing running: stop the launch (it drains the ring), wait for the streams,
        // and rebuild the index from the stored plans
        if (launched) {
            *reinterpret_cast<volatile int32_t*>(P.ctl.p + 1) = 1;
            cudaEventSynchronize(P.kern_ev);
            *reinterpret_cast<volatile int32_t*>(P.ctl.p + 1) = 0;
        }
        cudaStreamSynchronize(P.tstream);
        if (tentative_used) {
            try {
                index_rebuild_all(c);
                cudaStreamSynchronize(P.tstream);
            } catch (...) {
            }
        }
        for (size_t q = op_head; q < op_ev.size(); ++q) P.ev_free.push_back(op_ev[q].ev);
        c->extra_limit = saved_limit;
        c->stream = user;
        throw;
    }
    for (size_t q = op_head; q < op_ev.size(); ++q) P.ev_free.push_back(op_ev[q].ev);
    c->extra_limit = saved_limit;
    c->stream = user;
    CK(cudaEventRecord(P.sync_ev, P.tstream));
    CK(cudaStreamWaitEvent(user, P.sync_ev, 0));
    if (c->profiling) collect_timers(c);

    // results: verdict from the tail check, separation report from the exact pass
    CK(cudaMemcpyAsync(B.h_sep.p, B.sepo.p, n * sizeof(SepOut), cudaMemcpyDeviceToHost, user));
    CK(cudaStreamSynchronize(user));
    for (int32_t k = 0; k < n; ++k) {
        SepOut so = B.h_sep.p[k];
        const int32_t fc = so.first_conflict == INT_MAX ? -1 : so.first_conflict;
        const int32_t ft = so.first_terrain == INT_MAX ? -1 : so.first_terrain;
        require(fc == P.rec.p[k].first_conflict && ft == P.rec.p[k].first_terrain, FMDP_ERR_CUDA,
                "internal: the exact separation report disagrees with the rollout's conflict check");
        so.verdict = verdict[k];
        fill_result(fin_ro[k], so, res + k);
        res[k].plan_id = ids[k];
        res[k].replanned = replans[k];
    }
    c->call_ms.assign(n, 0.0);
    for (int32_t k = 0; k < n; ++k) c->call_ms[k] = 1e3 * done_at[k];
    c->stats.batch_rollouts += n_dispatch;
    c->stats.batch_replans += n_replans;
    c->stats.rollout_steps += steps_sum;
    c->stats.pipe_drains += n_drains;
    c->stats.pipe_resumes += n_resumes;
    c->stats.pipe_rechecks += n_rechecks;
    c->stats.pipe_publishes += n_publish;
    c->stats.pipe_withdrawals += n_withdraw;
    const double wall = elapsed();
    c->stats.pipe_cta_s += cta_time;
    c->stats.pipe_slot_s += wall * n_ctas;
    c->stats.pipe_ctas = n_ctas;
    c->stats.pipe_resident = resident;
    if (!keep_points) copy_points_back(c, n, res);
    if (serve) {
        std::vector<double> lat(n);
        double mx = 0.0, sum = 0.0, last = 0.0;
        for (int32_t i = 0; i < n; ++i) {
            lat[i] = 1e3 * std::max(0.0, done_at[i] - serve->arrival_s[i]);
            if (serve->latency_ms) serve->latency_ms[i] = lat[i];
            mx = std::max(mx, lat[i]);
            sum += lat[i];
            last = std::max(last, done_at[i]);
        }
        if (serve->rep) {
            std::vector<double> sorted = lat;
            std::sort(sorted.begin(), sorted.end());
            auto pct = [&](double q) {
                const size_t i = (size_t)std::min<double>((double)sorted.size() - 1, std::ceil(q * sorted.size()) - 1);
                return sorted[i];
            };
            fmdp_serve_report& r = *serve->rep;
            r = fmdp_serve_report{};
            r.wall_s = last;
            r.throughput_rps = last > 0.0 ? n / last : 0.0;
            r.latency_p50_ms = pct(0.50);
            r.latency_p99_ms = pct(0.99);
            r.latency_mean_ms = sum / n;
            r.latency_max_ms = mx;
            r.waves = 0;
            r.rollouts = n_dispatch;
            r.replans = n_replans;
            r.expiries = expiries;
            r.plans_expired = expired;
            r.final_t_base = c->book.t_base;
            r.admitted = admitted;
            r.rejected = n - admitted;
            r.max_in_flight_seen = max_seen;
            r.deferred_for_memory = deferred;
            r.pipelined = 1;
            r.drains = n_drains;
            r.rollout_occupancy = wall > 0.0 ? cta_time / (wall * n_ctas) : 0.0;
            r.persistent_ctas = n_ctas;
        }
    }
    return admitted;
}

}  // namespace fmdp
