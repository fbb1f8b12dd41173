// Speculative batches: waves of concurrent rollouts, the influence test and the
// arrival-order walk; departure-time candidates; the launch-shape autotuner.
#include "speculator.cuh"

namespace fmdp {

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

// kernels of one wave: admit, reset, rollout, sep_check, influence (+ index append, rebuild)
int wave_kernels(const fmdp_ctx* c) { return (c->index_on ? 8 : 5) + (c->learned_mode ? 4 : 0); }

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
        index_append_admitted(c, B.traj.p, cap, B.rout.p, B.rq, B.sepo.p, slots, store, B.ctr.p + 3, n_cap,
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
    for (int32_t i = 0, s = -1; i < n_new; ++i) {
        s = c->book.free_slots.next(s + 1);
        bound = std::max(bound, s + 1);
    }
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
    const NvtxRange range("fmdp batch FCFS");
    if (pipeline_eligible(c) && pipeline_fits(c, n, nullptr))
        return run_pipeline(c, reqs, n, res, dev_reqs, keep_points, nullptr);
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
    c->call_ms.assign(n, 0.0);
    const auto t_start = std::chrono::steady_clock::now();
    for (int32_t b0 = 0; b0 < n; b0 += bs) {
        const int32_t m = std::min(bs, n - b0);
        sp.set_geometry(batch_geometry(c, m, m));
        for (int32_t i = 0; i < m; ++i) sp.add(b0 + i);
        sp.adm_all.clear();
        try {
            while (!sp.U.empty()) {
                const size_t before = resolved.size();
                sp.wave(resolved);
                const double t =
                    std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
                for (size_t q = before; q < resolved.size(); ++q) c->call_ms[resolved[q]] = t;
            }
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
                index_append_admitted(c, aa.traj, B.cap, aa.rout, aa.reqs, aa.sep, aa.slots, nullptr, nullptr, 1, d0,
                                      d0 + cand[pick].horizon + 1);
                CK(cudaStreamSynchronize(c->stream));
            } catch (...) {
                c->book.free_slots.insert(slot);
                throw;
            }
            id = c->book.next_id++;
            c->book.add(id, PlanMeta{slot, cand[pick].depart_step, B.h_rout.p[pick].n_points});
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

}  // namespace fmdp
