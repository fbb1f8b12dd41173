// Host runtime of libfmdp: model constants, the device plan table and its spatial index,
// launch geometry, slot allocation, the sliding time window, and the FCFS sequence
// enqueue shared by the sequential paths.
#include "host.cuh"

namespace fmdp {

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


IndexArgs index_args(fmdp_ctx* c) {
    IndexArgs a{};
    a.tab = table_view(c);
    a.cstart = c->ix_cstart;
    a.nextra = c->ix_nextra;
    a.nres = c->ix_nres;
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
    a.extra_limit = c->extra_limit;
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


void set_index_args(fmdp_ctx* c, RolloutArgs& ra, const Geometry& g) {
    ra.indexed = c->index_on ? 1 : 0;
    ra.icap = g.icap;
    ra.iv = index_view(c);
    ra.items_ctr = (c->index_on && c->profiling && !c->capturing) ? c->items_ctr : nullptr;
    ra.qe_ctr = ra.items_ctr ? c->items_ctr + 1 : nullptr;
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
    CK(cudaMemsetAsync(c->ix_nres, 0, ((size_t)c->T_win + 16) * sizeof(int32_t), c->stream));
    CK(cudaMemsetAsync(c->ix_dirty, 0, (size_t)c->T_win * sizeof(int32_t), c->stream));
}
// Appends admitted trajectories (request work items; see IndexAppendArgs) to the extra
// lists of their rows and publishes them; then (rebuild_dirty) rebuilds the rows that grew
// past the limit among [a, b).
void index_append_admitted(fmdp_ctx* c, const float* traj, int32_t cap, const RolloutOut* rout,
                           const fmdp_request* reqs, const SepOut* sep, const int32_t* slots, const int32_t* idx,
                           const int32_t* n_dev, int32_t n_items, int64_t a, int64_t b, bool rebuild_dirty) {
    if (!c->index_on) return;
    IndexAppendArgs ia{};
    ia.ix = index_args(c);
    ia.slots = slots;
    ia.traj = traj;
    ia.cap = cap;
    ia.rout = rout;
    ia.reqs = reqs;
    ia.sep = sep;
    ia.idx = idx;
    ia.n_dev = n_dev;
    LAUNCH(c, launch_index_append(ia, n_items, cap, c->stream));
    LAUNCH(c, launch_index_publish(ia.ix, c->stream));
    if (rebuild_dirty) index_rebuild(c, a, b, true);
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
    return {c->A, c->opt.combine, bit_length((int64_t)c->book.size()), bit_length(wave)};
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
Geometry geometry_indexed(fmdp_ctx* c, int32_t S_scan, int32_t wave) {
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
    const int32_t s = c->book.free_slots.lowest();
    c->book.free_slots.erase(s);
    return s;
}

void recompute_hw(fmdp_ctx* c) {
    c->book.S_hw = c->book.slot_bound();
}

// Enqueue rollout -> sep_check -> admission for n requests (device array c->reqs, slots in
// c->slots) in FCFS order on the context's stream.
void enqueue_sequence(fmdp_ctx* c, SeqBuffers& B, const fmdp_request* host_reqs, int32_t n, int32_t cap,
                      const Geometry& g, bool plan) {
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
        index_append_admitted(c, ra.traj, cap, ra.out, ra.reqs, sa.out, aa.slots, nullptr, nullptr, 1, d0,
                              d0 + host_reqs[i].horizon + 1);
        if (c->req_ev_base >= 0) CK(cudaEventRecord(c->req_ev[c->req_ev_base + i], c->stream));
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
void store_plans(fmdp_ctx* c, int32_t n_plans, const int64_t* t0s, const int32_t* counts, const float* xyz,
                 uint64_t* ids_out) {
    const NvtxRange range("fmdp store plans");
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
                ia.slots = c->slots.p;
                ia.traj = c->traj.p;
                ia.force = 1;
                ia.t0s = c->t0s.p;
                ia.counts = c->counts.p;
                ia.offs = c->offs.p;
                LAUNCH(c, launch_index_append(ia, n_plans, maxc, c->stream));
                LAUNCH(c, launch_index_publish(ia.ix, c->stream));
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
        c->book.add(id, PlanMeta{sl[i], t0s[i], counts[i]});
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

void expire_to(fmdp_ctx* c, int64_t t_now, int64_t* n_expired, bool sync) {
    const NvtxRange range("fmdp expiry");
    if (t_now <= c->book.t_base) return;
    Book& bk = c->book;
    const int64_t n = bk.expire(t_now);
    clear_rows(c, c->book.t_base, t_now);
    c->book.t_base = t_now;
    // the slot high-water mark stays an upper bound (it only sizes scans): lowered only when
    // the table empties, not by walking every plan
    if (bk.empty()) c->book.S_hw = 0;
    if (sync) CK(cudaStreamSynchronize(c->stream));
    if (n_expired) *n_expired += n;
}

void destroy_ctx(fmdp_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    pipe_release(c);
    for (float* p : {c->X, c->Y, c->Z, c->sX, c->sY, c->sZ})
        if (p) cudaFree(p);
    if (c->hm) cudaFree(c->hm);
    if (c->statics) cudaFree(c->statics);
    if (c->err) cudaFree(c->err);
    for (void* p : {(void*)c->ix_cstart, (void*)c->ix_nextra, (void*)c->ix_nres, (void*)c->ix_dirty, (void*)c->ix_items,
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
    for (cudaEvent_t e : c->req_ev) cudaEventDestroy(e);
    if (c->own) cudaStreamDestroy(c->own);
    delete c;
}

}  // namespace fmdp
