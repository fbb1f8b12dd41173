// C ABI of libfmdp (include/fmdp.h): argument checks and marshalling around the host
// runtime; every entry point returns an fmdp_status and never throws.
#include "speculator.cuh"

using namespace fmdp;

namespace {
thread_local std::string g_create_error;
}  // namespace

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
        require(o.batch_mode == 0 || o.batch_mode == 1, FMDP_ERR_ARG, "batch_mode must be 0 (pipelined) or 1 (waves)");
        require(o.pipe_rebuild_items >= 0, FMDP_ERR_ARG, "pipe_rebuild_items must be >= 0");
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
        CK(preload_index_kernels());
        CK(preload_table_kernels());
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
        c->book.reset(c->S_max, c->T_win);
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
            CK(cudaMalloc(&c->ix_nres, ((size_t)c->T_win + 16) * sizeof(int32_t)));
            CK(cudaMalloc(&c->ix_dirty, (size_t)c->T_win * sizeof(int32_t)));
            CK(cudaMalloc(&c->ix_items, plane * 2 * sizeof(float4)));
            CK(cudaMalloc(&c->items_ctr, 4 * sizeof(unsigned long long)));  // items; q_eval counters
            CK(cudaMemsetAsync(c->items_ctr, 0, 4 * sizeof(unsigned long long), c->stream));
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

// ---- plan table file: header, one record per plan, then every sample (little-endian, the
// layout of the structs below)
namespace {
struct PlanFileHeader {
    char magic[8];      // "FMDPPLN1"
    int64_t t_base;     // the table window's first step when saved
    int64_t n_plans;
    int64_t n_samples;  // sum of the records' counts
};
struct PlanFileRecord {
    int64_t t0;     // first step of the saved samples
    int32_t count;  // samples
    int32_t pad;
};
const char kPlanMagic[8] = {'F', 'M', 'D', 'P', 'P', 'L', 'N', '1'};
}  // namespace

fmdp_status fmdp_save_plans(fmdp_ctx* c, const char* path, int64_t* n_out) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        require(path != nullptr, FMDP_ERR_ARG, "null path");
        // the samples of every stored plan that are still in the window, in id order
        std::vector<int32_t> slots, counts;
        std::vector<int64_t> t0s, offs;
        int64_t total = 0;
        int32_t maxc = 0;
        c->book.for_each([&](uint64_t, const PlanMeta& p) {
            const int64_t a = std::max<int64_t>(p.t0, c->book.t_base), b = p.t0 + p.n;
            if (b <= a) return;
            slots.push_back(p.slot);
            t0s.push_back(a);
            counts.push_back((int32_t)(b - a));
            offs.push_back(total);
            total += b - a;
            maxc = std::max(maxc, (int32_t)(b - a));
        });
        const int64_t n = (int64_t)t0s.size();
        std::vector<float> xyz((size_t)total * 3);
        if (n > 0) {
            c->slots.ensure((size_t)n);
            c->t0s.ensure((size_t)n);
            c->offs.ensure((size_t)n);
            c->counts.ensure((size_t)n);
            c->traj.ensure((size_t)total * 3);
            CK(cudaMemcpyAsync(c->slots.p, slots.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
            CK(cudaMemcpyAsync(c->t0s.p, t0s.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
            CK(cudaMemcpyAsync(c->offs.p, offs.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
            CK(cudaMemcpyAsync(c->counts.p, counts.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
            LAUNCH(c, launch_gather_plans(c->X, c->Y, c->Z, c->S_pad, c->T_win, c->slots.p, c->t0s.p, c->counts.p,
                                          c->offs.p, c->traj.p, (int)n, maxc, c->stream));
            CK(cudaMemcpyAsync(xyz.data(), c->traj.p, (size_t)total * 3 * sizeof(float), cudaMemcpyDeviceToHost,
                               c->stream));
            CK(cudaStreamSynchronize(c->stream));
        }
        FILE* f = std::fopen(path, "wb");
        require(f != nullptr, FMDP_ERR_IO, "cannot open the plan file for writing");
        PlanFileHeader h{};
        std::memcpy(h.magic, kPlanMagic, 8);
        h.t_base = c->book.t_base;
        h.n_plans = n;
        h.n_samples = total;
        bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1;
        for (int64_t i = 0; ok && i < n; ++i) {
            const PlanFileRecord r{t0s[i], counts[i], 0};
            ok = std::fwrite(&r, sizeof(r), 1, f) == 1;
        }
        if (ok && total > 0) ok = std::fwrite(xyz.data(), sizeof(float), xyz.size(), f) == xyz.size();
        ok = (std::fclose(f) == 0) && ok;
        require(ok, FMDP_ERR_IO, "writing the plan file failed");
        if (n_out) *n_out = n;
    });
}

fmdp_status fmdp_load_plans(fmdp_ctx* c, const char* path, uint64_t* ids_out, int64_t cap, int64_t* n_out) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        require(path != nullptr && cap >= 0 && (cap == 0 || ids_out), FMDP_ERR_ARG, "null path or ids");
        FILE* f = std::fopen(path, "rb");
        require(f != nullptr, FMDP_ERR_IO, "cannot open the plan file");
        PlanFileHeader h{};
        std::vector<PlanFileRecord> recs;
        std::vector<float> xyz;
        bool ok = std::fread(&h, sizeof(h), 1, f) == 1 && std::memcmp(h.magic, kPlanMagic, 8) == 0 &&
                  h.n_plans >= 0 && h.n_samples >= 0 && h.n_plans <= (int64_t)c->S_max &&
                  h.n_samples <= (int64_t)c->S_max * c->T_win;
        if (ok) {
            recs.resize((size_t)h.n_plans);
            xyz.resize((size_t)h.n_samples * 3);
            ok = (h.n_plans == 0 || std::fread(recs.data(), sizeof(PlanFileRecord), recs.size(), f) == recs.size()) &&
                 (h.n_samples == 0 || std::fread(xyz.data(), sizeof(float), xyz.size(), f) == xyz.size());
        }
        std::fclose(f);
        require(ok, FMDP_ERR_IO, "not a plan file, or a truncated one");
        int64_t sum = 0;
        for (const auto& r : recs) {
            require(r.count >= 1, FMDP_ERR_IO, "a plan record without samples");
            sum += r.count;
        }
        require(sum == h.n_samples, FMDP_ERR_IO, "the records do not account for the samples");
        // an empty table takes the saved window (its rows are cleared on the way)
        if (c->book.empty() && h.t_base > c->book.t_base) expire_to(c, h.t_base, nullptr);
        std::vector<int64_t> t0s(recs.size());
        std::vector<int32_t> counts(recs.size());
        for (size_t i = 0; i < recs.size(); ++i) {
            t0s[i] = recs[i].t0;
            counts[i] = recs[i].count;
        }
        std::vector<uint64_t> ids(recs.size());
        int64_t off = 0;
        for (size_t i0 = 0; i0 < recs.size();) {  // in chunks of the packed call's size
            const int32_t m = (int32_t)std::min<size_t>(recs.size() - i0, 1u << 20);
            store_plans(c, m, t0s.data() + i0, counts.data() + i0, xyz.data() + 3 * off, ids.data() + i0);
            for (int32_t i = 0; i < m; ++i) off += counts[i0 + i];
            i0 += m;
        }
        for (int64_t i = 0; i < std::min<int64_t>(cap, (int64_t)ids.size()); ++i) ids_out[i] = ids[i];
        if (n_out) *n_out = (int64_t)recs.size();
    });
}

fmdp_status fmdp_query_plans(fmdp_ctx* c, int64_t t_begin, int64_t t_end, uint64_t* ids, int32_t cap,
                             int32_t* n_out) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        require(n_out && (cap == 0 || ids) && cap >= 0, FMDP_ERR_ARG, "null output");
        int32_t n = 0;
        c->book.for_each([&](uint64_t id, const PlanMeta& p) {
            if (p.t0 < t_end && p.t0 + p.n > t_begin) {
                if (n < cap) ids[n] = id;
                ++n;
            }
        });
        *n_out = n;
    });
}

fmdp_status fmdp_get_plan(fmdp_ctx* c, uint64_t id, int64_t* t0_out, float* xyz, int32_t cap, int32_t* n_out) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        const PlanMeta* pp = c->book.find(id);
        require(pp != nullptr, FMDP_ERR_NOTFOUND, "no such plan");
        const PlanMeta p = *pp;
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
        const size_t plans_before = c->book.size();
        int32_t st = FMDP_OK;
        try {
            run_fcfs(c, r, 2, nullptr, false, true, 1);
        } catch (const ApiError& f) {
            st = f.code;
        }
        if (observed) *observed = st;
        require(st == FMDP_ERR_TIMEOUT, FMDP_ERR_CUDA, "the self-test wait did not report a timeout");
        require(c->book.size() == plans_before, FMDP_ERR_CUDA, "the self-test admitted a plan");
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
        c->book.reset(c->S_max, c->T_win);
        c->book.t_base = tb;
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
        if (c->items_ctr) CK(cudaMemsetAsync(c->items_ctr, 0, 4 * sizeof(unsigned long long), c->stream));
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
            unsigned long long n[4] = {0, 0, 0, 0};
            CK(cudaMemcpyAsync(n, c->items_ctr, sizeof(n), cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
            out->items_scanned = (int64_t)n[0];
            out->qe_items = (int64_t)n[1];
            out->qe_near = (int64_t)n[2];
            out->qe_wells = (int64_t)n[3];
        }
        out->cluster_size = c->last_cs;
        out->threads_per_cta = c->last_threads;
        out->slots_per_cta = c->last_chunk;
    });
}

fmdp_status fmdp_set_batch_mode(fmdp_ctx* c, int32_t mode) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        require(mode == 0 || mode == 1, FMDP_ERR_ARG, "batch_mode must be 0 (pipelined) or 1 (waves)");
        c->opt.batch_mode = mode;
    });
}

fmdp_status fmdp_last_call_times(fmdp_ctx* c, double* ms, int32_t cap, int32_t* n_out) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        require(n_out && cap >= 0 && (cap == 0 || ms), FMDP_ERR_ARG, "null output");
        const int32_t n = (int32_t)std::min<size_t>(c->call_ms.size(), (size_t)cap);
        std::copy(c->call_ms.begin(), c->call_ms.begin() + n, ms);
        *n_out = (int32_t)c->call_ms.size();
    });
}

fmdp_status fmdp_probe_peaks(fmdp_ctx* c, fmdp_peaks* out) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        require(out != nullptr, FMDP_ERR_ARG, "null output");
        CK(cudaStreamSynchronize(c->stream));
        CK(probe_peaks(c->n_sm, c->stream, out));
    });
}

}  // extern "C"
