// Learned proposal orchestration: parameters, training on the GPU with the library's own
// kernels, training-set collection from FastMDP rollouts, and the proposal evaluation.
#include "host.cuh"

namespace fmdp {



// ------------------------------------------------------------------ learned proposal


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


void learned_collect(fmdp_ctx* c, const fmdp_request* reqs, int32_t n) {
    const NvtxRange range("fmdp learned collect");
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

}  // namespace fmdp
