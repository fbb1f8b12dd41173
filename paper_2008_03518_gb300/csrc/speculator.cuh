// The speculative state of a batched call or a serving run (host side).
#pragma once

#include "host.cuh"

namespace fmdp {

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
                    c->book.add(id, PlanMeta{slot, reqs[k].depart_step, fin_ro[k].n_points});
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
            index_append_admitted(c, B.traj.p, B.cap, B.rout.p, B.rq, B.sepo.p, aa.slots, aa.idx, aa.n_dev, n_cap,
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
            c->book.erase(pr.first);
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


}  // namespace fmdp
