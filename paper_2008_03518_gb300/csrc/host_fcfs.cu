// First-come-first-served planning one request after another (Sec. I, Sec. V): each
// admitted trajectory is stored before the next request is planned, and the whole
// per-request chain (rollout -> separation check -> admission) is decided on the device.
#include "host.cuh"

namespace fmdp {

int32_t run_fcfs(fmdp_ctx* c, const fmdp_request* reqs, int32_t n, fmdp_result* res, bool staged,
                 bool cosim, int32_t absent) {
    const NvtxRange range("fmdp sequential FCFS");
    SeqBuffers& B = staged ? c->stg : c->seq;
    const bool keep_on_device = staged;
    int32_t admitted = 0;
    int32_t done = 0;
    // completion time of each request: an event after its admission step ([0] the start)
    while ((int32_t)c->req_ev.size() < n + 1) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        c->req_ev.push_back(e);
    }
    CK(cudaEventRecord(c->req_ev[n], c->stream));
    c->call_ms.assign(n, 0.0);
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
            c->req_ev_base = cosim ? -1 : done;
            enqueue_sequence(c, B, reqs + done, m, cap, g, !cosim);
            c->req_ev_base = -1;
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
            if (!cosim)
                for (int32_t i = 0; i < m; ++i) {
                    float ms = 0.f;
                    CK(cudaEventElapsedTime(&ms, c->req_ev[n], c->req_ev[done + i]));
                    c->call_ms[done + i] = ms;
                }
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
                c->book.add(id, PlanMeta{sl[i], rq.depart_step, ro.n_points});
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

}  // namespace fmdp
