// Serving loop over an arrival trace.
#include "speculator.cuh"

namespace fmdp {


// ------------------------------------------------------------------ serving loop


// Continuous batching over an arrival trace (see fmdp_serve in the header).
void run_serve(fmdp_ctx* c, const fmdp_request* reqs, const double* arrival_s, int32_t n,
               const fmdp_serve_options& o, fmdp_result* res, double* latency_ms, fmdp_serve_report* rep) {
    const NvtxRange range("fmdp serve");
    const PipeServe ps{arrival_s, o, latency_ms, rep};
    if (pipeline_eligible(c) && pipeline_fits(c, n, &ps)) {  // continuous batching without waves
        run_pipeline(c, reqs, n, res, nullptr, false, &ps);
        return;
    }
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
                const int64_t active = (int64_t)c->book.size();
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
                c->book.for_each([&](uint64_t, const PlanMeta& p) { first_end = std::min(first_end, p.t0 + p.n); });
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

}  // namespace fmdp
