// Randomised check of the pipelined engine's influence test (paper_2008_03518_gb300/csrc/
// pipe_influence.cuh): first_influenced, which skips steps with chunk and group bounding
// boxes of both trajectories and the range of table-operation counts each chunk read,
// against the rule it accelerates taken step by step with no skipping:
//   - a decision step i of k (one with a next point) whose index read has a count in
//     [q_lo, q_hi) is influenced when k's state there lies within R_w + rho + 1 m of one of
//     j's wells one step later (centre p_j(t + 1) + tau_w v_j(t + 1), rho = k's step length
//     + the largest climb step + 1 m), counting only j's samples from jfloor on;
//   - when k's conflict check read the index with a count in [q_lo, q_hi), the verdict may
//     change if k and j come within the separation minima (+ 1 m, carried in H and V) at a
//     step, again only from jfloor on.
// The result is the first influenced decision step (-1: none) and the verdict flag, which
// counts the steps up to that one. Usage: influence_check <seed> <cases>. Prints
// "ok <hits> <seps> <clear>" and exits 0 when every case agrees.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "pipe_influence.cuh"

using fmdp::InflRule;
using fmdp::TrajBoxes;

namespace {

int rule_step_by_step(const InflRule& P, const float* pj, int nj, int64_t tj, int32_t q_lo, int32_t q_hi,
                      const float* pk, int nk, int64_t tk, double speed_k, const int32_t* obs_k, int32_t tail_obs,
                      bool* sep, int32_t jfloor) {
    *sep = false;
    if (nk <= 0 || nj <= 0 || !(tk < tj + nj && tj < tk + nk) || jfloor >= nj || q_lo >= q_hi) return -1;
    const bool sep_unseen = q_lo <= tail_obs && tail_obs < q_hi;
    const double rho = speed_k * P.dt + P.dzmax + 1.0;
    for (int i = 0; i < nk; ++i) {
        const double sx = pk[3 * i], sy = pk[3 * i + 1], sz = pk[3 * i + 2];
        const int64_t t0 = tk + i - tj;
        if (sep_unseen && t0 >= jfloor && t0 >= 0 && t0 < nj) {
            const double dx = sx - pj[3 * t0], dy = sy - pj[3 * t0 + 1], dz = sz - pj[3 * t0 + 2];
            if (dx * dx + dy * dy < P.H * P.H && std::fabs(dz) < P.V) *sep = true;
        }
        const int64_t t1 = t0 + 1;
        if (i + 1 >= nk || obs_k[i] < q_lo || obs_k[i] >= q_hi || t1 < 0 || t1 >= nj || t1 < jfloor) continue;
        const float* q1 = pj + 3 * t1;
        double vx = 0.0, vy = 0.0, vz = 0.0;
        if (t1 + 1 < nj) {
            vx = ((double)q1[3] - q1[0]) / P.dt;
            vy = ((double)q1[4] - q1[1]) / P.dt;
            vz = ((double)q1[5] - q1[2]) / P.dt;
        }
        for (int w = 0; w < P.n_wells; ++w) {
            const double r = P.R[w] + 1.0 + rho;
            const double dx = sx - (q1[0] + P.tau[w] * vx), dy = sy - (q1[1] + P.tau[w] * vy),
                         dz = sz - (q1[2] + P.tau[w] * vz);
            if (dx * dx + dy * dy + dz * dz < r * r) return i;
        }
    }
    return -1;
}

// a random flight: straight legs with turns, speed v (m per step), climbs up to 4 m per step
std::vector<float> flight(std::mt19937_64& rng, int n, double x, double y, double z, double v) {
    std::uniform_real_distribution<double> U(0.0, 1.0);
    std::vector<float> p(3 * (size_t)n);
    double h = U(rng) * 6.283185307179586, c = 0.0;
    for (int i = 0; i < n; ++i) {
        p[3 * i] = (float)x;
        p[3 * i + 1] = (float)y;
        p[3 * i + 2] = (float)z;
        if (U(rng) < 0.05) h += (U(rng) - 0.5) * 1.5;
        if (U(rng) < 0.05) c = (U(rng) - 0.5) * 8.0;
        x += v * std::cos(h);
        y += v * std::sin(h);
        z += c;
    }
    return p;
}

}  // namespace

int main(int argc, char** argv) {
    if (argc != 3) {
        std::printf("usage: influence_check <seed> <cases>\n");
        return 2;
    }
    std::mt19937_64 rng(std::strtoull(argv[1], nullptr, 10));
    const int cases = std::atoi(argv[2]);
    std::uniform_real_distribution<double> U(0.0, 1.0);
    InflRule P{};
    P.dt = 1.0;
    P.H = 151.0;
    P.V = 31.0;
    P.dzmax = 4.0;
    P.n_wells = 5;
    const double tau[5] = {0.0, 10.0, 20.0, -10.0, 30.0}, R[5] = {150.0, 200.0, 250.0, 100.0, 300.0};
    for (int w = 0; w < 5; ++w) {
        P.tau[w] = tau[w];
        P.R[w] = R[w];
    }
    long long hits = 0, seps = 0, clear = 0;
    for (int cs = 0; cs < cases; ++cs) {
        const int nk = 1 + (int)(rng() % 700), nj = 1 + (int)(rng() % 700);
        const double vk = 20.0 + 60.0 * U(rng), vj = 20.0 + 60.0 * U(rng);
        const double spread = U(rng) < 0.5 ? 3000.0 : 30000.0;  // crowded or far apart
        const int64_t tk = (int64_t)(rng() % 400);
        int64_t tj = (int64_t)(rng() % 400);
        const std::vector<float> pk = flight(rng, nk, spread * U(rng), spread * U(rng), 100.0 + 400.0 * U(rng), vk);
        std::vector<float> pj = flight(rng, nj, spread * U(rng), spread * U(rng), 100.0 + 400.0 * U(rng), vj);
        if (U(rng) < 0.7) {  // an encounter: j's sample s at k's sample m's step, a few hundred metres off
            const int m = (int)(rng() % (uint64_t)nk), s = (int)(rng() % (uint64_t)nj);
            tj = tk + m - s;
            const double a = 6.283185307179586 * U(rng), d = 600.0 * U(rng), dz = 80.0 * (U(rng) - 0.5);
            const double ox = pk[3 * m] + d * std::cos(a) - pj[3 * s], oy = pk[3 * m + 1] + d * std::sin(a) - pj[3 * s + 1],
                         oz = pk[3 * m + 2] + dz - pj[3 * s + 2];
            for (int i = 0; i < nj; ++i) {
                pj[3 * i] = (float)(pj[3 * i] + ox);
                pj[3 * i + 1] = (float)(pj[3 * i + 1] + oy);
                pj[3 * i + 2] = (float)(pj[3 * i + 2] + oz);
            }
        }
        // table-operation counts each step of k read: non-decreasing, starting anywhere
        std::vector<int32_t> obs(nk);
        int32_t q = (int32_t)(rng() % 50);
        for (int i = 0; i < nk; ++i) {
            if (U(rng) < 0.1) q += 1 + (int32_t)(rng() % 5);
            obs[i] = q;
        }
        const int32_t q_lo = (int32_t)(rng() % (uint64_t)(q + 10)), q_hi = q_lo + 1 + (int32_t)(rng() % 40);
        const int32_t tail_obs = U(rng) < 0.5 ? q_lo + (int32_t)(rng() % 40) : q + 1;
        const int32_t jfloor = U(rng) < 0.5 ? 0 : (int32_t)(rng() % (uint64_t)(nj + 2));
        TrajBoxes bk, bj;
        bk.build(pk.data(), nk, P.dt, obs.data());
        bj.build(pj.data(), nj, P.dt);
        bool s_fast = false, s_ref = false;
        const int f = fmdp::first_influenced(P, pj.data(), nj, tj, bj, q_lo, q_hi, pk.data(), nk, tk, vk, bk,
                                             obs.data(), tail_obs, &s_fast, jfloor);
        const int g = rule_step_by_step(P, pj.data(), nj, tj, q_lo, q_hi, pk.data(), nk, tk, vk, obs.data(), tail_obs,
                                        &s_ref, jfloor);
        if (f != g || s_fast != s_ref) {
            std::printf("case %d: first influenced step %d vs %d, verdict flag %d vs %d\n", cs, f, g, (int)s_fast,
                        (int)s_ref);
            return 1;
        }
        hits += f >= 0;
        seps += s_fast;
        clear += f < 0 && !s_fast;
    }
    std::printf("ok %lld %lld %lld\n", hits, seps, clear);
    return 0;
}
