// The pipelined engine's influence test on the host (Sec. III: a known plan changes a
// FastMDP step only through wells that reach the step's successors; Sec. V: a conflict is a
// pair inside both separation minima at one step). Included by the pipelined engine only;
// plain C++ with no CUDA types, so that it can be compiled and checked on a host.
#pragma once

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <vector>

namespace fmdp {

constexpr int kBoxChunk = 32;   // steps per bounding box of a trajectory
constexpr int kBoxSuper = 8;    // chunks per coarse box
constexpr int kInflWells = 8;   // wells per plan the rule holds (the model's maximum)

// ---------------------------------------------------------------- influence (host side)

// Bounding boxes of a trajectory over chunks of kBoxChunk steps and over groups of kBoxSuper
// chunks, its largest speed, and for each chunk and group the range of table-operation
// counts its decision steps read (obs: per step, or null).
struct TrajBoxes {
    std::vector<float> b;                // [chunks][6]: min x y z, max x y z
    std::vector<int32_t> omin, omax;     // [chunks]
    std::vector<float> sb;               // [groups][6]
    std::vector<int32_t> somin, somax;   // [groups]
    int32_t amin = INT32_MAX, amax = INT32_MIN;  // over every step
    double vmax = 0.0;
    void build(const float* p, int n, double dt, const int32_t* obs = nullptr) {
        const int nc = (n + kBoxChunk - 1) / kBoxChunk;
        b.assign((size_t)nc * 6, 0.f);
        omin.assign(nc, INT32_MAX);
        omax.assign(nc, INT32_MIN);
        if (obs)
            for (int i = 0; i + 1 < n; ++i) {
                omin[i / kBoxChunk] = std::min(omin[i / kBoxChunk], obs[i]);
                omax[i / kBoxChunk] = std::max(omax[i / kBoxChunk], obs[i]);
            }
        double v2 = 0.0;
        for (int c = 0; c < nc; ++c) {
            float* o = b.data() + 6 * c;
            o[0] = o[1] = o[2] = INFINITY;
            o[3] = o[4] = o[5] = -INFINITY;
            for (int i = c * kBoxChunk; i < std::min(n, (c + 1) * kBoxChunk); ++i)
                for (int a = 0; a < 3; ++a) {
                    o[a] = std::min(o[a], p[3 * i + a]);
                    o[3 + a] = std::max(o[3 + a], p[3 * i + a]);
                }
        }
        for (int i = 0; i + 1 < n; ++i) {
            const double dx = p[3 * i + 3] - p[3 * i], dy = p[3 * i + 4] - p[3 * i + 1], dz = p[3 * i + 5] - p[3 * i + 2];
            v2 = std::max(v2, dx * dx + dy * dy + dz * dz);
        }
        vmax = std::sqrt(v2) / dt;
        const int ng = (nc + kBoxSuper - 1) / kBoxSuper;
        sb.assign((size_t)ng * 6, 0.f);
        somin.assign(ng, INT32_MAX);
        somax.assign(ng, INT32_MIN);
        for (int g = 0; g < ng; ++g) {
            float* o = sb.data() + 6 * g;
            o[0] = o[1] = o[2] = INFINITY;
            o[3] = o[4] = o[5] = -INFINITY;
            for (int c = g * kBoxSuper; c < std::min(nc, (g + 1) * kBoxSuper); ++c) {
                for (int a = 0; a < 3; ++a) {
                    o[a] = std::min(o[a], b[6 * c + a]);
                    o[3 + a] = std::max(o[3 + a], b[6 * c + 3 + a]);
                }
                somin[g] = std::min(somin[g], omin[c]);
                somax[g] = std::max(somax[g], omax[c]);
            }
            amin = std::min(amin, somin[g]);
            amax = std::max(amax, somax[g]);
        }
    }
    // the box of steps [lo, hi] (clamped to the trajectory), from the coarsest boxes that fit
    void span(int64_t lo, int64_t hi, float* out) const {
        out[0] = out[1] = out[2] = INFINITY;
        out[3] = out[4] = out[5] = -INFINITY;
        int64_t c = lo / kBoxChunk;
        const int64_t c1 = hi / kBoxChunk;
        while (c <= c1) {
            const float* o;
            if (c % kBoxSuper == 0 && c + kBoxSuper - 1 <= c1) {
                o = sb.data() + 6 * (c / kBoxSuper);
                c += kBoxSuper;
            } else {
                o = b.data() + 6 * c;
                c += 1;
            }
            for (int a = 0; a < 3; ++a) {
                out[a] = std::min(out[a], o[a]);
                out[3 + a] = std::max(out[3 + a], o[3 + a]);
            }
        }
    }
};

struct InflRule {
    double dt, H, V, dzmax;
    int n_wells;
    double tau[kInflWells], R[kInflWells];
};

// Could trajectory j (of a request before k) change request k's plan or verdict at the steps
// where its presence in k's table differs from what k's rollout read? The rule of the
// batched path's influence kernel (one-step window), taken only at those steps: k's state at
// a step whose index rows were read with a table-operation count in [q_lo, q_hi) within
// reach of one of j's wells one step later (well w at p_j + tau_w v_j, radius R_w, reach R_w
// + the successor offset + 1 m); or, when k's conflict check read the index with a count in
// [q_lo, q_hi), the two within the separation minima + 1 m at one step. Chunk bounding boxes
// skip the steps where the two are far apart. Returns the first decision step j could
// change (-1: none); *sep: j could change the verdict. The steps before the first one keep
// their decisions, so the plan may go on from its state there.
// jfloor: j's items below this index (item i: sample i and the next one) did not change
// (only the items at or past it can make a difference).
inline int first_influenced(const InflRule& P, const float* pj, int nj, int64_t tj, const TrajBoxes& bj, int32_t q_lo,
                     int32_t q_hi, const float* pk, int nk, int64_t tk, double speed_k, const TrajBoxes& bk,
                     const int32_t* obs_k, int32_t tail_obs, bool* sep, int32_t jfloor = 0) {
    *sep = false;
    if (nk <= 0 || nj <= 0 || !(tk < tj + nj && tj < tk + nk) || jfloor >= nj || q_lo >= q_hi) return -1;
    const bool sep_unseen = q_lo <= tail_obs && tail_obs < q_hi;
    if (!sep_unseen && (bk.amax < q_lo || bk.amin >= q_hi)) return -1;  // no step read j differently
    const double rho = speed_k * P.dt + P.dzmax + 1.0;
    double e = std::max(P.H, P.V);
    for (int w = 0; w < P.n_wells; ++w) e = std::max(e, P.R[w] + 1.0 + rho + std::fabs(P.tau[w]) * bj.vmax);
    e += 1.0;
    // k's steps i that can meet one of j's items at or past jfloor: the same step's sample
    // (t0 = tk + i - tj), the next one and the one after it, so t0 in [jfloor - 2, nj)
    const int64_t i_lo = std::max<int64_t>(0, tj + jfloor - 2 - tk), i_hi = std::min<int64_t>(nk, tj + nj - tk);
    if (i_lo >= i_hi) return -1;
    // j's boxes over the samples a range of k's steps [i0, i1) can meet: the same step, the
    // next, and the one after it (the next sample's velocity); false when the range is apart
    auto near = [&](const float* ok, int64_t i0, int64_t i1) {
        const int64_t jlo = std::max<int64_t>(std::max<int64_t>(0, jfloor - 2), tk + i0 - tj);
        const int64_t jhi = std::min<int64_t>(nj - 1, tk + i1 - 1 - tj + 2);
        if (jlo > jhi) return false;
        float jb[6];
        bj.span(jlo, jhi, jb);
        for (int a = 0; a < 3; ++a)
            if (ok[a] > jb[3 + a] + e || ok[3 + a] < jb[a] - e) return false;
        return true;
    };
    const int c_lo = (int)(i_lo / kBoxChunk), c_hi = (int)((i_hi - 1) / kBoxChunk);
    for (int c = c_lo; c <= c_hi; ++c) {
        if (c % kBoxSuper == 0 || c == c_lo) {  // a group of chunks: skip it whole when it can
            const int g = c / kBoxSuper;
            const bool wells_g = bk.somax[g] >= q_lo && bk.somin[g] < q_hi;
            const int64_t g0 = std::max<int64_t>((int64_t)c * kBoxChunk, i_lo);
            const int64_t g1 = std::min<int64_t>(std::min<int64_t>((int64_t)(g + 1) * kBoxSuper * kBoxChunk, nk), i_hi);
            if ((!wells_g && (!sep_unseen || *sep)) || !near(bk.sb.data() + 6 * g, g0, g1)) {
                c = std::min(c_hi, (g + 1) * kBoxSuper - 1);
                continue;
            }
        }
        const int i0 = std::max<int>(c * kBoxChunk, (int)i_lo), i1 = std::min<int>(std::min(nk, (c + 1) * kBoxChunk), (int)i_hi);
        const bool wells_here = bk.omax[c] >= q_lo && bk.omin[c] < q_hi;
        if (!wells_here && (!sep_unseen || *sep)) continue;
        if (!near(bk.b.data() + 6 * c, i0, i1)) continue;
        for (int i = i0; i < i1; ++i) {
            const double sx = pk[3 * i], sy = pk[3 * i + 1], sz = pk[3 * i + 2];
            const int64_t t0 = tk + i - tj;
            if (sep_unseen && !*sep && t0 >= jfloor && t0 >= 0 && t0 < nj) {
                const double dx = sx - pj[3 * t0], dy = sy - pj[3 * t0 + 1], dz = sz - pj[3 * t0 + 2];
                if (dx * dx + dy * dy < P.H * P.H && std::fabs(dz) < P.V) *sep = true;
            }
            const int64_t t1 = t0 + 1;
            // no decision at the last point; a step outside [q_lo, q_hi) read j as it stands
            if (i + 1 >= nk || obs_k[i] < q_lo || obs_k[i] >= q_hi || t1 < 0 || t1 >= nj || t1 < jfloor)
                continue;
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
    }
    return -1;
}

}  // namespace fmdp
