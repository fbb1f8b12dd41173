// FastMDP rollout with a lookahead window of W sub-steps (sm_103a).
//
// Sec. IV "Forward project" holds each action for W time steps of dt (the paper runs
// W = 10 at dt = 0.1 s), and the compute-value kernel (Alg. 9) keeps, per action, the
// largest value met along those W projected states. The state then advances by one step
// of dt to the chosen action's first projected state (Alg. 1, Delta_1). Here:
//   x_1 = s + move(a), x_j = x_(j-1) + move(a) (FP64, rounded at each sub-step);
//   value(x_j) = goal term - aggregate of the wells of the plans present at t + j (their
//                sample at t + j, velocity from t + j to t + j + 1) - hard-deck penalty;
//   Q(a) = max over j with x_j inside the box; a is valid when x_1 is inside.
//
// One CTA per request, 256 threads. Per step:
//   1. one thread per action builds its W projected states (the exact FP64 chain) and
//      their fp32 offsets from s;
//   2. goal terms per (action, sub-step) as a log2 offset from the goal term at s, from
//      the exact identity d - d_s = (|o|^2 - 2 G.o) / (d + d_s), G = goal - s, o the offset,
//      which keeps fp32 accurate to micrometres at any distance; static wells and the
//      terrain clearance per (action, sub-step) in fp32 with an FP64 re-evaluation inside
//      their bands;
//   3. every (sub-step, slot) pair of the W slices: a culled distance test per pair; a
//      pair within reach is handed to the warp, whose lanes (one per action) score its
//      wells for that sub-step in fp32, deciding d < R in FP64 inside the band;
//   4. per action, the W values g - N compared as (sign, log2 |g - N|), so that a large
//      penalty at one sub-step leaves the goal term's resolution at the others; Q in FP64;
//   5. argmax (lowest index on ties), near-tie record, exact FP64 advance, terminal tests.
// Every decision that is a threshold (box, well radius, clearance, capture) is taken in
// FP64 with the oracle's operation order wherever fp32 could be on the wrong side.
#include <climits>
#include <cmath>

#include "fmdp_internal.cuh"

namespace fmdp {

namespace {

constexpr int kLookThreads = 256;
constexpr unsigned kFullMask = 0xffffffffu;

struct LookLayout {
    size_t X, Y, Z, ox, oy, oz, inb, rel, lN, keys, sums, stat, Dx, Dy, Dz, Qa, Sa, misc, total;
};

__host__ __device__ inline LookLayout look_layout(int A, int W) {
    LookLayout L;
    const size_t AW = (size_t)A * W;
    size_t o = 0;
    auto al = [&](size_t a) { o = (o + a - 1) & ~(a - 1); };
    L.X = o; o += AW * 8;
    L.Y = o; o += AW * 8;
    L.Z = o; o += AW * 8;
    L.ox = o; o += AW * 4;
    L.oy = o; o += AW * 4;
    L.oz = o; o += AW * 4;
    L.inb = o; o += AW * 4;
    L.rel = o; o += AW * 4;   // log2 of goal term at x_j minus log2 of goal term at s
    L.lN = o; o += AW * 4;    // log2 of (penalty + deck) at x_j, -inf when zero
    L.keys = o; o += AW * 4;  // float keys of the largest well log-value (MAX)
    al(8);
    L.sums = o; o += AW * 8;  // fixed-point sums of well values (SUM)
    L.stat = o; o += (size_t)kMaxStatic * 3 * 4;  // static-well centres minus s (fp32)
    al(8);
    L.Dx = o; o += kHeadings * 8;
    L.Dy = o; o += kHeadings * 8;
    L.Dz = o; o += kMaxActions * 8;
    L.Qa = o; o += kMaxActions * 8;
    L.Sa = o; o += kMaxActions * 8;
    L.misc = o; o += 256;
    L.total = (o + 127) & ~size_t(127);
    return L;
}

// Per-step shared scalars.
struct LookState {
    double s[3];      // exact state
    double lgs;       // log2 of the goal term at s
    double step, cap2;
    float Gx, Gy, Gz, ds;  // goal - s (fp32) and its length
    float shx, shy, shz, slx, sly, slz;  // s as double-float
    double prev[3];   // state one step earlier (co-simulation velocity)
    int h, k, done, status, choice, near_ties;
};

// Grid barrier of a cooperative launch (all CTAs resident), bounded: false when the wait
// ran past about a second of SM cycles.
__device__ bool look_grid_sync(int32_t* bar, int n_ctas, int& gen) {
    __syncthreads();
    int ok = 1;
    if (threadIdx.x == 0) {
        __threadfence();
        const int g = gen;
        if (atomicAdd(&bar[0], 1) == n_ctas - 1) {
            atomicExch(&bar[0], 0);
            __threadfence();
            atomicExch(&bar[1], g + 1);
        } else {
            const long long t0 = clock64();
            while (atomicAdd(&bar[1], 0) == g) {
                if (clock64() - t0 > (1ll << 31)) {
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        gen = g + 1;
        __threadfence();
    }
    return __syncthreads_and(ok) != 0;
}

__device__ __forceinline__ unsigned long long look_sum_term(float l, float ref) {
    const float t = exp2f(l - ref) * 1099511627776.0f;  // 2^40 fixed point
    return (unsigned long long)__float2ull_rn(t);
}

// d < R for a plan well, in FP64 with the oracle's order of operations (no FMA).
__device__ __noinline__ bool look_well_exact(const Model& m, int w, double x, double y, double z, float p1x, float p1y,
                                             float p1z, float p2x, float p2y, float p2z, bool has2) {
    double vx = 0.0, vy = 0.0, vz = 0.0;
    if (has2) {
        vx = __ddiv_rn(__dsub_rn((double)p2x, (double)p1x), m.dt);
        vy = __ddiv_rn(__dsub_rn((double)p2y, (double)p1y), m.dt);
        vz = __ddiv_rn(__dsub_rn((double)p2z, (double)p1z), m.dt);
    }
    const double tau = m.w_tau64[w];
    const double cx = __dadd_rn((double)p1x, __dmul_rn(tau, vx));
    const double cy = __dadd_rn((double)p1y, __dmul_rn(tau, vy));
    const double cz = __dadd_rn((double)p1z, __dmul_rn(tau, vz));
    return norm3_64(__dsub_rn(x, cx), __dsub_rn(y, cy), __dsub_rn(z, cz)) < m.w_R64[w];
}

// d < R for a well of another aircraft of a co-simulated batch: centre = s_m + tau * v_m.
__device__ __noinline__ bool look_member_exact(const Model& m, int w, double x, double y, double z, double sx,
                                               double sy, double sz, double vx, double vy, double vz) {
    const double tau = m.w_tau64[w];
    const double cx = __dadd_rn(sx, __dmul_rn(tau, vx));
    const double cy = __dadd_rn(sy, __dmul_rn(tau, vy));
    const double cz = __dadd_rn(sz, __dmul_rn(tau, vz));
    return norm3_64(__dsub_rn(x, cx), __dsub_rn(y, cy), __dsub_rn(z, cz)) < m.w_R64[w];
}

__device__ __noinline__ bool look_static_exact(const Model& m, int w, double x, double y, double z) {
    const double* c = m.statics + 6 * w;
    return norm3_64(__dsub_rn(x, c[0]), __dsub_rn(y, c[1]), __dsub_rn(z, c[2])) < c[3];
}

__device__ __noinline__ float look_deck_exact(const Model& m, double x, double y, double z) {
    const double c = __dsub_rn(z, terrain64(m, x, y));
    return c < m.clearance ? (float)__dsub_rn(m.deck, c) : 0.f;
}

}  // namespace

size_t lookahead_smem_bytes(int A, int W) { return look_layout(A, W).total; }

__global__ void __launch_bounds__(kLookThreads) lookahead_kernel(const __grid_constant__ LookArgs a) {
    extern __shared__ __align__(128) unsigned char lsm[];
    const Model& m = a.m;
    const int A = m.A, W = a.W, AW = A * W;
    const LookLayout L = look_layout(A, W);
    double* X = reinterpret_cast<double*>(lsm + L.X);
    double* Y = reinterpret_cast<double*>(lsm + L.Y);
    double* Z = reinterpret_cast<double*>(lsm + L.Z);
    float* ox = reinterpret_cast<float*>(lsm + L.ox);
    float* oy = reinterpret_cast<float*>(lsm + L.oy);
    float* oz = reinterpret_cast<float*>(lsm + L.oz);
    int* inb = reinterpret_cast<int*>(lsm + L.inb);
    float* rel = reinterpret_cast<float*>(lsm + L.rel);
    float* lN = reinterpret_cast<float*>(lsm + L.lN);
    int* keys = reinterpret_cast<int*>(lsm + L.keys);
    unsigned long long* sums = reinterpret_cast<unsigned long long*>(lsm + L.sums);
    float* stc = reinterpret_cast<float*>(lsm + L.stat);
    double* Dx = reinterpret_cast<double*>(lsm + L.Dx);
    double* Dy = reinterpret_cast<double*>(lsm + L.Dy);
    double* Dz = reinterpret_cast<double*>(lsm + L.Dz);
    double* Qa = reinterpret_cast<double*>(lsm + L.Qa);
    double* Sa = reinterpret_cast<double*>(lsm + L.Sa);
    LookState* st = reinterpret_cast<LookState*>(lsm + L.misc);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int r = blockIdx.x;
    if (r >= a.n_req) return;
    const fmdp_request req = a.reqs[r];
    float* traj = a.traj + (size_t)r * a.cap * 3;
    uint8_t* acts = a.acts + (size_t)r * a.cap;
    const int KEY_NONE = float_key(-INFINITY);
    const float inv_dt = (float)(1.0 / m.dt);
    const int S = a.S_scan;
    double* q_trace = a.trace ? a.q_trace + (size_t)r * a.cap * A : nullptr;
    double* st_trace = a.trace ? a.st_trace + (size_t)r * a.cap * 3 : nullptr;
    int32_t* hd_trace = a.trace ? a.hd_trace + (size_t)r * a.cap : nullptr;
    uint8_t* tie_trace = a.trace ? a.tie_trace + (size_t)r * a.cap : nullptr;

    // ---- prologue: heading table (the bearing turned by k * 15 degrees), climb moves
    if (tid < kHeadings) {
        const double dx = __dsub_rn(req.gx, req.ox), dy = __dsub_rn(req.gy, req.oy);
        const double Lh = __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
        double c0 = 1.0, s0 = 0.0;
        if (Lh > 0.0) {
            c0 = __ddiv_rn(dx, Lh);
            s0 = __ddiv_rn(dy, Lh);
        }
        double ck, sk;
        unit15(tid, ck, sk);
        const double C = __dsub_rn(__dmul_rn(c0, ck), __dmul_rn(s0, sk));
        const double Sn = __dadd_rn(__dmul_rn(s0, ck), __dmul_rn(c0, sk));
        const double step = __dmul_rn(req.speed_mps, m.dt);
        Dx[tid] = __dmul_rn(step, C);
        Dy[tid] = __dmul_rn(step, Sn);
    }
    if (tid < kMaxActions) Dz[tid] = tid < A ? __dmul_rn(m.climb[tid], m.dt) : 0.0;
    if (tid == 0) {
        st->s[0] = req.ox;
        st->s[1] = req.oy;
        st->s[2] = req.oz;
        st->h = 0;
        st->k = 0;
        st->near_ties = 0;
        st->step = __dmul_rn(req.speed_mps, m.dt);
        st->cap2 = __dmul_rn(st->step, st->step);
        traj[0] = (float)req.ox;
        traj[1] = (float)req.oy;
        traj[2] = (float)req.oz;
        st->prev[0] = req.ox;
        st->prev[1] = req.oy;
        st->prev[2] = req.oz;
        if (a.trace) {
            st_trace[0] = req.ox;
            st_trace[1] = req.oy;
            st_trace[2] = req.oz;
            hd_trace[0] = 0;
        }
        const double ex = __dsub_rn(req.gx, req.ox), ey = __dsub_rn(req.gy, req.oy), ez = __dsub_rn(req.gz, req.oz);
        const bool cap0 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez)) <= st->cap2;
        st->done = cap0 || req.horizon <= 0;
        st->status = cap0 ? kStatusCaptured : FMDP_REJ_HORIZON;
    }
    __syncthreads();
    // largest horizontal + vertical move of one sub-step (culling bound)
    float lstep = 0.f;
    for (int q = 0; q < A; ++q) lstep = fmaxf(lstep, fabsf((float)Dz[q]));
    lstep = sqrtf((float)(st->step * st->step) + lstep * lstep) * 1.0001f + 0.01f;

    int gen = 0;
    const int n_mem = a.cosim ? a.n_req : 0;
    for (int64_t tc = a.cosim ? a.t_start : req.depart_step;; ++tc) {
        const double* recs = nullptr;  // co-simulation: every aircraft's record of this step
        if (a.cosim) {
            double* mine = a.mem + ((size_t)(tc & 1) * n_mem + r) * 8;
            if (tid == 0) {
                const bool flying = !st->done && tc >= req.depart_step;
                for (int c = 0; c < 3; ++c) {
                    mine[c] = st->s[c];
                    mine[3 + c] = st->k > 0 ? __ddiv_rn(__dsub_rn(st->s[c], st->prev[c]), m.dt) : 0.0;
                }
                mine[6] = flying ? 1.0 : 0.0;
                mine[7] = st->done ? 0.0 : 1.0;
            }
            if (!look_grid_sync(a.bar, a.n_req + a.absent, gen)) {
                if (tid == 0) {
                    atomicExch(a.err, FMDP_ERR_TIMEOUT);
                    st->done = 1;
                }
                __syncthreads();
                break;
            }
            recs = a.mem + (size_t)(tc & 1) * n_mem * 8;
            int alive = 0;
            for (int q = tid; q < n_mem; q += kLookThreads) alive |= __ldcg(recs + (size_t)q * 8 + 7) != 0.0;
            if (!__syncthreads_or(alive)) break;
            if (st->done || tc < req.depart_step) continue;  // waiting for departure, or finished
        } else if (st->done) {
            break;
        }
        const int k = st->k;
        const int64_t t = req.depart_step + k;
        // ---- 1. projected states (thread per action) and per-step constants
        if (tid < A) {
            int hn = st->h + m.dh[tid];
            hn += hn < 0 ? 24 : 0;
            hn -= hn >= 24 ? 24 : 0;
            double x = st->s[0], y = st->s[1], z = st->s[2];
            for (int j = 0; j < W; ++j) {
                x = __dadd_rn(x, Dx[hn]);
                y = __dadd_rn(y, Dy[hn]);
                z = __dadd_rn(z, Dz[tid]);
                const int q = tid * W + j;
                X[q] = x;
                Y[q] = y;
                Z[q] = z;
                ox[q] = (float)__dsub_rn(x, st->s[0]);
                oy[q] = (float)__dsub_rn(y, st->s[1]);
                oz[q] = (float)__dsub_rn(z, st->s[2]);
                inb[q] = x >= m.box[0] && x <= m.box[3] && y >= m.box[1] && y <= m.box[4] && z >= m.box[2] &&
                         z <= m.box[5];
            }
        } else if (tid == 64) {
            const double Gx = __dsub_rn(req.gx, st->s[0]), Gy = __dsub_rn(req.gy, st->s[1]),
                         Gz = __dsub_rn(req.gz, st->s[2]);
            const double ds = norm3_64(Gx, Gy, Gz);
            st->lgs = __dadd_rn(m.log2rg, __dmul_rn(ds, m.lg64));
            st->Gx = (float)Gx;
            st->Gy = (float)Gy;
            st->Gz = (float)Gz;
            st->ds = (float)ds;
            st->shx = (float)st->s[0];
            st->shy = (float)st->s[1];
            st->shz = (float)st->s[2];
            st->slx = (float)__dsub_rn(st->s[0], (double)st->shx);
            st->sly = (float)__dsub_rn(st->s[1], (double)st->shy);
            st->slz = (float)__dsub_rn(st->s[2], (double)st->shz);
        } else if (tid >= 96 && tid - 96 < m.n_static) {
            const int w = tid - 96;
            const double* c = m.statics + 6 * w;
            stc[3 * w] = (float)__dsub_rn(c[0], st->s[0]);
            stc[3 * w + 1] = (float)__dsub_rn(c[1], st->s[1]);
            stc[3 * w + 2] = (float)__dsub_rn(c[2], st->s[2]);
        }
        for (int q = tid; q < AW; q += kLookThreads) {
            keys[q] = KEY_NONE;
            sums[q] = 0ull;
        }
        __syncthreads();
        const float shx = st->shx, shy = st->shy, shz = st->shz, slx = st->slx, sly = st->sly, slz = st->slz;

        // ---- 2. goal term offsets and static wells per (action, sub-step)
        for (int q = tid; q < AW; q += kLookThreads) {
            const float px = ox[q], py = oy[q], pz = oz[q];
            const float ex = st->Gx - px, ey = st->Gy - py, ez = st->Gz - pz;
            const float d = sqrtf(fmaf(ex, ex, fmaf(ey, ey, ez * ez)));
            const float num = fmaf(px, px, fmaf(py, py, pz * pz)) -
                              2.f * fmaf(st->Gx, px, fmaf(st->Gy, py, st->Gz * pz));
            const float den = d + st->ds;
            const float dd = den > 0.f ? num / den : 0.f;  // d(x_j) - d(s)
            rel[q] = dd * m.lg32;
            // static negative peaks (restricted volumes / terrain wells)
            float mb = -INFINITY;
            unsigned long long sb = 0ull;
            for (int w = 0; w < m.n_static; ++w) {
                const float ux = px - stc[3 * w], uy = py - stc[3 * w + 1], uz = pz - stc[3 * w + 2];
                const float d2 = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
                const float R2 = m.st_R2[w];
                bool in = d2 < R2;
                if (fabsf(d2 - R2) <= m.st_band[w]) in = look_static_exact(m, w, X[q], Y[q], Z[q]);
                if (in) {
                    const float l = fmaf(sqrtf(d2), m.st_lg[w], m.st_L[w]);
                    mb = fmaxf(mb, l);
                    if (m.combine) sb += look_sum_term(l, m.sum_ref);
                }
            }
            if (mb > -INFINITY) atomicMax(&keys[q], float_key(mb));
            if (sb) atomicAdd(&sums[q], sb);
        }

        // ---- 3. plan wells: every (sub-step, slot) pair, warp-cooperative scoring
        const int npairs = W * S;
        for (int base = warp * 32; base < npairs; base += kLookThreads) {
            const int idx = base + lane;
            int j = 0, i = 0;
            bool near = false;
            float p1x = 0.f, p1y = 0.f, p1z = 0.f, p2x = 0.f, p2y = 0.f, p2z = 0.f;
            if (idx < npairs) {
                j = idx / S;
                i = idx - j * S;
                const int64_t t1 = t + j + 1, t2 = t1 + 1;
                if (t1 >= a.tab.t_base && t1 < a.tab.t_base + a.tab.T_win) {
                    int64_t r1 = t1 % a.tab.T_win;
                    r1 += r1 < 0 ? a.tab.T_win : 0;
                    const size_t o1 = (size_t)r1 * a.tab.S_pad + i;
                    p1x = a.tab.X[o1];
                    p1y = a.tab.Y[o1];
                    p1z = a.tab.Z[o1];
                    p2x = __int_as_float(0x7fc00000);
                    if (t2 < a.tab.t_base + a.tab.T_win) {
                        int64_t r2 = t2 % a.tab.T_win;
                        r2 += r2 < 0 ? a.tab.T_win : 0;
                        const size_t o2 = (size_t)r2 * a.tab.S_pad + i;
                        p2x = a.tab.X[o2];
                        p2y = a.tab.Y[o2];
                        p2z = a.tab.Z[o2];
                    }
                    if (p1x == p1x) {
                        const float qx = (p1x - shx) - slx, qy = (p1y - shy) - sly, qz = (p1z - shz) - slz;
                        float vv = 0.f;
                        if (p2x == p2x) {
                            const float vx = (p2x - p1x) * inv_dt, vy = (p2y - p1y) * inv_dt, vz = (p2z - p1z) * inv_dt;
                            vv = sqrtf(vx * vx + vy * vy + vz * vz);
                        }
                        const float reach = (float)(j + 1) * lstep + m.reach_base + m.tau_absmax * vv;
                        near = qx * qx + qy * qy + qz * qz < reach * reach;
                    }
                }
            }
            unsigned mask = __ballot_sync(kFullMask, near);
            while (mask) {
                const int b = __ffs(mask) - 1;
                mask &= mask - 1;
                const int jb = __shfl_sync(kFullMask, j, b);
                const float b1x = __shfl_sync(kFullMask, p1x, b), b1y = __shfl_sync(kFullMask, p1y, b),
                            b1z = __shfl_sync(kFullMask, p1z, b);
                const float b2x = __shfl_sync(kFullMask, p2x, b), b2y = __shfl_sync(kFullMask, p2y, b),
                            b2z = __shfl_sync(kFullMask, p2z, b);
                if (lane < A) {
                    const int q = lane * W + jb;
                    const bool has2 = b2x == b2x;
                    const float qx = (b1x - shx) - slx, qy = (b1y - shy) - sly, qz = (b1z - shz) - slz;
                    float vx = 0.f, vy = 0.f, vz = 0.f;
                    if (has2) {
                        vx = (b2x - b1x) * inv_dt;
                        vy = (b2y - b1y) * inv_dt;
                        vz = (b2z - b1z) * inv_dt;
                    }
                    const float px = ox[q], py = oy[q], pz = oz[q];
                    float mb = -INFINITY;
                    unsigned long long sb = 0ull;
                    for (int w = 0; w < m.n_wells; ++w) {
                        const float tau = m.w_tau[w];
                        const float ux = px - fmaf(tau, vx, qx), uy = py - fmaf(tau, vy, qy), uz = pz - fmaf(tau, vz, qz);
                        const float d2 = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
                        const float R2 = m.w_R2[w];
                        bool in = d2 < R2;
                        if (fabsf(d2 - R2) <= m.w_band[w])
                            in = look_well_exact(m, w, X[q], Y[q], Z[q], b1x, b1y, b1z, b2x, b2y, b2z, has2);
                        if (in) {
                            const float l = fmaf(sqrtf(d2), m.w_lg[w], m.w_L[w]);
                            mb = fmaxf(mb, l);
                            if (m.combine) sb += look_sum_term(l, m.sum_ref);
                        }
                    }
                    if (mb > -INFINITY) atomicMax(&keys[q], float_key(mb));
                    if (sb) atomicAdd(&sums[q], sb);
                }
            }
        }

        // ---- 3'. co-simulation: the wells of every other aircraft in flight, at its
        // position at t plus tau times its last move (the same peaks for every sub-step)
        if (recs) {
            const int nmp = W * n_mem;
            for (int base = warp * 32; base < nmp; base += kLookThreads) {
                const int idx = base + lane;
                int j = 0;
                bool near = false;
                double msx = 0.0, msy = 0.0, msz = 0.0, mvx = 0.0, mvy = 0.0, mvz = 0.0;
                if (idx < nmp) {
                    j = idx / n_mem;
                    const int mm = idx - j * n_mem;
                    const double* rc = recs + (size_t)mm * 8;
                    if (mm != r && __ldcg(rc + 6) != 0.0) {
                        msx = __ldcg(rc);
                        msy = __ldcg(rc + 1);
                        msz = __ldcg(rc + 2);
                        mvx = __ldcg(rc + 3);
                        mvy = __ldcg(rc + 4);
                        mvz = __ldcg(rc + 5);
                        const float qx = (float)__dsub_rn(msx, st->s[0]), qy = (float)__dsub_rn(msy, st->s[1]),
                                    qz = (float)__dsub_rn(msz, st->s[2]);
                        const float vv = sqrtf((float)(mvx * mvx + mvy * mvy + mvz * mvz));
                        const float reach = (float)(j + 1) * lstep + m.reach_base + m.tau_absmax * vv;
                        near = qx * qx + qy * qy + qz * qz < reach * reach;
                    }
                }
                unsigned mask = __ballot_sync(kFullMask, near);
                while (mask) {
                    const int b = __ffs(mask) - 1;
                    mask &= mask - 1;
                    const int jb = __shfl_sync(kFullMask, j, b);
                    const double bsx = __shfl_sync(kFullMask, msx, b), bsy = __shfl_sync(kFullMask, msy, b),
                                 bsz = __shfl_sync(kFullMask, msz, b);
                    const double bvx = __shfl_sync(kFullMask, mvx, b), bvy = __shfl_sync(kFullMask, mvy, b),
                                 bvz = __shfl_sync(kFullMask, mvz, b);
                    if (lane < A) {
                        const int q = lane * W + jb;
                        const float qx = (float)__dsub_rn(bsx, st->s[0]), qy = (float)__dsub_rn(bsy, st->s[1]),
                                    qz = (float)__dsub_rn(bsz, st->s[2]);
                        const float vx = (float)bvx, vy = (float)bvy, vz = (float)bvz;
                        const float px = ox[q], py = oy[q], pz = oz[q];
                        float mb = -INFINITY;
                        unsigned long long sb = 0ull;
                        for (int w = 0; w < m.n_wells; ++w) {
                            const float tau = m.w_tau[w];
                            const float ux = px - fmaf(tau, vx, qx), uy = py - fmaf(tau, vy, qy),
                                        uz = pz - fmaf(tau, vz, qz);
                            const float d2 = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
                            const float R2 = m.w_R2[w];
                            bool in = d2 < R2;
                            if (fabsf(d2 - R2) <= m.w_band[w])
                                in = look_member_exact(m, w, X[q], Y[q], Z[q], bsx, bsy, bsz, bvx, bvy, bvz);
                            if (in) {
                                const float l = fmaf(sqrtf(d2), m.w_lg[w], m.w_L[w]);
                                mb = fmaxf(mb, l);
                                if (m.combine) sb += look_sum_term(l, m.sum_ref);
                            }
                        }
                        if (mb > -INFINITY) atomicMax(&keys[q], float_key(mb));
                        if (sb) atomicAdd(&sums[q], sb);
                    }
                }
            }
        }
        __syncthreads();

        // ---- penalty + deck per (action, sub-step), as log2
        for (int q = tid; q < AW; q += kLookThreads) {
            float P = 0.f;
            if (m.combine) {
                if (sums[q]) P = (float)((double)sums[q] * m.sum_scale);
            } else if (keys[q] != KEY_NONE) {
                P = exp2f(key_float(keys[q]));
            }
            float D = 0.f;
            if (m.hm) {
                const float c32 = (float)Z[q] - terrain32(m, (float)X[q], (float)Y[q]);
                if (fabsf(c32 - (float)m.clearance) <= kClrBand + kTerrBand)
                    D = look_deck_exact(m, X[q], Y[q], Z[q]);
                else if (c32 < (float)m.clearance)
                    D = (float)m.deck - c32;
            }
            const float N = P + D;
            lN[q] = N > 0.f ? log2f(N) : -INFINITY;
        }
        __syncthreads();

        // ---- 4. per action: the largest value over its projected states inside the box.
        // A value g - N (goal term g = 2^Lg, penalty + deck N = 2^lN) is held as a sign and
        // log2 |g - N|, which keeps the goal term's resolution when N at another sub-step
        // is larger by hundreds of binary orders.
        if (tid < A) {
            const int q0 = tid * W;
            int bs = -2;  // no candidate yet
            double bL = 0.0, bsc = 0.0;
            for (int j = 0; j < W; ++j) {
                const int q = q0 + j;
                if (j > 0 && !inb[q]) continue;
                const double Lg = __dadd_rn(st->lgs, (double)rel[q]);
                const float ln = lN[q];
                int sg;
                double Lv, Ls;
                if (ln == -INFINITY) {
                    sg = 1;
                    Lv = Lg;
                    Ls = Lg;
                } else {
                    const double x = __dsub_rn((double)ln, Lg);  // log2 (N / g)
                    Ls = fmax(Lg, (double)ln);
                    if (x < -30.0) {
                        sg = 1;
                        Lv = Lg;
                    } else if (x > 30.0) {
                        sg = -1;
                        Lv = (double)ln;
                    } else {
                        const float r = exp2f((float)x);
                        if (r < 1.f) {
                            sg = 1;
                            Lv = __dadd_rn(Lg, (double)log2f(1.f - r));
                        } else if (r > 1.f) {
                            sg = -1;
                            Lv = __dadd_rn(Lg, (double)log2f(r - 1.f));
                        } else {
                            sg = 0;
                            Lv = 0.0;
                        }
                    }
                }
                bool better;
                if (bs == -2) better = true;
                else if (sg != bs) better = sg > bs;
                else better = sg > 0 ? Lv > bL : (sg < 0 ? Lv < bL : false);
                if (better) {
                    bs = sg;
                    bL = Lv;
                    bsc = Ls;
                }
            }
            Qa[tid] = inb[q0] ? (bs == 0 ? 0.0 : (double)bs * exp2(bL)) : -INFINITY;
            Sa[tid] = exp2(bsc);
        }
        __syncthreads();

        // ---- 5. argmax, near-tie record, advance (warp 0)
        if (warp == 0) {
            const double q = lane < A ? Qa[lane] : -INFINITY;
            double mx = q;
            for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(kFullMask, mx, o));
            const unsigned bm = __ballot_sync(kFullMask, lane < A && q == mx && mx > -INFINITY);
            const int a1 = bm ? __ffs(bm) - 1 : -1;
            double q2 = (lane < A && lane != a1) ? q : -INFINITY;
            for (int o = 16; o; o >>= 1) q2 = fmax(q2, __shfl_xor_sync(kFullMask, q2, o));
            const unsigned b2 = __ballot_sync(kFullMask, lane < A && lane != a1 && q == q2 && q2 > -INFINITY);
            const int a2 = b2 ? __ffs(b2) - 1 : -1;
            if (a.trace && lane < A) q_trace[(size_t)k * A + lane] = q;
            if (lane == 0) {
                bool tie = false;
                if (a1 >= 0 && a2 >= 0) {
                    double sc = fmax(fabs(Qa[a1]), fabs(Qa[a2]));
                    sc = fmax(sc, fmax(Sa[a1], Sa[a2]));
                    tie = __dsub_rn(Qa[a1], Qa[a2]) < kTieRel * sc;
                }
                if (a.trace) tie_trace[k] = tie ? 1 : 0;
                st->near_ties += tie ? 1 : 0;
                if (a1 < 0) {
                    st->status = FMDP_REJ_NO_ACTION;
                    st->done = 1;
                } else {
                    const int q0 = a1 * W;
                    st->prev[0] = st->s[0];
                    st->prev[1] = st->s[1];
                    st->prev[2] = st->s[2];
                    st->s[0] = X[q0];
                    st->s[1] = Y[q0];
                    st->s[2] = Z[q0];
                    int hn = st->h + m.dh[a1];
                    hn += hn < 0 ? 24 : 0;
                    hn -= hn >= 24 ? 24 : 0;
                    st->h = hn;
                    acts[k] = (uint8_t)a1;
                    const int np = k + 1;
                    traj[3 * np] = (float)st->s[0];
                    traj[3 * np + 1] = (float)st->s[1];
                    traj[3 * np + 2] = (float)st->s[2];
                    if (a.trace) {
                        st_trace[3 * np] = st->s[0];
                        st_trace[3 * np + 1] = st->s[1];
                        st_trace[3 * np + 2] = st->s[2];
                        hd_trace[np] = hn;
                    }
                    st->k = np;
                    const double ex = __dsub_rn(req.gx, st->s[0]), ey = __dsub_rn(req.gy, st->s[1]),
                                 ez = __dsub_rn(req.gz, st->s[2]);
                    if (__dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez)) <= st->cap2) {
                        st->status = kStatusCaptured;
                        st->done = 1;
                    } else if (np >= req.horizon) {
                        st->status = FMDP_REJ_HORIZON;
                        st->done = 1;
                    }
                }
            }
        }
        __syncthreads();
    }
    if (tid == 0) {
        RolloutOut o;
        o.n_points = st->k + 1;
        o.status = st->status;
        o.near_ties = st->near_ties;
        o.steps = st->k;
        a.out[r] = o;
    }
}

cudaError_t prepare_lookahead_kernel() {
    return cudaFuncSetAttribute(lookahead_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)look_layout(kMaxActions, kMaxLookahead).total);
}

int lookahead_max_resident(int A, int W) {
    int per_sm = 0, dev = 0, n_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lookahead_kernel, kLookThreads,
                                                      look_layout(A, W).total) != cudaSuccess ||
        cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm * n_sm;
}

cudaError_t launch_lookahead(const LookArgs& a, cudaStream_t s) {
    if (a.n_req <= 0) return cudaSuccess;
    if (!a.cosim) {
        lookahead_kernel<<<a.n_req, kLookThreads, look_layout(a.m.A, a.W).total, s>>>(a);
        return cudaGetLastError();
    }
    // co-simulation: every CTA must be resident at once (they wait for one another)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)a.n_req, 1, 1);
    cfg.blockDim = dim3(kLookThreads, 1, 1);
    cfg.dynamicSmemBytes = look_layout(a.m.A, a.W).total;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, lookahead_kernel, a);
}

}  // namespace fmdp
