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
    size_t ox, oy, oz, inb, rel, lN, vsg, vlv, vlr, vls, keys, sums, stat, Dx, Dy, Dz, Dh, Dz2, hna, sg, Lk, Lq, Ls,
        misc, total;
};

__host__ __device__ inline LookLayout look_layout(int A, int W) {
    LookLayout L;
    const size_t AW = (size_t)A * W;
    size_t o = 0;
    auto al = [&](size_t a) { o = (o + a - 1) & ~(a - 1); };
    L.ox = o; o += AW * 4;    // offsets of the projected states from s (fp32)
    L.oy = o; o += AW * 4;
    L.oz = o; o += AW * 4;
    L.inb = o; o += AW * 4;   // projected state inside the box
    L.rel = o; o += AW * 4;   // log2 of the goal term at x_j minus log2 of the goal term at s
    L.lN = o; o += AW * 4;    // log2 of (penalty + deck) at x_j, -inf when zero
    L.vsg = o; o += AW * 4;   // value g - N at x_j: sign class (2 bits) and whether vlv is absolute
    L.vlv = o; o += AW * 4;   // log2 |g - N| (relative to n0, or absolute when penalty dominated)
    L.vlr = o; o += AW * 4;   // log2 |g - N| relative to n0 (for comparisons)
    L.vls = o; o += AW * 4;   // log2 of the term scale max(g, N) relative to n0
    L.keys = o; o += AW * 4;  // float keys of the largest well log-value (MAX)
    al(8);
    L.sums = o; o += AW * 8;  // fixed-point sums of well values (SUM)
    L.stat = o; o += (size_t)kMaxStatic * 3 * 4;  // static-well centres minus s (fp32)
    al(8);
    L.Dx = o; o += kHeadings * 8;    // exact moves per heading (FP64)
    L.Dy = o; o += kHeadings * 8;
    L.Dz = o; o += kMaxActions * 8;  // exact climb per action (FP64)
    L.Dh = o; o += kHeadings * 4 * 4;     // the moves as double-float: xh, xl, yh, yl per heading
    L.Dz2 = o; o += kMaxActions * 2 * 4;  // climb as double-float
    L.hna = o; o += kMaxActions * 4;      // heading index after each action's turn
    L.sg = o; o += kMaxActions * 4;       // per action: sign class of Q (-1, 0, 1), -2 invalid
    al(8);
    L.Lk = o; o += kMaxActions * 8;       // per action: log2 |Q| (FP64, absolute)
    L.Lq = o; o += kMaxActions * 8;       // per action: log2 of the term scale max(g, N)
    L.Ls = o; o += kMaxActions * 8;       // per action: argmax key
    L.misc = o; o += 256;
    L.total = (o + 127) & ~size_t(127);
    return L;
}

// Per-step shared scalars.
struct LookState {
    double s[3];      // exact state
    double prev[3];   // state one step earlier (co-simulation velocity)
    double step, cap2;
    float shx, shy, shz, slx, sly, slz;  // s as double-float
    float Ghx, Ghy, Ghz, Glx, Gly, Glz;  // goal - s as double-float
    float Gx, Gy, Gz, ds, phi;           // goal - s (fp32), its length, log2 g(s) - n0
    int n0;                              // integer part of log2 of the goal term at s
    int h, k, done, status, near_ties;
    int tie_k, tie_a1, tie_a2;  // near-tie test of step tie_k still to do (tie_k < 0: none)
    int tie_s1, tie_s2;
    double tie_L1, tie_L2, tie_T1, tie_T2;
    int64_t row0;     // ring row of t + 1 for the current step
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
    const float t = exp2f(l - ref) * kSumUnits;  // fixed point, 2^-kSumBits of the largest |r|
    return (unsigned long long)__float2ull_rn(t);
}

// ---- double-float (fp32 pair) arithmetic: exact sums of fp32 numbers
__device__ __forceinline__ void lk_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void lk_fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ void lk_df_add(float& hi, float& lo, float dh, float dl) {
    float s, e;
    lk_two_sum(hi, dh, s, e);
    e = __fadd_rn(e, __fadd_rn(lo, dl));
    lk_fast_two_sum(s, e, hi, lo);
}
// log2 of the goal term |r_g| gamma^|G| at a state whose goal vector is the double-float G,
// split as n0 (integer) + phi (fraction in [0, 1)); also |G| in fp32
__device__ __forceinline__ void lk_goal_log(const Model& m, float Ghx, float Ghy, float Ghz, float Glx, float Gly,
                                            float Glz, int& n0, float& phi, float& dsf) {
    const float lg_hi = (float)m.lg64, lg_lo = (float)(m.lg64 - (double)(float)m.lg64);
    const float l2r_hi = (float)m.log2rg, l2r_lo = (float)(m.log2rg - (double)(float)m.log2rg);
    const float p0 = Ghx * Ghx, p1 = Ghy * Ghy, p2 = Ghz * Ghz;
    const float e0 = fmaf(Ghx, Ghx, -p0), e1 = fmaf(Ghy, Ghy, -p1), e2 = fmaf(Ghz, Ghz, -p2);
    float s1, t1, s2, t2;
    lk_two_sum(p0, p1, s1, t1);
    lk_two_sum(s1, p2, s2, t2);
    const float lo = t1 + t2 + e0 + e1 + e2 + 2.f * (Ghx * Glx + Ghy * Gly + Ghz * Glz);
    float Sh, Sl;
    lk_fast_two_sum(s2, lo, Sh, Sl);
    const float rt = Sh > 0.f ? sqrtf(Sh) : 0.f;
    const float rr = fmaf(-rt, rt, Sh);
    const float rl = rt > 0.f ? (rr + Sl) * (0.5f / rt) : 0.f;
    const float p = rt * lg_hi;
    const float pe = fmaf(rt, lg_hi, -p);
    const float lo2 = pe + rt * lg_lo + rl * lg_hi;
    float Lh, Le;
    lk_two_sum(p, l2r_hi, Lh, Le);
    Le = Le + (lo2 + l2r_lo);
    float LH, LL;
    lk_fast_two_sum(Lh, Le, LH, LL);
    float fl = floorf(LH);
    float fr = (LH - fl) + LL;
    if (fr >= 1.f) { fr -= 1.f; fl += 1.f; }
    if (fr < 0.f) { fr += 1.f; fl -= 1.f; }
    n0 = (int)fl;
    phi = fr;
    dsf = rt;
}

// The exact FP64 projected state x_(j+1) of a move (Dxa, Dya, Dza) from s: j + 1 rounded
// additions, as the oracle forms it. Called only where an fp32 decision falls in its band.
__device__ __noinline__ void look_state_exact(const double* s, double Dxa, double Dya, double Dza, int j, double& x,
                                              double& y, double& z) {
    x = s[0];
    y = s[1];
    z = s[2];
    for (int i = 0; i <= j; ++i) {
        x = __dadd_rn(x, Dxa);
        y = __dadd_rn(y, Dya);
        z = __dadd_rn(z, Dza);
    }
}

// d < R for a plan well, in FP64 with the oracle's order of operations (no FMA).
__device__ __noinline__ bool look_well_exact(const Model& m, int w, const double* s, double Dxa, double Dya, double Dza,
                                             int j, float p1x, float p1y, float p1z, float p2x, float p2y, float p2z,
                                             bool has2) {
    double x, y, z;
    look_state_exact(s, Dxa, Dya, Dza, j, x, y, z);
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
__device__ __noinline__ bool look_member_exact(const Model& m, int w, const double* s, double Dxa, double Dya,
                                               double Dza, int j, double sx, double sy, double sz, double vx,
                                               double vy, double vz) {
    double x, y, z;
    look_state_exact(s, Dxa, Dya, Dza, j, x, y, z);
    const double tau = m.w_tau64[w];
    const double cx = __dadd_rn(sx, __dmul_rn(tau, vx));
    const double cy = __dadd_rn(sy, __dmul_rn(tau, vy));
    const double cz = __dadd_rn(sz, __dmul_rn(tau, vz));
    return norm3_64(__dsub_rn(x, cx), __dsub_rn(y, cy), __dsub_rn(z, cz)) < m.w_R64[w];
}

__device__ __noinline__ bool look_static_exact(const Model& m, int w, const double* s, double Dxa, double Dya,
                                               double Dza, int j) {
    double x, y, z;
    look_state_exact(s, Dxa, Dya, Dza, j, x, y, z);
    const double* c = m.statics + 6 * w;
    return norm3_64(__dsub_rn(x, c[0]), __dsub_rn(y, c[1]), __dsub_rn(z, c[2])) < c[3];
}

__device__ __noinline__ float look_deck_exact(const Model& m, const double* s, double Dxa, double Dya, double Dza,
                                              int j) {
    double x, y, z;
    look_state_exact(s, Dxa, Dya, Dza, j, x, y, z);
    const double c = __dsub_rn(z, terrain64(m, x, y));
    return c < m.clearance ? (float)__dsub_rn(m.deck, c) : 0.f;
}

__device__ __noinline__ bool look_box_exact(const Model& m, const double* s, double Dxa, double Dya, double Dza,
                                            int j) {
    double x, y, z;
    look_state_exact(s, Dxa, Dya, Dza, j, x, y, z);
    return x >= m.box[0] && x <= m.box[3] && y >= m.box[1] && y <= m.box[4] && z >= m.box[2] && z <= m.box[5];
}

__device__ __noinline__ bool look_capture_exact(const double* s, const fmdp_request& req, double cap2) {
    const double ex = __dsub_rn(req.gx, s[0]), ey = __dsub_rn(req.gy, s[1]), ez = __dsub_rn(req.gz, s[2]);
    return __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez)) <= cap2;
}

// Monotone 64-bit argmax key of a value held as (sign class, log2 |Q|): valid keys are > 0,
// Q > 0 above Q = 0 above Q < 0, and within a class ordered by Q (two low bits of log2 |Q|
// dropped).
__device__ __forceinline__ unsigned long long look_key(int sg, double L) {
    unsigned long long u = (unsigned long long)__double_as_longlong(L);
    u = (u >> 63) ? ~u : (u | 0x8000000000000000ull);  // increasing in L
    if (sg > 0) return (3ull << 62) | (u >> 2);
    if (sg == 0) return 2ull << 62;
    return (1ull << 62) | ((~u) >> 2);  // larger |Q| is a worse negative value
}

// Near-tie test of the two best actions from their (sign, log2 |Q|) and log2 scales:
// (Q1 - Q2) < 1e-4 * max(|Q1|, |Q2|, T1, T2), evaluated in the log domain.
__device__ __noinline__ bool look_near_tie(int s1, double L1, double T1, int s2, double L2, double T2) {
    double M = fmax(T1, T2);
    if (s1 != 0) M = fmax(M, L1);
    if (s2 != 0) M = fmax(M, L2);
    double gap;  // log2 (Q1 - Q2)
    if (s1 == s2) {
        if (s1 == 0) return true;
        const double hi = s1 > 0 ? L1 : L2, lo = s1 > 0 ? L2 : L1;  // Q1 >= Q2
        if (hi == lo) return true;
        gap = hi + (double)log2f(1.f - exp2f((float)(lo - hi)));
    } else if (s1 > 0 && s2 < 0) {
        const double hi = fmax(L1, L2), lo = fmin(L1, L2);
        gap = hi + (double)log2f(1.f + exp2f((float)(lo - hi)));
    } else {
        gap = s1 == 0 ? L2 : L1;  // one of them is zero
    }
    return gap < M - 13.287712379549449;  // log2(1e-4)
}

}  // namespace

size_t lookahead_smem_bytes(int A, int W) { return look_layout(A, W).total; }

__global__ void __launch_bounds__(kLookThreads) lookahead_kernel(const __grid_constant__ LookArgs a) {
    extern __shared__ __align__(128) unsigned char lsm[];
    const Model& m = a.m;
    const int A = m.A, W = a.W, AW = A * W;
    const LookLayout L = look_layout(A, W);
    float* ox = reinterpret_cast<float*>(lsm + L.ox);
    float* oy = reinterpret_cast<float*>(lsm + L.oy);
    float* oz = reinterpret_cast<float*>(lsm + L.oz);
    int* inb = reinterpret_cast<int*>(lsm + L.inb);
    float* rel = reinterpret_cast<float*>(lsm + L.rel);
    float* lN = reinterpret_cast<float*>(lsm + L.lN);
    int* vsg = reinterpret_cast<int*>(lsm + L.vsg);
    float* vlv = reinterpret_cast<float*>(lsm + L.vlv);
    float* vlr = reinterpret_cast<float*>(lsm + L.vlr);
    float* vls = reinterpret_cast<float*>(lsm + L.vls);
    int* keys = reinterpret_cast<int*>(lsm + L.keys);
    unsigned long long* sums = reinterpret_cast<unsigned long long*>(lsm + L.sums);
    float* stc = reinterpret_cast<float*>(lsm + L.stat);
    double* Dx = reinterpret_cast<double*>(lsm + L.Dx);
    double* Dy = reinterpret_cast<double*>(lsm + L.Dy);
    double* Dz = reinterpret_cast<double*>(lsm + L.Dz);
    float* Dh = reinterpret_cast<float*>(lsm + L.Dh);    // [24][4]: xh, xl, yh, yl
    float* Dz2 = reinterpret_cast<float*>(lsm + L.Dz2);  // [32][2]: zh, zl
    int* hna = reinterpret_cast<int*>(lsm + L.hna);
    int* sga = reinterpret_cast<int*>(lsm + L.sg);
    double* Lka = reinterpret_cast<double*>(lsm + L.Lk);
    double* Lqa = reinterpret_cast<double*>(lsm + L.Lq);
    unsigned long long* Ksa = reinterpret_cast<unsigned long long*>(lsm + L.Ls);
    LookState* st = reinterpret_cast<LookState*>(lsm + L.misc);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wi = blockIdx.x;
    if (wi >= a.n_req || (a.n_dev && wi >= *a.n_dev)) return;
    const int r = a.idx ? a.idx[wi] : wi;
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
    // near-tie flag of a finished step, taken off the step's chain (one thread)
    auto deferred_tie = [&]() {
        if (st->tie_k < 0) return;
        bool tie = false;
        if (st->tie_a1 >= 0 && st->tie_a2 >= 0)
            tie = look_near_tie(st->tie_s1, st->tie_L1, st->tie_T1, st->tie_s2, st->tie_L2, st->tie_T2);
        if (a.trace) tie_trace[st->tie_k] = tie ? 1 : 0;
        st->near_ties += tie ? 1 : 0;
        st->tie_k = -1;
    };
    const float box0 = (float)m.box[0], box1 = (float)m.box[1], box2 = (float)m.box[2];
    const float box3 = (float)m.box[3], box4 = (float)m.box[4], box5 = (float)m.box[5];
    constexpr float kBoxBandL = 0.01f;  // metres from a box face: decided in FP64
    constexpr float kCapBandL = 0.5f;   // metres around the capture radius: decided in FP64

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
        const double X = __dmul_rn(step, C), Y = __dmul_rn(step, Sn);
        Dx[tid] = X;
        Dy[tid] = Y;
        const float xh = (float)X, yh = (float)Y;
        Dh[4 * tid] = xh;
        Dh[4 * tid + 1] = (float)__dsub_rn(X, (double)xh);
        Dh[4 * tid + 2] = yh;
        Dh[4 * tid + 3] = (float)__dsub_rn(Y, (double)yh);
    }
    if (tid < kMaxActions) {
        const double dz = tid < A ? __dmul_rn(m.climb[tid], m.dt) : 0.0;
        Dz[tid] = dz;
        const float zh = (float)dz;
        Dz2[2 * tid] = zh;
        Dz2[2 * tid + 1] = (float)__dsub_rn(dz, (double)zh);
    }
    if (tid == 0) {
        st->s[0] = req.ox;
        st->s[1] = req.oy;
        st->s[2] = req.oz;
        st->h = 0;
        st->k = 0;
        st->near_ties = 0;
        st->tie_k = -1;
        st->step = __dmul_rn(req.speed_mps, m.dt);
        st->cap2 = __dmul_rn(st->step, st->step);
        traj[0] = (float)req.ox;
        traj[1] = (float)req.oy;
        traj[2] = (float)req.oz;
        st->prev[0] = req.ox;
        st->prev[1] = req.oy;
        st->prev[2] = req.oz;
        const double s0[3] = {req.ox, req.oy, req.oz}, g0[3] = {req.gx, req.gy, req.gz};
        float* sh = &st->shx;
        float* sl = &st->slx;
        float* gh = &st->Ghx;
        float* gl = &st->Glx;
        for (int c = 0; c < 3; ++c) {
            sh[c] = (float)s0[c];
            sl[c] = (float)__dsub_rn(s0[c], (double)sh[c]);
            const double G = __dsub_rn(g0[c], s0[c]);
            gh[c] = (float)G;
            gl[c] = (float)__dsub_rn(G, (double)gh[c]);
        }
        int64_t row = (req.depart_step + 1) % a.tab.T_win;
        st->row0 = row < 0 ? row + a.tab.T_win : row;
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
    for (int q = 0; q < A; ++q) lstep = fmaxf(lstep, fabsf(Dz2[2 * q]));
    const float stepf = (float)st->step;
    lstep = sqrtf(stepf * stepf + lstep * lstep) * 1.0001f + 0.01f;
    // Wells of a plan sample (offset q from s, velocity v) that can reach a projected state
    // within rho of s: centre within R + rho + 1 m. A well left out is more than 1 m outside
    // its radius at every projected state, so no fp32 rounding or band decision can flip it.
    auto well_mask = [&](float qx, float qy, float qz, float vx, float vy, float vz, float rho) {
        unsigned msk = 0u;
        for (int w = 0; w < m.n_wells; ++w) {
            const float tau = m.w_tau[w];
            const float cx = fmaf(tau, vx, qx), cy = fmaf(tau, vy, qy), cz = fmaf(tau, vz, qz);
            const float lim = sqrtf(m.w_R2[w]) + rho + 1.f;
            if (fmaf(cx, cx, fmaf(cy, cy, cz * cz)) < lim * lim) msk |= 1u << w;
        }
        return msk;
    };

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
        const int64_t row0 = st->row0;  // ring row of t + 1
        // ---- 1. per step: the goal term at s, static-well offsets, each action's heading
        if (tid < A) {
            int hn = st->h + m.dh[tid];
            hn += hn < 0 ? 24 : 0;
            hn -= hn >= 24 ? 24 : 0;
            hna[tid] = hn;
        } else if (tid == 64) {
            int n0;
            float phi, dsf;
            lk_goal_log(m, st->Ghx, st->Ghy, st->Ghz, st->Glx, st->Gly, st->Glz, n0, phi, dsf);
            st->n0 = n0;
            st->phi = phi;
            st->ds = dsf;
            st->Gx = st->Ghx + st->Glx;
            st->Gy = st->Ghy + st->Gly;
            st->Gz = st->Ghz + st->Glz;
        } else if (tid == 32) {
            deferred_tie();  // the previous step's near-tie flag
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

        // ---- 2. projected states (fp32 offsets (j + 1) * move), box test, goal-term offset,
        // static wells, per (action, sub-step)
        for (int q = tid; q < AW; q += kLookThreads) {
            const int ac = q / W, j = q - ac * W;
            const int hn = hna[ac];
            const float fj = (float)(j + 1);
            const float px = fmaf(fj, Dh[4 * hn], fj * Dh[4 * hn + 1]);
            const float py = fmaf(fj, Dh[4 * hn + 2], fj * Dh[4 * hn + 3]);
            const float pz = fmaf(fj, Dz2[2 * ac], fj * Dz2[2 * ac + 1]);
            ox[q] = px;
            oy[q] = py;
            oz[q] = pz;
            const float sx = shx + (slx + px), sy = shy + (sly + py), sz = shz + (slz + pz);
            const float mb = fminf(fminf(fminf(sx - box0, sy - box1), sz - box2), fminf(fminf(box3 - sx, box4 - sy), box5 - sz));
            int in;
            if (mb > kBoxBandL) in = 1;
            else if (mb < -kBoxBandL) in = 0;
            else in = look_box_exact(m, st->s, Dx[hn], Dy[hn], Dz[ac], j) ? 1 : 0;
            inb[q] = in;
            const float ex = st->Gx - px, ey = st->Gy - py, ez = st->Gz - pz;
            const float d = sqrtf(fmaf(ex, ex, fmaf(ey, ey, ez * ez)));
            const float num = fmaf(px, px, fmaf(py, py, pz * pz)) - 2.f * fmaf(st->Gx, px, fmaf(st->Gy, py, st->Gz * pz));
            const float den = d + st->ds;
            const float dd = den > 0.f ? num / den : 0.f;  // d(x_j) - d(s)
            rel[q] = dd * m.lg32;
            // static negative peaks (restricted volumes / terrain wells)
            float mbw = -INFINITY;
            unsigned long long sb = 0ull;
            for (int w = 0; w < m.n_static; ++w) {
                const float ux = px - stc[3 * w], uy = py - stc[3 * w + 1], uz = pz - stc[3 * w + 2];
                const float d2 = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
                const float R2 = m.st_R2[w];
                bool inw = d2 < R2;
                if (fabsf(d2 - R2) <= m.st_band[w]) inw = look_static_exact(m, w, st->s, Dx[hn], Dy[hn], Dz[ac], j);
                if (inw) {
                    const float l = fmaf(sqrtf(d2), m.st_lg[w], m.st_L[w]);
                    mbw = fmaxf(mbw, l);
                    if (m.combine) sb += look_sum_term(l, m.sum_ref);
                }
            }
            if (mbw > -INFINITY) atomicMax(&keys[q], float_key(mbw));
            if (sb) atomicAdd(&sums[q], sb);
        }
        __syncthreads();

        // ---- 3. plan wells: every (sub-step, slot) pair, warp-cooperative scoring
        const int npairs = W * S;
        const int64_t t_hi = a.tab.t_base + a.tab.T_win;
        for (int base = warp * 32; base < npairs; base += kLookThreads) {
            const int idx = base + lane;
            int j = 0, i = 0;
            unsigned wm = 0u;  // wells of this pair that can reach a projected state of sub-step j
            float p1x = 0.f, p1y = 0.f, p1z = 0.f, p2x = 0.f, p2y = 0.f, p2z = 0.f;
            if (idx < npairs) {
                j = idx / S;
                i = idx - j * S;
                const int64_t t1 = t + j + 1, t2 = t1 + 1;
                if (t1 >= a.tab.t_base && t1 < t_hi) {
                    int64_t r1 = row0 + j;  // rows of t + j + 1 and t + j + 2 (j < T_win)
                    r1 -= r1 >= a.tab.T_win ? a.tab.T_win : 0;
                    const size_t o1 = (size_t)r1 * a.tab.S_pad + i;
                    p1x = a.tab.X[o1];
                    p1y = a.tab.Y[o1];
                    p1z = a.tab.Z[o1];
                    p2x = __int_as_float(0x7fc00000);
                    if (t2 < t_hi) {
                        int64_t r2 = r1 + 1;
                        r2 -= r2 >= a.tab.T_win ? a.tab.T_win : 0;
                        const size_t o2 = (size_t)r2 * a.tab.S_pad + i;
                        p2x = a.tab.X[o2];
                        p2y = a.tab.Y[o2];
                        p2z = a.tab.Z[o2];
                    }
                    if (p1x == p1x) {
                        const float qx = (p1x - shx) - slx, qy = (p1y - shy) - sly, qz = (p1z - shz) - slz;
                        float vx = 0.f, vy = 0.f, vz = 0.f;
                        if (p2x == p2x) {
                            vx = (p2x - p1x) * inv_dt;
                            vy = (p2y - p1y) * inv_dt;
                            vz = (p2z - p1z) * inv_dt;
                        }
                        wm = well_mask(qx, qy, qz, vx, vy, vz, (float)(j + 1) * lstep);
                    }
                }
            }
            unsigned mask = __ballot_sync(kFullMask, wm != 0u);
            while (mask) {
                const int b = __ffs(mask) - 1;
                mask &= mask - 1;
                const int jb = __shfl_sync(kFullMask, j, b);
                const unsigned bwm = __shfl_sync(kFullMask, wm, b);
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
                        if (!((bwm >> w) & 1u)) continue;
                        const float tau = m.w_tau[w];
                        const float ux = px - fmaf(tau, vx, qx), uy = py - fmaf(tau, vy, qy), uz = pz - fmaf(tau, vz, qz);
                        const float d2 = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
                        const float R2 = m.w_R2[w];
                        bool in = d2 < R2;
                        if (fabsf(d2 - R2) <= m.w_band[w]) {
                            const int hn = hna[lane];
                            in = look_well_exact(m, w, st->s, Dx[hn], Dy[hn], Dz[lane], jb, b1x, b1y, b1z, b2x, b2y,
                                                 b2z, has2);
                        }
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
                unsigned wm = 0u;
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
                        wm = well_mask(qx, qy, qz, (float)mvx, (float)mvy, (float)mvz, (float)(j + 1) * lstep);
                    }
                }
                unsigned mask = __ballot_sync(kFullMask, wm != 0u);
                while (mask) {
                    const int b = __ffs(mask) - 1;
                    mask &= mask - 1;
                    const int jb = __shfl_sync(kFullMask, j, b);
                    const unsigned bwm = __shfl_sync(kFullMask, wm, b);
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
                            if (!((bwm >> w) & 1u)) continue;
                            const float tau = m.w_tau[w];
                            const float ux = px - fmaf(tau, vx, qx), uy = py - fmaf(tau, vy, qy),
                                        uz = pz - fmaf(tau, vz, qz);
                            const float d2 = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
                            const float R2 = m.w_R2[w];
                            bool in = d2 < R2;
                            if (fabsf(d2 - R2) <= m.w_band[w]) {
                                const int hn = hna[lane];
                                in = look_member_exact(m, w, st->s, Dx[hn], Dy[hn], Dz[lane], jb, bsx, bsy, bsz, bvx,
                                                       bvy, bvz);
                            }
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
                const float sx = shx + (slx + ox[q]), sy = shy + (sly + oy[q]), sz = shz + (slz + oz[q]);
                const float c32 = sz - terrain32(m, sx, sy);
                if (fabsf(c32 - (float)m.clearance) <= kClrBand + kTerrBand) {
                    const int ac = q / W, hn = hna[ac];
                    D = look_deck_exact(m, st->s, Dx[hn], Dy[hn], Dz[ac], q - ac * W);
                } else if (c32 < (float)m.clearance) {
                    D = (float)m.deck - c32;
                }
            }
            const float N = P + D;
            const float ln = N > 0.f ? log2f(N) : -INFINITY;
            lN[q] = ln;
            // the value g - N at x_j relative to 2^n0 (g = 2^(phi + rel), N = 2^(ln - n0))
            const float lg = st->phi + rel[q];
            int sg;
            float lv, lsc;
            bool vabs = false;
            if (ln == -INFINITY) {
                sg = 1;
                lv = lg;
                lsc = lg;
            } else {
                const float lnr = ln - (float)st->n0;
                const float x = lnr - lg;  // log2 (N / g)
                lsc = fmaxf(lg, lnr);
                if (x < -30.f) {
                    sg = 1;
                    lv = lg;
                } else if (x > 30.f) {
                    sg = -1;
                    lv = ln;
                    vabs = true;
                } else {
                    const float rr = exp2f(x);
                    if (rr < 1.f) {
                        sg = 1;
                        lv = lg + log2f(1.f - rr);
                    } else if (rr > 1.f) {
                        sg = -1;
                        lv = lg + log2f(rr - 1.f);
                    } else {
                        sg = 0;
                        lv = 0.f;
                    }
                }
            }
            vsg[q] = (sg + 1) | (vabs ? 4 : 0);
            vlv[q] = lv;
            vlr[q] = vabs ? lv - (float)st->n0 : lv;
            vls[q] = lsc;
        }
        __syncthreads();

        // ---- 4. per action: the largest value over its projected states inside the box.
        // Values are held relative to 2^n0 (n0: integer part of log2 of the goal term at s):
        // g = 2^(phi + rel), N = 2^(lN - n0); g - N as (sign, log2 |g - N|), which keeps the
        // goal term's resolution when N at another sub-step is larger by hundreds of binary
        // orders. Only the winner per action is turned into an absolute FP64 log2.
        if (tid < A) {
            const int q0 = tid * W;
            int bq = -1, bs = -2;
            float br = 0.f;
            for (int j = 0; j < W; ++j) {
                const int q = q0 + j;
                if (j > 0 && !inb[q]) continue;
                const int sg = (vsg[q] & 3) - 1;
                const float lr = vlr[q];
                bool better;
                if (bs == -2) better = true;
                else if (sg != bs) better = sg > bs;
                else better = sg > 0 ? lr > br : (sg < 0 ? lr < br : false);
                if (better) {
                    bq = q;
                    bs = sg;
                    br = lr;
                }
            }
            const bool valid = inb[q0] != 0;
            const bool babs = (vsg[bq] & 4) != 0;
            const double Lk = babs ? (double)vlv[bq] : __dadd_rn((double)st->n0, (double)vlv[bq]);
            sga[tid] = valid ? bs : -2;
            Lka[tid] = Lk;
            Lqa[tid] = __dadd_rn((double)st->n0, (double)vls[bq]);
            Ksa[tid] = valid ? look_key(bs, Lk) : 0ull;
        }
        __syncthreads();

        // ---- 5. argmax, near-tie record, advance (warp 0)
        if (warp == 0) {
            const unsigned long long kq = lane < A ? Ksa[lane] : 0ull;
            unsigned long long mx = kq;
            for (int o = 16; o; o >>= 1) {
                const unsigned long long y = __shfl_xor_sync(kFullMask, mx, o);
                mx = y > mx ? y : mx;
            }
            const unsigned bm = __ballot_sync(kFullMask, lane < A && kq == mx && mx != 0ull);
            const int a1 = bm ? __ffs(bm) - 1 : -1;
            unsigned long long k2 = (lane < A && lane != a1) ? kq : 0ull;
            for (int o = 16; o; o >>= 1) {
                const unsigned long long y = __shfl_xor_sync(kFullMask, k2, o);
                k2 = y > k2 ? y : k2;
            }
            const unsigned b2 = __ballot_sync(kFullMask, lane < A && lane != a1 && kq == k2 && k2 != 0ull);
            const int a2 = b2 ? __ffs(b2) - 1 : -1;
            if (a.trace && lane < A) {
                const int sgl = sga[lane];
                q_trace[(size_t)k * A + lane] = sgl == -2 ? -INFINITY : (sgl == 0 ? 0.0 : (double)sgl * exp2(Lka[lane]));
            }
            if (lane == 0) {
                st->tie_k = k;  // tested during the next step (deferred_tie)
                st->tie_a1 = a1;
                st->tie_a2 = a2;
                if (a1 >= 0 && a2 >= 0) {
                    st->tie_s1 = sga[a1];
                    st->tie_s2 = sga[a2];
                    st->tie_L1 = Lka[a1];
                    st->tie_L2 = Lka[a2];
                    st->tie_T1 = Lqa[a1];
                    st->tie_T2 = Lqa[a2];
                }
                if (a1 < 0) {
                    st->status = FMDP_REJ_NO_ACTION;
                    st->done = 1;
                } else {
                    const int hn = hna[a1];
                    // exact advance (FP64, the oracle's x_1) and its double-float copies
                    st->prev[0] = st->s[0];
                    st->prev[1] = st->s[1];
                    st->prev[2] = st->s[2];
                    st->s[0] = __dadd_rn(st->s[0], Dx[hn]);
                    st->s[1] = __dadd_rn(st->s[1], Dy[hn]);
                    st->s[2] = __dadd_rn(st->s[2], Dz[a1]);
                    lk_df_add(st->shx, st->slx, Dh[4 * hn], Dh[4 * hn + 1]);
                    lk_df_add(st->shy, st->sly, Dh[4 * hn + 2], Dh[4 * hn + 3]);
                    lk_df_add(st->shz, st->slz, Dz2[2 * a1], Dz2[2 * a1 + 1]);
                    lk_df_add(st->Ghx, st->Glx, -Dh[4 * hn], -Dh[4 * hn + 1]);
                    lk_df_add(st->Ghy, st->Gly, -Dh[4 * hn + 2], -Dh[4 * hn + 3]);
                    lk_df_add(st->Ghz, st->Glz, -Dz2[2 * a1], -Dz2[2 * a1 + 1]);
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
                    st->row0 = st->row0 + 1 == a.tab.T_win ? 0 : st->row0 + 1;
                    const float gx = st->Ghx + st->Glx, gy = st->Ghy + st->Gly, gz = st->Ghz + st->Glz;
                    const float gd = sqrtf(gx * gx + gy * gy + gz * gz);
                    bool cap = false;
                    if (gd < stepf + kCapBandL) cap = look_capture_exact(st->s, req, st->cap2);
                    if (cap) {
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
        deferred_tie();
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
