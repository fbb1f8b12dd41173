// Persistent FastMDP rollout kernel (sm_103a).
//
// One thread-block cluster plans one request from departure to capture, horizon or
// dead end without returning to the host (the paper's CPU loop of Fig. 3 runs nine
// kernels and a device-to-host copy per step; here the whole loop is one launch).
//
// Roles inside each CTA (the CTA owns a contiguous partition of the plan-table slots):
//   warp 0      control: per-action work that does not depend on other plans (box test,
//               goal term, terrain clearance, static wells; Alg. 1, Alg. 4, Alg. 6) while
//               the other warps scan, then the exchange, argmax and state advance;
//   warps 1..   scanners: stride over the partition's slots of slice t+1 (wells) and t+2
//               (plan velocity); a slot whose wells cannot reach any successor is culled
//               with one distance test, and for each near slot the whole warp evaluates
//               the five wells of Table 3 with lane a scoring action a (Alg. 5-7);
//   warp 1 l.0  producer: TMA bulk copies of upcoming slices into an 8-deep ring (the
//               table does not depend on the aircraft, so it runs steps ahead).
// Per-action maxima of log2(|r| gamma^d) are combined within the CTA by shared-memory
// atomics and across the cluster by DSMEM pushes (st.async + mbarrier), so no cluster-wide
// barrier is needed per step.
//
// Numerics. GB300 executes FP64 at 1/64 of the FP32 rate with ~63-cycle latency, so the
// serial per-step chain is FP32: the state is carried as an exact FP64 triple (advanced by
// three rounded adds, exactly as the method defines it) plus a double-float copy for
// plan offsets; action values are compared through a (sign, log2|Q|) key. Every threshold
// decision (box edge, well edge, clearance, capture) whose FP32 estimate lies within a
// thin band of the threshold is re-evaluated in FP64 in the method's operation order, so
// decisions match an FP64 evaluation bit for bit.
#include <cfloat>
#include <climits>

#include "fmdp_internal.cuh"
#include "sep_pair.cuh"

namespace fmdp {

namespace {

constexpr int kRingDepth = 8;  // maximum ring depth (slices in flight + in use)
constexpr unsigned kFull = 0xffffffffu;
constexpr float kBoxBand = 0.01f;  // metres: FP32 box test margin before an exact check
constexpr float kCapBand = 0.5f;   // metres: FP32 capture margin before an exact check

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: gives up after ~2^31 SM cycles (about a second) and reports false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > (1ll << 31)) return false;
    }
    return true;
}
__device__ __forceinline__ void tma_bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// named CTA barrier over `threads` threads (a multiple of 32, whole warps)
__device__ __forceinline__ void named_barrier(int id, int threads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t dsmem_addr(uint32_t local, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
    return r;
}
__device__ __forceinline__ int ld_cluster_s32(uint32_t addr) {
    int v;
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ int ld_acquire_gpu(const int32_t* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void st_async_s32(uint32_t addr, int v, uint32_t bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.s32 [%0], %1, [%2];" ::"r"(addr), "r"(v),
                 "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void st_async_u64(uint32_t addr, unsigned long long v, uint32_t bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];" ::"r"(addr), "l"(v),
                 "r"(bar)
                 : "memory");
}

// ---- double-float (fp32 pair) arithmetic: exact sums of fp32 numbers
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
// (hi, lo) += (dh, dl)
__device__ __forceinline__ void df_add(float& hi, float& lo, float dh, float dl) {
    float s, e;
    two_sum(hi, dh, s, e);
    e = __fadd_rn(e, __fadd_rn(lo, dl));
    fast_two_sum(s, e, hi, lo);
}
__device__ __forceinline__ float approx_sqrt(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }

struct StepState {
    float wlim2[kMaxWells];  // per well: (R + largest successor offset + 1 m)^2, the reach test
    // the well constants the scanners read every step, copied from the kernel parameters
    // (parameter-space reads with a run-time index wait on the constant cache)
    float w_tau[kMaxWells], w_R2[kMaxWells], w_band[kMaxWells], w_lg[kMaxWells], w_L[kMaxWells];
    double s[3];       // exact state (FP64)
    double cap2;       // (speed * dt)^2
    double step;       // speed * dt
    float s_hi[3], s_lo[3];  // double-float copy of s
    float G_hi[3], G_lo[3];  // goal - s, double-float
    float phi;         // log2 of the goal term at s minus n0, in [0, 1)
    int n0;            // integer part of log2 of the goal term at s
    int h;             // heading index (15-degree units from the initial bearing)
    int done;
    int status;
    int n_points;
    int near_ties;
    int steps;
    int ent_valid[kRingDepth];
    int abort_flag[2];  // staging of step k timed out (indexed by k & 1)
    int last_best[2];   // action chosen at step k (99: none), by k & 1
};

// Shared-memory carve-up (identical on host and device).
// Indexed mode: what one staging buffer holds. The first n_s of the `total` items are in
// shared memory; the rest are read from the index in global memory through the ranges.
constexpr int kMaxRanges = 8;
struct IdxMeta {
    int total, n_s, nr;
    int pub;  // pipelined mode: admissions published when the extra list's length was read
    long long row_off;  // first float4 of the row's items
    int beg[kMaxRanges], cnt[kMaxRanges];
};
constexpr int kIBufs = 3;  // staging buffers: the step being scanned and the next two

struct Layout {
    size_t ring, ibuf, imeta, bars, xbar, st, tabs, keys, sums, xkeys, xsums, xab, stat, aux, misc, total;
};
// chunk, depth: full-scan slice ring (chunk = 0 in indexed mode); icap: indexed staging
// buffer capacity in items (0 in full-scan mode)
__host__ __device__ inline Layout make_layout(int chunk, int depth, int icap) {
    Layout L;
    size_t o = 0;
    auto al = [&](size_t a) { o = (o + a - 1) & ~(a - 1); };
    L.ring = o;
    o += (size_t)depth * 3 * chunk * sizeof(float);
    al(128);
    L.ibuf = o;  // [kIBufs][icap] items of two float4
    o += icap > 0 ? (size_t)kIBufs * icap * 2 * sizeof(float4) : 0;
    al(16);
    L.imeta = o;
    o += icap > 0 ? kIBufs * sizeof(IdxMeta) : 0;
    al(16);
    L.bars = o;
    o += kRingDepth * sizeof(uint64_t);
    L.xbar = o;
    o += 2 * sizeof(uint64_t);
    al(16);
    L.st = o;
    o += sizeof(StepState);
    al(16);
    L.tabs = o;  // Dx[24] Dy[24] Dz[32] doubles; dxh dxl dyh dyl [24] dzh dzl [32] floats
    o += (24 + 24 + 32) * sizeof(double) + (4 * 24 + 2 * 32) * sizeof(float);
    al(16);
    L.keys = o;
    o += kMaxActions * sizeof(int);
    al(16);
    L.sums = o;
    o += kMaxActions * sizeof(unsigned long long);
    L.xkeys = o;
    o += 2 * kMaxCluster * kMaxActions * sizeof(int);
    al(16);
    L.xsums = o;
    o += 2 * kMaxCluster * kMaxActions * sizeof(unsigned long long);
    L.xab = o;
    o += 2 * kMaxCluster * sizeof(int);
    al(16);
    L.stat = o;  // static-well centres as double-float: hi[64][3], lo[64][3]
    o += 2 * kMaxStatic * 3 * sizeof(float);
    al(16);
    L.aux = o;   // valid, Delta, deck, goal term; key, class, log2|Q|, log2 scale by step parity
    o += 12 * kMaxActions * sizeof(int);
    L.misc = o;  // work-queue slot of the persistent batch mode; pipelined mode: [0..3] the
                 // item taken, [4..6] the tail check's first conflict and terrain sample and
                 // the admissions published before it read the index, [8..9] the item's window
    o += 48;
    L.total = (o + 127) & ~size_t(127);
    return L;
}


// Exact (FP64, method order) well-edge decision for a plan well.
__device__ __noinline__ bool well_inside_exact(const Model& m, const StepState* st, double Dx, double Dy,
                                               double Dz, float p1x, float p1y, float p1z, float p2x, float p2y,
                                               float p2z, bool has2, int w) {
    const double x = __dadd_rn(st->s[0], Dx), y = __dadd_rn(st->s[1], Dy), z = __dadd_rn(st->s[2], Dz);
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

__device__ __noinline__ bool static_inside_exact(const Model& m, const StepState* st, double Dx, double Dy,
                                                 double Dz, int w) {
    const double x = __dadd_rn(st->s[0], Dx), y = __dadd_rn(st->s[1], Dy), z = __dadd_rn(st->s[2], Dz);
    const double* c = m.statics + 6 * w;
    return norm3_64(__dsub_rn(x, c[0]), __dsub_rn(y, c[1]), __dsub_rn(z, c[2])) < c[3];
}

__device__ __noinline__ bool box_inside_exact(const Model& m, const StepState* st, double Dx, double Dy, double Dz) {
    const double x = __dadd_rn(st->s[0], Dx), y = __dadd_rn(st->s[1], Dy), z = __dadd_rn(st->s[2], Dz);
    return x >= m.box[0] && x <= m.box[3] && y >= m.box[1] && y <= m.box[4] && z >= m.box[2] && z <= m.box[5];
}

__device__ __noinline__ float deck_exact(const Model& m, const StepState* st, double Dx, double Dy, double Dz) {
    const double x = __dadd_rn(st->s[0], Dx), y = __dadd_rn(st->s[1], Dy), z = __dadd_rn(st->s[2], Dz);
    const double c = __dsub_rn(z, terrain64(m, x, y));
    return c < m.clearance ? (float)__dsub_rn(m.deck, c) : 0.f;
}

__device__ __noinline__ bool capture_exact(const StepState* st, const fmdp_request& req) {
    const double ex = __dsub_rn(req.gx, st->s[0]), ey = __dsub_rn(req.gy, st->s[1]), ez = __dsub_rn(req.gz, st->s[2]);
    return __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez)) <= st->cap2;
}

__device__ __noinline__ bool capture_exact_at(double x, double y, double z, const fmdp_request& req, double cap2) {
    const double ex = __dsub_rn(req.gx, x), ey = __dsub_rn(req.gy, y), ez = __dsub_rn(req.gz, z);
    return __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez)) <= cap2;
}

// log2 of the goal term, log2|r| + |G| log2(gamma), from a double-float goal vector G, split
// into an integer n0 and a fraction phi in [0, 1) (fp32 pair arithmetic, ~1e-12 relative).
__device__ __forceinline__ void goal_log_split(float Ghx, float Ghy, float Ghz, float Glx, float Gly, float Glz,
                                               float lg_hi, float lg_lo, float l2r_hi, float l2r_lo, int& n0,
                                               float& phi) {
    const float p0 = Ghx * Ghx, p1 = Ghy * Ghy, p2 = Ghz * Ghz;
    const float e0 = fmaf(Ghx, Ghx, -p0), e1 = fmaf(Ghy, Ghy, -p1), e2 = fmaf(Ghz, Ghz, -p2);
    float s1, t1, s2, t2;
    two_sum(p0, p1, s1, t1);
    two_sum(s1, p2, s2, t2);
    const float lo = t1 + t2 + e0 + e1 + e2 + 2.f * (Ghx * Glx + Ghy * Gly + Ghz * Glz);
    float Sh, Sl;
    fast_two_sum(s2, lo, Sh, Sl);
    const float rt = approx_sqrt(Sh);
    const float rr = fmaf(-rt, rt, Sh);
    const float rl = rt > 0.f ? (rr + Sl) * (0.5f * rsqrtf(Sh)) : 0.f;
    const float p = rt * lg_hi;
    const float pe = fmaf(rt, lg_hi, -p);
    const float lo2 = pe + rt * lg_lo + rl * lg_hi;
    float Lh, Le;
    two_sum(p, l2r_hi, Lh, Le);
    Le = Le + (lo2 + l2r_lo);
    float LH, LL;
    fast_two_sum(Lh, Le, LH, LL);
    float fl = floorf(LH);
    float fr = (LH - fl) + LL;
    if (fr >= 1.f) { fr -= 1.f; fl += 1.f; }
    if (fr < 0.f) { fr += 1.f; fl -= 1.f; }
    n0 = (int)fl;
    phi = fr;
}

// Clearance penalty decided in FP64 at an exact successor (band around the threshold).
// Static negative peaks (restricted volumes / terrain wells) for one action.
__device__ __noinline__ void fold_statics(const Model& m, const StepState* st, const float* sch, const float* scl,
                                          float shx, float shy, float shz, float slx, float sly, float slz,
                                          float dxa, float dya, float dza, double Dxh, double Dyh, double Dza,
                                          float& mloc, unsigned long long& sloc) {
    for (int w = 0; w < m.n_static; ++w) {
        const float qx = (sch[3 * w] - shx) + (scl[3 * w] - slx);
        const float qy = (sch[3 * w + 1] - shy) + (scl[3 * w + 1] - sly);
        const float qz = (sch[3 * w + 2] - shz) + (scl[3 * w + 2] - slz);
        const float ex = dxa - qx, ey = dya - qy, ez = dza - qz;
        const float d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
        const float R2 = m.st_R2[w], bw = m.st_band[w];
        if (d2 < R2 + bw) {
            const bool inside = d2 < R2 - bw ? true : static_inside_exact(m, st, Dxh, Dyh, Dza, w);
            if (inside) {
                const float l = fmaf(approx_sqrt(d2), m.st_lg[w], m.st_L[w]);
                mloc = fmaxf(mloc, l);
                if (m.combine) {
                    const float t = exp2f(l - m.sum_ref) * kSumUnits;
                    sloc += (unsigned long long)__float2ull_rn(t);
                }
            }
        }
    }
}

// FP64 action value for the trace output only (never used for the decision).
__device__ __noinline__ double trace_q(const Model& m, bool has_goal, int n0, float phi, float Dl, float Lp,
                                       unsigned long long ssum, float Vd) {
    double g = 0.0;
    if (has_goal) g = exp2((double)n0 + (double)phi + (double)Dl * m.lg64);
    double P = 0.0;
    if (m.combine) P = (double)ssum * m.sum_scale;
    else if (Lp > -INFINITY) P = exp2((double)Lp);
    return __dsub_rn(__dsub_rn(g, P), (double)Vd);
}

// Diagnostic near-tie flag of the two best actions:
// (Q1 - Q2) < 1e-4 * max(|Q1|, |Q2|, T1, T2), evaluated on log-magnitudes.
__device__ __noinline__ bool near_tie(int c1, int c2, float la1, float la2, float lt1, float lt2) {
    const float lsc = fmaxf(fmaxf(la1, la2), fmaxf(lt1, lt2));
    const float hi = fmaxf(la1, la2), lo = fminf(la1, la2);
    float lgap;
    if (c1 == c2 && c1 != 1) lgap = hi + __log2f(fmaxf(1.f - exp2f(lo - hi), 1e-30f));
    else lgap = hi + __log2f(1.f + exp2f(lo - hi));
    return lgap < lsc - 13.287712f;  // log2(1e-4)
}

// Near-tie flag of the previous step from the keys the control warp stored (warp-wide call).
__device__ __forceinline__ void deferred_tie(StepState* st, const uint32_t* qkey_b, const int* cls_b,
                                             const float* la_b, const float* lt_b, int par, int lane,
                                             uint8_t* trace_slot) {
    const int b = st->last_best[par];
    if (b >= 99) return;
    const uint32_t* qkey_s = qkey_b + par * kMaxActions;
    const int* cls_s = cls_b + par * kMaxActions;
    const float* la_s = la_b + par * kMaxActions;
    const float* lt_s = lt_b + par * kMaxActions;
    const uint32_t qk = qkey_s[lane];
    const uint32_t k2nd = __reduce_max_sync(kFull, lane == b ? 0u : qk);
    const unsigned sm2 = __ballot_sync(kFull, qk == k2nd && k2nd != 0u && lane != b);
    if (lane == 0) {
        bool tie = false;
        if (sm2) {
            const int sec = __ffs(sm2) - 1;
            tie = near_tie(cls_s[b], cls_s[sec], la_s[b], la_s[sec], lt_s[b], lt_s[sec]);
        }
        if (tie) st->near_ties += 1;
        if (trace_slot) *trace_slot = tie ? 1 : 0;
    }
}

// Monotone 32-bit argmax key: valid actions > 0; Q > 0 above Q = 0 above Q < 0; within a
// class ordered by k2 (one float bit dropped, 2.4e-7 of log2|Q|).
__device__ __forceinline__ uint32_t action_key(int cls, float k2) {
    const uint32_t u = ((uint32_t)float_key(k2) ^ 0x80000000u) >> 1;
    if (cls == 2) return 0x80000000u | u;
    if (cls == 1) return 0x80000000u;
    return u;
}

__device__ __forceinline__ unsigned long long sum_term(float l, float ref) {
    const float t = exp2f(l - ref) * kSumUnits;  // fixed point, 2^-kSumBits of the largest |r|
    return (unsigned long long)__float2ull_rn(t);
}

// Scores one well of a plan for this lane's action: max-fold of log2(|r| gamma^d).
__device__ __forceinline__ void fold_well(const StepState* st, int w, float qx, float qy, float qz, float vx,
                                          float vy, float vz, float dxa, float dya, float dza, float& mloc,
                                          unsigned long long& sloc, bool& band, bool use_sum, float sum_ref) {
    const float tau = st->w_tau[w];
    const float ex = dxa - fmaf(tau, vx, qx);
    const float ey = dya - fmaf(tau, vy, qy);
    const float ez = dza - fmaf(tau, vz, qz);
    const float d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
    const float R2 = st->w_R2[w], bw = st->w_band[w];
    if (d2 < R2 + bw) {
        if (d2 < R2 - bw) {
            const float l = fmaf(approx_sqrt(d2), st->w_lg[w], st->w_L[w]);
            mloc = fmaxf(mloc, l);
            if (use_sum) sloc += sum_term(l, sum_ref);
        } else {
            band = true;
        }
    }
}

}  // namespace

// Plans request r with this CTA (and its cluster peers). Every thread of the cluster calls
// it; all shared memory it uses is re-initialised, so a CTA can plan requests back to back.
// k0 > 0 (pipelined mode): the plan keeps its first k0 steps and resumes from its state at
// step k0, as stored by the run that planned them. tbase: the first step of the table window
// the plan reads (the launch's, or in pipelined mode the one its item was dispatched with). IDX: indexed mode (one CTA, no cluster),
// compiled apart from the full-scan mode so that each step's code stays small; GEN: the
// general instance, with the uncommon features (the per-phase clock stamps of
// fmdp_set_profiling(2), the trace of fmdp_rollout_trace, the SUM combination, static wells); without it the
// step's code holds only the common configuration (the stamps' code alone lengthens a step by
// about 3 %).
template <bool IDX, bool GEN>
__device__ __forceinline__ void plan_request(const RolloutArgs& a, const int r, unsigned char* smem,
                                             const int64_t tbase, const int k0 = 0) {
    const Model& m = a.m;
    const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31, warp = tid >> 5, NW = NT >> 5;
    const int cs = IDX ? 1 : a.cs;
    const uint32_t rank = cs > 1 ? cluster_rank() : 0u;
    const fmdp_request req = a.reqs[r];
    const int A = m.A;
    const int chunk = a.chunk;
    const int c_begin = (int)rank * chunk;
    const int c_len = max(0, min(chunk, a.S_scan - c_begin));
    const int depth = a.ring;                    // 4 or 8 slices
    const int dshift = depth == 8 ? 3 : 2;
    constexpr bool indexed = IDX;
    const int icap = a.icap;
    const Layout L = make_layout(chunk, depth, indexed ? icap : 0);
    float4* ibuf = reinterpret_cast<float4*>(smem + L.ibuf);
    IdxMeta* imeta = reinterpret_cast<IdxMeta*>(smem + L.imeta);

    float* ring = reinterpret_cast<float*>(smem + L.ring);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bars);
    uint64_t* xbar = reinterpret_cast<uint64_t*>(smem + L.xbar);
    StepState* st = reinterpret_cast<StepState*>(smem + L.st);
    double* Dx = reinterpret_cast<double*>(smem + L.tabs);
    double* Dy = Dx + 24;
    double* Dz = Dy + 24;
    float* dxh = reinterpret_cast<float*>(Dz + 32);
    float* dxl = dxh + 24;
    float* dyh = dxl + 24;
    float* dyl = dyh + 24;
    float* dzh = dyl + 24;
    float* dzl = dzh + 32;
    int* keys = reinterpret_cast<int*>(smem + L.keys);
    unsigned long long* sums = reinterpret_cast<unsigned long long*>(smem + L.sums);
    int* xkeys = reinterpret_cast<int*>(smem + L.xkeys);                                 // [2][16][32]
    unsigned long long* xsums = reinterpret_cast<unsigned long long*>(smem + L.xsums);   // [2][16][32]
    int* xab = reinterpret_cast<int*>(smem + L.xab);                                     // [2][16]
    float* sch = reinterpret_cast<float*>(smem + L.stat);
    float* scl = sch + 3 * kMaxStatic;
    int* valid_s = reinterpret_cast<int*>(smem + L.aux);
    float* Dl_s = reinterpret_cast<float*>(valid_s + kMaxActions);
    float* Vd_s = Dl_s + kMaxActions;
    float* gh_s = Vd_s + kMaxActions;  // goal term at the successor over 2^n0
    // keys of a step for the deferred near-tie flag, [2][32] by step parity
    uint32_t* qkey_s = reinterpret_cast<uint32_t*>(gh_s + kMaxActions);
    int* cls_s = reinterpret_cast<int*>(qkey_s + 2 * kMaxActions);
    float* la_s = reinterpret_cast<float*>(cls_s + 2 * kMaxActions);
    float* lt_s = la_s + 2 * kMaxActions;

    const bool lead = (rank == 0);
    float* traj = a.traj + (size_t)r * a.cap * 3;
    uint8_t* acts = a.acts + (size_t)r * a.cap;
    const int64_t t_lo = tbase, t_hi = tbase + a.tab.T_win;  // the table window this plan reads
    const int64_t last_j = (int64_t)req.horizon + 1;
    const int KEY_NONE = float_key(-INFINITY);
    // FCFS ordinal of this request: tentative plans of later requests are not part of its table
    const int32_t my_ord = a.pipe.on ? a.pipe.ord0 + r : INT_MAX;

    // ---------------------------------------------------------------- prologue
    if (tid < kHeadings) {
        const double dx = __dsub_rn(req.gx, req.ox), dy = __dsub_rn(req.gy, req.oy);
        const double Lh = __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
        double c0 = 1.0, s0 = 0.0;
        if (Lh > 0.0) { c0 = __ddiv_rn(dx, Lh); s0 = __ddiv_rn(dy, Lh); }
        double ck, sk;
        unit15(tid, ck, sk);
        const double C = __dsub_rn(__dmul_rn(c0, ck), __dmul_rn(s0, sk));
        const double S = __dadd_rn(__dmul_rn(s0, ck), __dmul_rn(c0, sk));
        const double step = __dmul_rn(req.speed_mps, m.dt);
        const double X = __dmul_rn(step, C), Y = __dmul_rn(step, S);
        Dx[tid] = X;
        Dy[tid] = Y;
        dxh[tid] = (float)X;
        dxl[tid] = (float)__dsub_rn(X, (double)dxh[tid]);
        dyh[tid] = (float)Y;
        dyl[tid] = (float)__dsub_rn(Y, (double)dyh[tid]);
    }
    if (tid < kMaxActions) {
        const double dz = tid < A ? __dmul_rn(m.climb[tid], m.dt) : 0.0;
        Dz[tid] = dz;
        dzh[tid] = (float)dz;
        dzl[tid] = (float)__dsub_rn(dz, (double)dzh[tid]);
        keys[tid] = KEY_NONE;
        sums[tid] = 0ull;
    }
    for (int w = tid; w < m.n_static; w += NT) {
        const double* c = m.statics + 6 * w;
        for (int q = 0; q < 3; ++q) {
            sch[3 * w + q] = (float)c[q];
            scl[3 * w + q] = (float)__dsub_rn(c[q], (double)sch[3 * w + q]);
        }
    }
    if (tid == 0) {
        for (int e = 0; e < kRingDepth; ++e) mbar_init(&bars[e], 1);
        mbar_init(&xbar[0], 1);
        mbar_init(&xbar[1], 1);
        mbar_fence_init();
        const double step = __dmul_rn(req.speed_mps, m.dt);
        st->step = step;
        st->cap2 = __dmul_rn(step, step);
        {
            // a successor lies within step + max |climb| dt of the state; a well whose centre
            // is farther than R + that + 1 m misses every successor by more than 1 m
            float dzm = 0.f;
            for (int q = 0; q < A; ++q) dzm = fmaxf(dzm, fabsf((float)__dmul_rn(m.climb[q], m.dt)));
            for (int w = 0; w < m.n_wells; ++w) {
                const float lim = sqrtf(m.w_R2[w]) + (float)step + dzm + 1.f;
                st->wlim2[w] = lim * lim;
                st->w_tau[w] = m.w_tau[w];
                st->w_R2[w] = m.w_R2[w];
                st->w_band[w] = m.w_band[w];
                st->w_lg[w] = m.w_lg[w];
                st->w_L[w] = m.w_L[w];
            }
        }
        const double s0[3] = {req.ox, req.oy, req.oz};
        const double g0[3] = {req.gx, req.gy, req.gz};
        for (int q = 0; q < 3; ++q) {
            st->s[q] = s0[q];
            st->s_hi[q] = (float)s0[q];
            st->s_lo[q] = (float)__dsub_rn(s0[q], (double)st->s_hi[q]);
            const double G = __dsub_rn(g0[q], s0[q]);
            st->G_hi[q] = (float)G;
            st->G_lo[q] = (float)__dsub_rn(G, (double)st->G_hi[q]);
        }
        st->h = 0;
        const bool captured = capture_exact(st, req);
        st->done = captured || req.horizon <= 0;
        st->status = captured ? kStatusCaptured : FMDP_REJ_HORIZON;
        st->n_points = 1;
        st->near_ties = 0;
        st->steps = 0;
        if (k0 > 0) {
            // resume at step k0: the state as the step that reached it published it, and the
            // goal vector formed from its double-float copy exactly as a step forms it
            const size_t o = (size_t)r * a.cap + k0;
            for (int q = 0; q < 3; ++q) {
                st->s[q] = a.pipe.st_s[3 * o + q];
                st->s_hi[q] = a.pipe.st_df[6 * o + 2 * q];
                st->s_lo[q] = a.pipe.st_df[6 * o + 2 * q + 1];
                float gh = (float)g0[q];
                float gl = (float)__dsub_rn(g0[q], (double)gh);
                df_add(gh, gl, -st->s_hi[q], -st->s_lo[q]);
                st->G_hi[q] = gh;
                st->G_lo[q] = gl;
            }
            st->h = a.pipe.st_h[o];
            st->done = 0;  // the run that planned these steps went on from step k0
            st->status = FMDP_REJ_HORIZON;
            st->n_points = k0 + 1;
            st->steps = k0;
        }
        st->abort_flag[0] = st->abort_flag[1] = 0;
        st->last_best[0] = st->last_best[1] = 99;
        for (int e = 0; e < kRingDepth; ++e) st->ent_valid[e] = 0;
        if (lead) {
            traj[0] = (float)req.ox; traj[1] = (float)req.oy; traj[2] = (float)req.oz;
            if (a.trace && r == 0) {
                a.st_trace[0] = req.ox; a.st_trace[1] = req.oy; a.st_trace[2] = req.oz;
                a.hd_trace[0] = 0;
            }
        }
    }
    if (cs > 1) cluster_barrier(); else __syncthreads();  // mbarriers initialised cluster-wide
    if (k0 > 0) {  // near ties of the kept steps
        int nt = 0;
        for (int i = tid; i < k0; i += NT) nt += a.pipe.ties[(size_t)r * a.cap + i];
        if (nt) atomicAdd(&st->near_ties, nt);
    }

    // ---- producer state (thread 32: warp 1, lane 0)
    const bool producer = (tid == 32);
    int64_t issued = 0, waited = 0;
    int64_t next_row = 0;  // ring row of slice `issued + 1`
    auto entry_of = [&](int64_t j) { return (int)((j - 1) & (depth - 1)); };
    auto parity_of = [&](int64_t j) { return (uint32_t)(((j - 1) >> dshift) & 1); };
    auto issue_upto = [&](int64_t jmax) {
        for (int64_t j = issued + 1; j <= jmax && j <= last_j; ++j) {
            const int e = entry_of(j);
            const int64_t T = req.depart_step + j;
            const bool valid = c_len > 0 && T >= t_lo && T < t_hi;
            st->ent_valid[e] = valid ? 1 : 0;
            if (valid) {
                const size_t off = (size_t)next_row * a.tab.S_pad + c_begin;
                const uint32_t bytes = (uint32_t)c_len * 4u;
                float* dst = ring + (size_t)e * 3 * chunk;
                mbar_arrive_expect_tx(&bars[e], 3u * bytes);
                tma_bulk_load(dst, a.tab.X + off, bytes, &bars[e]);
                tma_bulk_load(dst + chunk, a.tab.Y + off, bytes, &bars[e]);
                tma_bulk_load(dst + 2 * chunk, a.tab.Z + off, bytes, &bars[e]);
            } else {
                mbar_arrive(&bars[e]);
            }
            issued = j;
            if (++next_row == a.tab.T_win) next_row = 0;
        }
    };
    // returns 1 on timeout
    auto wait_upto = [&](int64_t jneed) -> int {
        while (waited < jneed && waited < issued) {
            const int64_t j = waited + 1;
            if (!mbar_wait_bounded(&bars[entry_of(j)], parity_of(j))) {
                atomicExch(a.err, FMDP_ERR_TIMEOUT);
                for (int e = 0; e < depth; ++e) st->ent_valid[e] = 0;
                return 1;
            }
            waited = j;
        }
        return 0;
    };
    // ---- indexed mode: the producer warp (warp 2) keeps a software pipeline over the spatial
    // index. At step k (state s_k known) it reads the cell starts of the query for step k + 2
    // (one cell row per lane; prefetched into L2 one step earlier), copies those items into a
    // staging buffer, and waits for the items of step k + 1, copied one step earlier. It runs
    // beside the step rather than in it: the other warps' reduction barrier leaves it out,
    // and it joins them at the start of the next step. The query for step j, made from state s_a (a <= j - 1), covers every
    // cell within Rq + (j - 1 - a) * step of s_a horizontally: an item whose wells can reach a
    // successor of s_j lies within reach0 + tau_max * vmax of s_j (items outside the extra
    // list move no faster than vmax), and s_j lies within (j - a) steps of s_a.
    IdxMeta* imeta_all = imeta;
    // pipeline state, identical in every lane of warp 2 (lane 0 waits, the warp follows)
    uint32_t ifill[kIBufs] = {0u, 0u, 0u};
    bool ipend[kIBufs] = {false, false, false};
    const IndexView& iv = a.iv;
    const int64_t cst_row_len = (int64_t)iv.ncell + 1;
    auto row_of = [&](int64_t T) {
        int64_t row = T % a.tab.T_win;
        return row < 0 ? row + a.tab.T_win : row;
    };
    auto cell_of = [&](float v, float o, int n) {
        const float f = floorf((v - o) * iv.inv_cell);
        return f < 0.f ? 0 : (f > (float)(n - 1) ? n - 1 : (int)f);
    };
    auto excl_scan = [&](int v, int& total) {  // warp exclusive prefix sum
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
        }
        total = __shfl_sync(kFull, x, 31);
        return x - v;
    };
    // bounded wait (lane 0) on a buffer's mbarrier; returns 1 on timeout, in every lane
    auto wait_bar = [&](uint64_t* bar, uint32_t& fills, bool& pend) -> int {
        if (!pend) return 0;
        int bad = 0;
        if (lane == 0) {
            bad = mbar_wait_bounded(bar, fills & 1u) ? 0 : 1;
            if (bad) atomicExch(a.err, FMDP_ERR_TIMEOUT);
        }
        bad = __shfl_sync(kFull, bad, 0);
        ++fills;
        pend = false;
        return bad;
    };
    // lanes 0 .. kMaxRanges-1 each carry one item range (cnt 0: none): record them in
    // buffer b's metadata and copy the first icap items into shared memory
    auto issue_items = [&](int b, int my_beg, int my_cnt, long long row_off, int pub) {
        IdxMeta& M = imeta_all[b];
        int total;
        const int off = excl_scan(lane < kMaxRanges ? my_cnt : 0, total);
        const int n_s = min(total, icap);
        if (lane < kMaxRanges) {
            M.beg[lane] = my_beg;
            M.cnt[lane] = my_cnt;
        }
        if (lane == 0) {
            M.total = total;
            M.n_s = n_s;
            M.nr = kMaxRanges;
            M.row_off = row_off;
            M.pub = pub;
            if (a.items_ctr && total > 0) atomicAdd(a.items_ctr, (unsigned long long)total);
            if (n_s > 0) mbar_arrive_expect_tx(&bars[b], (uint32_t)n_s * 32u);
            else mbar_arrive(&bars[b]);
        }
        __syncwarp();
        const int take = lane < kMaxRanges ? max(0, min(my_cnt, n_s - off)) : 0;
        if (take > 0)
            tma_bulk_load(ibuf + ((size_t)b * icap + off) * 2, iv.items + row_off + (long long)my_beg * 2,
                          (uint32_t)take * 32u, &bars[b]);
        ipend[b] = true;
    };
    // cell box of a query; lanes 0 .. nrows-1 take one cell row each (whole: one range over
    // full cell rows, its two ends in lanes 0 and 1); the extra list is range kMaxRanges-1
    struct Box { int cx0, cx1, cy0, cy1, nrows, whole; };
    auto box_of = [&](float sx, float sy, float R) {
        Box q;
        q.cx0 = cell_of(sx - R, iv.x0, iv.ncx);
        q.cx1 = cell_of(sx + R, iv.x0, iv.ncx);
        q.cy0 = cell_of(sy - R, iv.y0, iv.ncy);
        q.cy1 = cell_of(sy + R, iv.y0, iv.ncy);
        q.nrows = q.cy1 - q.cy0 + 1;
        q.whole = q.nrows > kMaxRanges - 1;
        return q;
    };
    // read the cell starts of step T's query (ring row `row` = T mod T_win) and issue it
    auto issue_direct = [&](int b, int64_t T, int64_t row, float sx, float sy, float R) {
        int my_beg = 0, my_cnt = 0;
        long long row_off = 0;
        int pub = INT_MAX;  // pipelined mode: published admissions this query can see (all: none in the row)
        if (T >= t_lo && T < t_hi) {
            const int32_t* cs_row = iv.cstart + row * cst_row_len;
            const Box q = box_of(sx, sy, R);
            int e0 = 0, e1 = 0;
            // L2 loads (.cg): the index may change between launches of a persistent kernel
            // (rows rebuilt, extra lists published), so nothing of it is kept in L1
            if (!q.whole && lane < q.nrows) {
                e0 = __ldcg(cs_row + (q.cy0 + lane) * iv.ncx + q.cx0);
                e1 = __ldcg(cs_row + (q.cy0 + lane) * iv.ncx + q.cx1 + 1);
            } else if (q.whole && lane == 0) {
                e0 = __ldcg(cs_row + q.cy0 * iv.ncx);
                e1 = __ldcg(cs_row + (q.cy1 + 1) * iv.ncx);
            } else if (lane == kMaxRanges - 1) {
                // the count of published admissions first (acquire), then the extra list's
                // length: every admission counted is in the list this query copies
                if (a.pipe.pub_seq) pub = ld_acquire_gpu(a.pipe.pub_seq);
                e0 = __ldcg(cs_row + iv.ncell);
                e1 = e0 + __ldcg(iv.nextra + row);
            }
            my_beg = e0;
            my_cnt = max(0, e1 - e0);
            row_off = (long long)row * a.tab.S_pad * 2;
        }
        pub = __shfl_sync(kFull, pub, kMaxRanges - 1);
        issue_items(b, my_beg, my_cnt, row_off, pub);
    };
    // L2 prefetch of the cell starts a query of step T would read (issued one step early, so
    // that the next step's issue finds them in L2 instead of waiting on DRAM)
    auto prefetch_cells = [&](int64_t T, int64_t row, float sx, float sy, float R) {
        if (T < t_lo || T >= t_hi) return;
        const int32_t* cs_row = iv.cstart + row * cst_row_len;
        const Box q = box_of(sx, sy, R);
        const int32_t* p0 = nullptr;
        const int32_t* p1 = nullptr;
        if (!q.whole && lane < q.nrows) {
            p0 = cs_row + (q.cy0 + lane) * iv.ncx + q.cx0;
            p1 = cs_row + (q.cy0 + lane) * iv.ncx + q.cx1 + 1;
        } else if (q.whole && lane == 0) {
            p0 = cs_row + q.cy0 * iv.ncx;
            p1 = cs_row + (q.cy1 + 1) * iv.ncx;
        } else if (lane == kMaxRanges - 1) {
            p0 = cs_row + iv.ncell;
            p1 = iv.nextra + row;
        }
        if (p0) asm volatile("prefetch.global.L2 [%0];" ::"l"(p0));
        if (p1) asm volatile("prefetch.global.L2 [%0];" ::"l"(p1));
    };
    // all outstanding copies, before the buffers are reused or the CTA leaves
    auto drain = [&]() {
        for (int b = 0; b < kIBufs; ++b) wait_bar(&bars[b], ifill[b], ipend[b]);
    };

    bool stalled = false;
    if (producer && !indexed && !st->done) {
        const int64_t T1 = req.depart_step + 1;
        int64_t row = T1 % a.tab.T_win;
        if (row < 0) row += a.tab.T_win;
        next_row = row;
        issue_upto(depth);
        stalled = wait_upto(2) != 0;
        st->abort_flag[0] = stalled ? 1 : 0;
    }

    // ---- per-lane action constants (every warp: lane a scores action a)
    const int my_dh = lane < A ? m.dh[lane] : 0;
    const float my_dzh = dzh[lane], my_dzl = dzl[lane];
    const double my_Dz = Dz[lane];
    float dzmax = 0.f;
    for (int i = 0; i < A; ++i) dzmax = fmaxf(dzmax, fabsf(dzh[i]));
    const float stepf = (float)st->step;
    const double cap2 = st->cap2;
    const float reach0 = m.reach_base + stepf + dzmax;
    const float inv_dt = (float)(1.0 / m.dt);
    const float Rq = reach0 + m.tau_absmax * a.iv.vmax * 1.0001f + stepf + 2.0f;  // indexed query radius
    if (indexed && warp == 2 && !st->done) {
        // steps k0 and k0 + 1 from the state at step k0 (the origin when k0 = 0)
        const float ox = k0 > 0 ? st->s_hi[0] + st->s_lo[0] : (float)req.ox;
        const float oy = k0 > 0 ? st->s_hi[1] + st->s_lo[1] : (float)req.oy;
        const int b0 = k0 % kIBufs, b1 = (k0 + 1) % kIBufs;
        issue_direct(b0, req.depart_step + k0 + 1, row_of(req.depart_step + k0 + 1), ox, oy, Rq);
        issue_direct(b1, req.depart_step + k0 + 2, row_of(req.depart_step + k0 + 2), ox, oy, Rq);
        const int to = wait_bar(&bars[b0], ifill[b0], ipend[b0]);
        if (lane == 0) st->abort_flag[k0 & 1] = to;
        stalled = to != 0;
    }
    // ring row of the query the producer issues at step k (for step k + 2): advanced by one
    // row per step, so the loop needs no 64-bit modulo
    int64_t prow = indexed ? row_of(req.depart_step + k0 + 3) : 0;
    float ghi[3], glo[3];  // goal as double-float
    {
        const double g0[3] = {req.gx, req.gy, req.gz};
        for (int q = 0; q < 3; ++q) {
            ghi[q] = (float)g0[q];
            glo[q] = (float)__dsub_rn(g0[q], (double)ghi[q]);
        }
    }
    const float box0 = (float)m.box[0], box1 = (float)m.box[1], box2 = (float)m.box[2];
    const float box3 = (float)m.box[3], box4 = (float)m.box[4], box5 = (float)m.box[5];
    const float lg_hi = (float)m.lg64, lg_lo = (float)(m.lg64 - (double)(float)m.lg64);
    const bool has_goal = m.goal_reward > 0.0;
    const float l2r_hi = has_goal ? (float)m.log2rg : 0.f;
    const float l2r_lo = has_goal ? (float)(m.log2rg - (double)(float)m.log2rg) : 0.f;
    const float clr = (float)m.clearance, deckf = (float)m.deck;
    const float* __restrict__ hm = m.hm;
    const int hm_nx = m.hm_nx, hm_ny = m.hm_ny;
    const float hm_sx = m.hm_sx, hm_sy = m.hm_sy;
    // SUM combination (an option): the general instance only
    const bool combine = GEN && m.combine != 0;
    const int n_static = m.n_static, n_wells = m.n_wells;
    const float lg32 = m.lg32, sum_ref = m.sum_ref, tau_absmax = m.tau_absmax;
    const float sum_unit = exp2f(sum_ref - (float)kSumBits);  // value of one unit of the fixed-point sum
    const bool trace0 = GEN && a.trace && lead && r == 0;
    if (tid == 0) {
        int n0;
        float phi;
        goal_log_split(st->G_hi[0], st->G_hi[1], st->G_hi[2], st->G_lo[0], st->G_lo[1], st->G_lo[2], lg_hi, lg_lo,
                       l2r_hi, l2r_lo, n0, phi);
        st->n0 = n0;
        st->phi = phi;
    }
    __syncthreads();

    const bool timing = GEN && a.phase != nullptr && lead;
    unsigned long long ph[6] = {0, 0, 0, 0, 0, 0};
    // indexed scanners' work (statistics): items culled, items inside the cull radius,
    // (item, reachable well) pairs evaluated for every action
    unsigned qe_items = 0u, qe_dnear = 0u, qe_wells = 0u;
    long long tp = 0;

    // ---------------------------------------------------------------- step loop
    int k = k0;
    for (;; ++k) {
        if (timing && tid == 0) tp = clock64();
        __syncthreads();  // S1: state and ring entries published
        if (timing && tid == 0) { const long long t = clock64(); ph[0] += t - tp; tp = t; }
        if (st->done) break;
        const int par = k & 1;
        const int h = st->h;
        int hn = h + my_dh;  // heading index after the action's turn, wrapped to [0, 24)
        hn += hn < 0 ? 24 : 0;
        hn -= hn >= 24 ? 24 : 0;
        const float dxa = dxh[hn], dya = dyh[hn], dza = my_dzh;  // fp32 of the exact offsets
        const float shx = st->s_hi[0], shy = st->s_hi[1], shz = st->s_hi[2];
        const float slx = st->s_lo[0], sly = st->s_lo[1], slz = st->s_lo[2];
        float mloc = -INFINITY;
        unsigned long long sloc = 0ull;

        // control warp: the successor of action `lane` as a complete next-step state, kept in
        // registers until the combine publishes the winner's
        bool capn = false;
        double X = 0.0, Y = 0.0, Z = 0.0;
        float tfx = 0.f, tfy = 0.f, tfz = 0.f;  // the successor as stored (fp32)
        float sc0 = 0.f;                        // 2^-n0 of the current state
        float nhx = 0.f, nlx = 0.f, nhy = 0.f, nly = 0.f, nhz = 0.f, nlz = 0.f;
        float Gnhx = 0.f, Gnlx = 0.f, Gnhy = 0.f, Gnly = 0.f, Gnhz = 0.f, Gnlz = 0.f;
        int n0n = 0;
        float phin = 0.f;

        if (warp == 0) {
            if (lane < A) {
                // exact successor (Alg. 3) and its double-float copy
                X = __dadd_rn(st->s[0], Dx[hn]);
                Y = __dadd_rn(st->s[1], Dy[hn]);
                Z = __dadd_rn(st->s[2], my_Dz);
                tfx = (float)X;
                tfy = (float)Y;
                tfz = (float)Z;
                sc0 = exp2f((float)-st->n0);
                nhx = shx; nlx = slx; df_add(nhx, nlx, dxh[hn], dxl[hn]);
                nhy = shy; nly = sly; df_add(nhy, nly, dyh[hn], dyl[hn]);
                nhz = shz; nlz = slz; df_add(nhz, nlz, my_dzh, my_dzl);
                // goal vector at the successor, its goal-term split and capture test
                Gnhx = ghi[0]; Gnlx = glo[0]; df_add(Gnhx, Gnlx, -nhx, -nlx);
                Gnhy = ghi[1]; Gnly = glo[1]; df_add(Gnhy, Gnly, -nhy, -nly);
                Gnhz = ghi[2]; Gnlz = glo[2]; df_add(Gnhz, Gnlz, -nhz, -nlz);
                goal_log_split(Gnhx, Gnhy, Gnhz, Gnlx, Gnly, Gnlz, lg_hi, lg_lo, l2r_hi, l2r_lo, n0n, phin);
                const float gx = Gnhx + Gnlx, gy = Gnhy + Gnly, gz = Gnhz + Gnlz;
                if (approx_sqrt(gx * gx + gy * gy + gz * gz) < stepf + kCapBand)
                    capn = capture_exact_at(X, Y, Z, req, cap2);
            }
            if (timing && tid == 0) { const long long t = clock64(); ph[1] += t - tp; tp = t; }
        } else if (warp == 1) {
            // evaluator warp: the per-action terms that do not involve other plans, and the
            // goal term over 2^n0 for the combine (its near-tie flag of the previous step
            // comes after the reduction barrier)
            if (lane < A) {
                // successor estimate (fp32); terrain loads first, they are the longest wait
                const float sx = shx + (slx + dxa), sy = shy + (sly + dya), sz = shz + (slz + dza);
                float h00 = 0.f, h10 = 0.f, h01 = 0.f, h11 = 0.f, ax = 0.f, ay = 0.f;
                if (hm) {
                    const float gxf = (sx - box0) * hm_sx;
                    const float gyf = (sy - box1) * hm_sy;
                    int ix = (int)floorf(gxf), iy = (int)floorf(gyf);
                    ix = min(max(ix, 0), hm_nx - 2);
                    iy = min(max(iy, 0), hm_ny - 2);
                    ax = gxf - (float)ix;
                    ay = gyf - (float)iy;
                    const float* r0 = hm + (size_t)iy * hm_nx + ix;
                    h00 = __ldg(r0);
                    h10 = __ldg(r0 + 1);
                    h01 = __ldg(r0 + hm_nx);
                    h11 = __ldg(r0 + hm_nx + 1);
                }
                // box validity: fp32 margin, exact comparison near a face
                const float mlo = fminf(fminf(sx - box0, sy - box1), sz - box2);
                const float mhi = fminf(fminf(box3 - sx, box4 - sy), box5 - sz);
                const float mb = fminf(mlo, mhi);
                bool valid;
                if (mb > kBoxBand) valid = true;
                else if (mb < -kBoxBand) valid = false;
                else valid = box_inside_exact(m, st, Dx[hn], Dy[hn], my_Dz);
                // goal distance change Delta = |G - delta| - |G| at the current state
                const float Gx = st->G_hi[0] + st->G_lo[0], Gy = st->G_hi[1] + st->G_lo[1],
                            Gz = st->G_hi[2] + st->G_lo[2];
                const float Gn = approx_sqrt(Gx * Gx + Gy * Gy + Gz * Gz);
                const float fx = Gx - dxa, fy = Gy - dya, fz = Gz - dza;
                const float da = approx_sqrt(fx * fx + fy * fy + fz * fz);
                const float num = (dxa * dxa + dya * dya + dza * dza) - 2.0f * (Gx * dxa + Gy * dya + Gz * dza);
                const float den = da + Gn;
                const float Dl = den > 0.f ? __fdividef(num, den) : 0.f;
                // hard deck: terrain clearance at the successor (Alg. 1)
                float Vd = 0.f;
                if (hm) {
                    const float hz = (1.f - ay) * ((1.f - ax) * h00 + ax * h10) + ay * ((1.f - ax) * h01 + ax * h11);
                    const float c = sz - hz;
                    if (fabsf(c - clr) < kClrBand) Vd = deck_exact(m, st, Dx[hn], Dy[hn], my_Dz);
                    else if (c < clr) Vd = deckf - c;
                }
                valid_s[lane] = valid ? 1 : 0;
                Dl_s[lane] = Dl;
                Vd_s[lane] = Vd;
                gh_s[lane] = has_goal ? exp2f(st->phi + Dl * lg32) : 0.f;  // g / 2^n0
                // static negative peaks (restricted volumes / terrain wells), CTA 0 only
                if (GEN && lead && n_static > 0)
                    fold_statics(m, st, sch, scl, shx, shy, shz, slx, sly, slz, dxa, dya, dza, Dx[hn], Dy[hn], my_Dz,
                                 mloc, sloc);
            }
        } else if (indexed && warp == 2) {
            // ---- indexed mode: the pipeline (items for k + 2, wait for k + 1)
            int to = 1;
            if (!stalled) {
                issue_direct((k + 2) % kIBufs, req.depart_step + k + 3, prow, shx + slx, shy + sly, Rq + stepf);
                prow = prow + 1 == a.tab.T_win ? 0 : prow + 1;  // ring row of the next step's query
                prefetch_cells(req.depart_step + k + 4, prow, shx + slx, shy + sly, Rq + 2.f * stepf);
                const int b1 = (k + 1) % kIBufs;
                to = wait_bar(&bars[b1], ifill[b1], ipend[b1]);
                if (to) stalled = true;
            }
            if (lane == 0) st->abort_flag[par ^ 1] = to;
        } else {
            // ---- scanners: cull, then wells of near slots with lanes as actions
            const long long ts = (timing && tid == NT - 32) ? clock64() : 0;
            // wells of one near slot or item ii (lanes = actions); p1 / p2: its samples at
            // t + 1 and t + 2, used again for the FP64 decision inside a radius band
            // wells of a near item (offset q, velocity v) whose centre is within reach of a successor
            auto well_mask = [&](float qx_, float qy_, float qz_, float vx_, float vy_, float vz_) {
                unsigned msk = 0u;
                for (int w = 0; w < n_wells; ++w) {
                    const float tau = st->w_tau[w];
                    const float cx = fmaf(tau, vx_, qx_), cy = fmaf(tau, vy_, qy_), cz = fmaf(tau, vz_, qz_);
                    if (fmaf(cx, cx, fmaf(cy, cy, cz * cz)) < st->wlim2[w]) msk |= 1u << w;
                }
                return msk;
            };
            auto fold_near = [&](auto&& item_at, int ii, float bqx, float bqy, float bqz, float bvx, float bvy,
                                 float bvz, unsigned bwm) {
                if (lane >= A) return;
                float mb = -INFINITY;
                unsigned long long sb = 0ull;
                // the wells that reach a successor (set bits of bwm); a well whose edge lies within
                // the FP32 band of this lane's successor is decided after the loop, so that the
                // loop stays short (its band branch, rarely taken, held the item read and an FP64
                // call)
                unsigned band = 0u;
                for (unsigned msk = bwm; msk; msk &= msk - 1u) {
                    const int w = __ffs(msk) - 1;
                    bool bw = false;
                    fold_well(st, w, bqx, bqy, bqz, bvx, bvy, bvz, dxa, dya, dza, mb, sb, bw, combine, sum_ref);
                    band |= bw ? 1u << w : 0u;
                }
                if (band) {
                    float p1x, p1y, p1z, p2x, p2y, p2z;
                    item_at(ii, p1x, p1y, p1z, p2x, p2y, p2z);
                    const bool has2 = p2x == p2x;
                    for (; band; band &= band - 1u) {
                        const int w = __ffs(band) - 1;
                        if (well_inside_exact(m, st, Dx[hn], Dy[hn], my_Dz, p1x, p1y, p1z, has2 ? p2x : 0.f,
                                              has2 ? p2y : 0.f, has2 ? p2z : 0.f, has2, w)) {
                            const float tau = st->w_tau[w];
                            const float ex = dxa - fmaf(tau, bvx, bqx), ey = dya - fmaf(tau, bvy, bqy),
                                        ez = dza - fmaf(tau, bvz, bqz);
                            const float l =
                                fmaf(approx_sqrt(fmaf(ex, ex, fmaf(ey, ey, ez * ez))), st->w_lg[w], st->w_L[w]);
                            mb = fmaxf(mb, l);
                            if (combine) sb += sum_term(l, sum_ref);
                        }
                    }
                }
                mloc = fmaxf(mloc, mb);
                sloc += sb;
            };
            if (indexed) {
                // items staged for this step (buffer par), the overflow read from the index
                const int b = k % kIBufs;
                const IdxMeta& M = imeta[b];
                const int total = M.total, n_s = M.n_s;
                const float4* sb4 = ibuf + (size_t)b * icap * 2;
                int itag = 0;  // tag of the item item_at read last
                auto item_at = [&](int i, float& p1x, float& p1y, float& p1z, float& p2x, float& p2y, float& p2z) {
                    float4 P1, P2;
                    if (i < n_s) {
                        P1 = sb4[2 * i];
                        P2 = sb4[2 * i + 1];
                    } else {
                        int q = 0, off = i;
                        while (q < M.nr - 1 && off >= M.cnt[q]) { off -= M.cnt[q]; ++q; }
                        const float4* g = a.iv.items + M.row_off + 2ll * (M.beg[q] + off);
                        P1 = __ldcg(g);
                        P2 = __ldcg(g + 1);
                    }
                    p1x = P1.x; p1y = P1.y; p1z = P1.z;
                    p2x = P2.x; p2y = P2.y; p2z = P2.z;
                    itag = __float_as_int(P1.w);
                };
                // items interleaved over the scanner warps (item i to warp i mod nscan): the
                // items within reach, each costing a well evaluation per action, sit next to
                // one another in the index (same cells), so this spreads them over the warps
                const int nscan = NW - 3, sw = warp - 3;
                const int wn = total > sw ? (total - sw + nscan - 1) / nscan : 0;  // items of this warp
                // one item per lane per pass: a warp rarely holds more than 32 items of a step,
                // and a second unrolled copy of the fold only lengthens the step's code
                constexpr int U = 1;
                for (int base = 0; base < wn; base += 32 * U) {
                    float qx[U], qy[U], qz[U], vx[U], vy[U], vz[U];
                    bool near[U];
                    unsigned wm[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int j = base + u * 32 + lane;
                        const int i = sw + j * nscan;
                        near[u] = false;
                        qx[u] = qy[u] = qz[u] = vx[u] = vy[u] = vz[u] = 0.f;
                        if (j < wn) {
                            float p1x, p1y, p1z, p2x, p2y, p2z;
                            item_at(i, p1x, p1y, p1z, p2x, p2y, p2z);
                            // not in this request's table (a later request's tentative plan,
                            // or a withdrawn one): culled like a plan far away
                            if (!tag_visible(itag, my_ord)) p1x = p2x = __int_as_float(0x7fc00000);
                            qx[u] = (p1x - shx) - slx;
                            qy[u] = (p1y - shy) - sly;
                            qz[u] = (p1z - shz) - slz;
                            if (p2x == p2x) {
                                vx[u] = (p2x - p1x) * inv_dt;
                                vy[u] = (p2y - p1y) * inv_dt;
                                vz[u] = (p2z - p1z) * inv_dt;
                            }
                            const float reach =
                                fmaf(tau_absmax, approx_sqrt(vx[u] * vx[u] + vy[u] * vy[u] + vz[u] * vz[u]), reach0);
                            near[u] = (qx[u] * qx[u] + qy[u] * qy[u] + qz[u] * qz[u]) < reach * reach;
                            ++qe_items;
                        }
                        qe_dnear += near[u] ? 1u : 0u;
                        wm[u] = near[u] ? well_mask(qx[u], qy[u], qz[u], vx[u], vy[u], vz[u]) : 0u;
                        near[u] = wm[u] != 0u;
                        qe_wells += __popc(wm[u]);
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        unsigned mask = __ballot_sync(kFull, near[u]);
                        while (mask) {
                            const int b = __ffs(mask) - 1;
                            mask &= mask - 1;
                            const int ii = sw + (base + u * 32 + b) * nscan;
                            fold_near(item_at, ii, __shfl_sync(kFull, qx[u], b), __shfl_sync(kFull, qy[u], b),
                                      __shfl_sync(kFull, qz[u], b), __shfl_sync(kFull, vx[u], b),
                                      __shfl_sync(kFull, vy[u], b), __shfl_sync(kFull, vz[u], b),
                                      __shfl_sync(kFull, wm[u], b));
                        }
                    }
                }
            } else {
            const int e1 = entry_of(k + 1), e2 = entry_of(k + 2);
            const bool v1 = st->ent_valid[e1] != 0;
            const bool v2 = (k + 2 <= last_j) && st->ent_valid[e2] != 0;
            if (v1) mbar_test_wait(&bars[e1], parity_of(k + 1));
            if (v2) mbar_test_wait(&bars[e2], parity_of(k + 2));
            const float* X1 = ring + (size_t)e1 * 3 * chunk;
            const float* Y1 = X1 + chunk;
            const float* Z1 = Y1 + chunk;
            const float* X2 = ring + (size_t)e2 * 3 * chunk;
            const float* Y2 = X2 + chunk;
            const float* Z2 = Y2 + chunk;
            auto item_at = [&](int i, float& p1x, float& p1y, float& p1z, float& p2x, float& p2y, float& p2z) {
                p1x = X1[i]; p1y = Y1[i]; p1z = Z1[i];
                if (v2) { p2x = X2[i]; p2y = Y2[i]; p2z = Z2[i]; }
                else { p2x = p2y = p2z = __int_as_float(0x7fc00000); }
            };
            const int scan_len = v1 ? c_len : 0;
            const int nscan = NW - 2;
            constexpr int U = 2;  // slots per lane per pass (independent chains)
            for (int base = (warp - 2) * 32 * U; base < scan_len; base += nscan * 32 * U) {
                float qx[U], qy[U], qz[U], vx[U], vy[U], vz[U];
                bool near[U];
                unsigned wm[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int i = base + u * 32 + lane;
                    near[u] = false;
                    qx[u] = qy[u] = qz[u] = vx[u] = vy[u] = vz[u] = 0.f;
                    if (i < scan_len) {
                        const float p1x = X1[i], p1y = Y1[i], p1z = Z1[i];
                        qx[u] = (p1x - shx) - slx;
                        qy[u] = (p1y - shy) - sly;
                        qz[u] = (p1z - shz) - slz;
                        if (v2) {
                            const float p2x = X2[i];
                            if (p2x == p2x) {
                                vx[u] = (p2x - p1x) * inv_dt;
                                vy[u] = (Y2[i] - p1y) * inv_dt;
                                vz[u] = (Z2[i] - p1z) * inv_dt;
                            }
                        }
                        const float reach =
                            fmaf(tau_absmax, approx_sqrt(vx[u] * vx[u] + vy[u] * vy[u] + vz[u] * vz[u]), reach0);
                        near[u] = (qx[u] * qx[u] + qy[u] * qy[u] + qz[u] * qz[u]) < reach * reach;  // NaN: false
                    }
                    wm[u] = near[u] ? well_mask(qx[u], qy[u], qz[u], vx[u], vy[u], vz[u]) : 0u;
                    near[u] = wm[u] != 0u;
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    unsigned mask = __ballot_sync(kFull, near[u]);
                    while (mask) {
                        const int b = __ffs(mask) - 1;
                        mask &= mask - 1;
                        const int ii = base + u * 32 + b;
                        fold_near(item_at, ii, __shfl_sync(kFull, qx[u], b), __shfl_sync(kFull, qy[u], b),
                                  __shfl_sync(kFull, qz[u], b), __shfl_sync(kFull, vx[u], b),
                                  __shfl_sync(kFull, vy[u], b), __shfl_sync(kFull, vz[u], b),
                                  __shfl_sync(kFull, wm[u], b));
                    }
                }
            }
            }
            if (ts) ph[4] += clock64() - ts;
        }
        if (lane < A) {
            if (mloc > -INFINITY) atomicMax(&keys[lane], float_key(mloc));
            if (combine && sloc) atomicAdd(&sums[lane], sloc);
        }
        __syncwarp();
        if (timing && tid == 0) tp = clock64();
        // S3: per-action partials of this CTA complete (indexed mode: the producer warp, which
        // adds no partials, goes on to the next step's start instead)
        if (indexed) {
            if (warp != 2) named_barrier(1, NT - 32);
        } else {
            __syncthreads();
        }
        if (timing && tid == 0) { const long long t = clock64(); ph[2] += t - tp; tp = t; }

        if (warp == 0) {
            // ---- exchange across the cluster (DSMEM push, one hop) or read locally
            int key = lane < A ? keys[lane] : KEY_NONE;
            unsigned long long ssum = (combine && lane < A) ? sums[lane] : 0ull;
            int ab = st->abort_flag[par];
            if (lane < A) {
                keys[lane] = KEY_NONE;
                if (combine) sums[lane] = 0ull;
            }
            if (cs > 1) {
                const uint32_t bytes = (uint32_t)cs * ((uint32_t)A * (combine ? 12u : 4u) + 4u);
                if (lane == 0) mbar_arrive_expect_tx(&xbar[par], bytes);
                const uint32_t kslot = smem_u32(&xkeys[(par * kMaxCluster + (int)rank) * kMaxActions + lane]);
                const uint32_t sslot = smem_u32(&xsums[(par * kMaxCluster + (int)rank) * kMaxActions + lane]);
                const uint32_t aslot = smem_u32(&xab[par * kMaxCluster + (int)rank]);
                const uint32_t bslot = smem_u32(&xbar[par]);
                for (int q = 0; q < cs; ++q) {
                    const uint32_t rb = dsmem_addr(bslot, (uint32_t)q);
                    if (lane < A) {
                        st_async_s32(dsmem_addr(kslot, (uint32_t)q), key, rb);
                        if (combine) st_async_u64(dsmem_addr(sslot, (uint32_t)q), ssum, rb);
                    }
                    if (lane == 31) st_async_s32(dsmem_addr(aslot, (uint32_t)q), ab, rb);
                }
                if (!mbar_wait_bounded(&xbar[par], (uint32_t)((k >> 1) & 1))) {
                    atomicExch(a.err, FMDP_ERR_TIMEOUT);
                    ab = 1;
                } else {
                    key = KEY_NONE;
                    ssum = 0ull;
                    int any = 0;
                    for (int q = 0; q < cs; ++q) {
                        if (lane < A) {
                            key = max(key, xkeys[(par * kMaxCluster + q) * kMaxActions + lane]);
                            ssum += xsums[(par * kMaxCluster + q) * kMaxActions + lane];
                        }
                        any |= xab[par * kMaxCluster + q];
                    }
                    ab = any;
                }
            }
            ab = __any_sync(kFull, ab != 0) ? 1 : 0;

            // ---- action values as (sign class, log2 |Q|) keys; Q = g - P - V (Alg. 1, Alg. 8)
            const int n0 = st->n0;
            const float phi = st->phi;
            const bool valid = lane < A && valid_s[lane] != 0;
            const float Dl = Dl_s[lane], Vd = Vd_s[lane];
            float Lp;
            if (combine) Lp = ssum ? __log2f((float)ssum) + (sum_ref - (float)kSumBits) : -INFINITY;
            else Lp = key_float(key);
            const float lgh = phi + Dl * lg32;  // log2(g) - n0
            // penalty + deck N, linear; the goal term g / 2^n0 comes from the evaluator
            const bool pen = (combine ? ssum != 0ull : Lp > -INFINITY) || Vd > 0.f;
            float Nl = 0.f;
            if (pen) Nl = (combine ? (float)ssum * sum_unit : (Lp > -INFINITY ? exp2f(Lp) : 0.f)) + Vd;
            int cls;   // 2: Q > 0, 1: Q = 0, 0: Q < 0
            float k2;  // larger is better within a class
            float la;  // log2 |Q|
            if (!pen) {
                cls = has_goal ? 2 : 1;
                k2 = has_goal ? lgh : 0.f;
                la = has_goal ? lgh + (float)n0 : -INFINITY;
            } else {
                const float gh = gh_s[lane];
                const float Nh = Nl * sc0;  // N / 2^n0 (inf when that overflows fp32)
                const float d = gh - Nh;
                if (has_goal && d > 0.f) {
                    cls = 2;
                    k2 = __log2f(d);
                    la = k2 + (float)n0;
                } else if (d == 0.f) {
                    cls = 1;
                    k2 = 0.f;
                    la = -INFINITY;
                } else {
                    cls = 0;
                    la = Nh < INFINITY ? __log2f(-d) + (float)n0 : __log2f(Nl);  // log2 (N - g)
                    k2 = -la;
                }
            }
            const uint32_t qkey = (lane < A && valid) ? action_key(cls, k2) : 0u;
            const uint32_t kmax = __reduce_max_sync(kFull, qkey);
            const unsigned bm = __ballot_sync(kFull, qkey == kmax && kmax != 0u);
            const int best = bm ? __ffs(bm) - 1 : 99;
            if (ab || best >= 99) {
                if (lane == 0) { st->done = 1; st->status = FMDP_REJ_NO_ACTION; st->steps = k; }
            } else if (lane == best) {
                // the winning lane publishes its successor as the next state
                st->s[0] = X; st->s[1] = Y; st->s[2] = Z;
                st->s_hi[0] = nhx; st->s_lo[0] = nlx;
                st->s_hi[1] = nhy; st->s_lo[1] = nly;
                st->s_hi[2] = nhz; st->s_lo[2] = nlz;
                st->G_hi[0] = Gnhx; st->G_lo[0] = Gnlx;
                st->G_hi[1] = Gnhy; st->G_lo[1] = Gnly;
                st->G_hi[2] = Gnhz; st->G_lo[2] = Gnlz;
                st->n0 = n0n;
                st->phi = phin;
                st->h = hn;
                const bool last = (k + 1) >= req.horizon;
                st->done = capn || last;
                st->status = capn ? kStatusCaptured : FMDP_REJ_HORIZON;
                st->steps = k + 1;
                const int np = k + 1;  // one point per step after the origin
                st->n_points = np + 1;
                if (lead) {
                    traj[3 * np] = tfx;
                    traj[3 * np + 1] = tfy;
                    traj[3 * np + 2] = tfz;
                    acts[k] = (uint8_t)best;
                    if (a.pipe.obs) {  // what a resumed plan and the host's influence test need
                        const size_t o = (size_t)r * a.cap;
                        a.pipe.obs[o + k] = imeta[k % kIBufs].pub;
                        double* ps = a.pipe.st_s + 3 * (o + np);
                        ps[0] = X; ps[1] = Y; ps[2] = Z;
                        float* pd = a.pipe.st_df + 6 * (o + np);
                        pd[0] = nhx; pd[1] = nlx; pd[2] = nhy; pd[3] = nly; pd[4] = nhz; pd[5] = nlz;
                        a.pipe.st_h[o + np] = (uint8_t)hn;
                    }
                    if (GEN && a.trace && r == 0) {
                        a.st_trace[3 * np] = X;
                        a.st_trace[3 * np + 1] = Y;
                        a.st_trace[3 * np + 2] = Z;
                        a.hd_trace[np] = hn;
                    }
                }
            }
            // keys of this step for the evaluator warp's deferred near-tie flag
            const float logN = pen ? __log2f(Nl) : -INFINITY;
            qkey_s[par * kMaxActions + lane] = qkey;
            cls_s[par * kMaxActions + lane] = cls;
            la_s[par * kMaxActions + lane] = la;
            lt_s[par * kMaxActions + lane] = fmaxf(has_goal ? lgh + (float)n0 : -INFINITY, logN);  // log2 max(g, N)
            if (lane == 0) st->last_best[par] = (ab || best >= 99) ? 99 : best;
            if (trace0 && lane < A)  // FP64 action values for the trace (not used for the decision)
                a.q_trace[(size_t)k * A + lane] = valid ? trace_q(m, has_goal, n0, phi, Dl, Lp, ssum, Vd) : -INFINITY;
            if (timing && tid == 0) ph[3] += clock64() - tp;
        } else {
            // evaluator warp: near-tie flag of the previous step, off the step's critical path
            if (warp == 1 && k > k0)
                deferred_tie(st, qkey_s, cls_s, la_s, lt_s, par ^ 1, lane,
                             trace0 ? a.tie_trace + (k - 1) : (a.pipe.ties ? a.pipe.ties + (size_t)r * a.cap + (k - 1) : nullptr));
        }
        if (producer && !indexed) {
            // ---- producer: slices needed two or more steps ahead
            const long long t0 = timing ? clock64() : 0;
            int to = 0;
            if (!stalled) {
                issue_upto((int64_t)k + 1 + depth);
                to = wait_upto((int64_t)k + 3);
                if (to) stalled = true;
            } else {
                to = 1;
            }
            st->abort_flag[par ^ 1] = to;
            if (timing) ph[5] += clock64() - t0;
        }
        __syncwarp();  // reconverge the control warp and the producer's warp before S1
    }

    // ---- epilogue: near-tie flag of the last step, drain the ring, outputs
    if (warp == 1 && k > k0)
        deferred_tie(st, qkey_s, cls_s, la_s, lt_s, (k - 1) & 1, lane,
                     trace0 ? a.tie_trace + (k - 1) : (a.pipe.ties ? a.pipe.ties + (size_t)r * a.cap + (k - 1) : nullptr));
    __syncthreads();
    if (indexed && warp == 2) drain();
    if (producer) {
        while (waited < issued) {
            const int64_t j = waited + 1;
            if (!mbar_wait_bounded(&bars[entry_of(j)], parity_of(j))) {
                atomicExch(a.err, FMDP_ERR_TIMEOUT);
                break;
            }
            waited = j;
        }
    }
    if (tid == 0 && lead) {
        RolloutOut o;
        o.n_points = st->n_points;
        o.status = st->status;
        o.near_ties = st->near_ties;
        o.steps = st->steps;
        a.out[r] = o;
    }
    if (timing && (tid == 0 || tid == NT - 32 || producer))
        for (int i = 0; i < 6; ++i)
            if (ph[i]) atomicAdd(&a.phase[i], ph[i]);
    if (a.qe_ctr && warp >= 3) {
        for (int off = 16; off; off >>= 1) {
            qe_items += __shfl_xor_sync(kFull, qe_items, off);
            qe_dnear += __shfl_xor_sync(kFull, qe_dnear, off);
            qe_wells += __shfl_xor_sync(kFull, qe_wells, off);
        }
        if (lane == 0 && qe_items) {
            atomicAdd(&a.qe_ctr[0], (unsigned long long)qe_items);
            atomicAdd(&a.qe_ctr[1], (unsigned long long)qe_dnear);
            atomicAdd(&a.qe_ctr[2], (unsigned long long)qe_wells);
        }
    }
    if (cs > 1) cluster_barrier(); else __syncthreads();  // peers may still address this CTA's shared memory
    if ((a.queue || a.pipe.on) && tid == 0) {  // the next request of this CTA initialises them again
        for (int e = 0; e < kRingDepth; ++e) mbar_inval(&bars[e]);
        mbar_inval(&xbar[0]);
        mbar_inval(&xbar[1]);
    }
}

// ---------------------------------------------------------------- pipelined FCFS

__device__ __forceinline__ int ld_acquire_sys(const int32_t* p) {
    int v;
    asm volatile("ld.acquire.sys.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_volatile_sys(const int32_t* p) {
    int v;
    asm volatile("ld.volatile.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ long long ld_volatile_sys64(const int64_t* p) {
    long long v;
    asm volatile("ld.volatile.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_sys(int32_t* p, int v) {
    asm volatile("st.release.sys.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Takes the next work item of the host-fed ring (thread 0). Returns its ring position, or
// -1 when the CTA should leave: the host asked it to stop and the ring is empty, no work
// came for idle_cycles, or a bounded wait of another CTA expired.
__device__ int pipe_take(const RolloutArgs& a, int* r_out, int* tok_out, int* start_out, long long* tb_out) {
    const PipeArgs& p = a.pipe;
    long long t0 = clock64();
    unsigned ns = 32;
    for (;;) {
        if (*reinterpret_cast<volatile const int32_t*>(a.err) != 0) return -1;
        const int h = *reinterpret_cast<volatile int32_t*>(p.head);
        const int t = ld_acquire_sys(p.tail);
        if (h < t) {
            if (atomicCAS(p.head, h, h + 1) == h) {
                const PipeItem* it = p.items + (h & p.qmask);
                *r_out = ld_volatile_sys(&it->r);
                *tok_out = ld_volatile_sys(&it->token);
                *tb_out = ld_volatile_sys64(&it->t_base);
                *start_out = ld_volatile_sys(&it->start);
                return h;
            }
            continue;
        }
        if (ld_volatile_sys(p.stop)) return -1;
        if (clock64() - t0 > p.idle_cycles) return -1;
        __nanosleep(ns);
        ns = ns < 4096 ? 2 * ns : 4096;
    }
}

// After a pipelined plan: its conflicts and terrain collisions against the plans the index
// holds now (each sample against the items of its step within the horizontal minimum, by
// cell, and the row's extra list), its trajectory and report to host-mapped memory, then
// its completion token. The index holds the plans admitted before this request (the host
// admits in arrival order and never past an unresolved request) and the tentative plans of
// earlier requests (the items of later requests' plans are skipped by their tag). The
// table-operation count read before the rows goes into the report: where the request's
// final table differs from what this check could have seen (a tentative plan replaced or
// withdrawn since, or published after that count), the host's influence test finds it and
// has the check (or the plan) done again.
__device__ void pipe_finish(const RolloutArgs& a, int r, int token, int* red, long long tbase) {
    int& s_first = red[0];
    int& s_terr = red[1];
    const int tid = threadIdx.x, NT = blockDim.x;
    if (tid == 0) {
        s_first = INT_MAX;
        s_terr = INT_MAX;
        red[2] = INT_MAX;
    }
    // admissions published before this thread's index reads (all of them are seen)
    const int my_pub = a.pipe.pub_seq ? ld_acquire_gpu(a.pipe.pub_seq) : INT_MAX;
    __syncthreads();
    atomicMin(&red[2], my_pub);
    const RolloutOut ro = a.out[r];
    const fmdp_request& rq = a.reqs[r];
    const int n = ro.n_points;
    const float* traj = a.traj + (size_t)r * a.cap * 3;
    const Model& m = a.m;
    const IndexView& iv = a.iv;
    const SepConsts sk = sep_consts(m.sep_h, m.sep_v);
    const float reach = (float)m.sep_h + 1.0f;  // past it every pair is clear horizontally
    const int32_t my_ord = a.pipe.ord0 + r;
    const int64_t cst_row_len = (int64_t)iv.ncell + 1;
    int first = INT_MAX, terr = INT_MAX;
    auto cell_of = [&](float v, float o, int nc) {
        const float f = floorf((v - o) * iv.inv_cell);
        return f < 0.f ? 0 : (f > (float)(nc - 1) ? nc - 1 : (int)f);
    };
    for (int i = tid; i < n; i += NT) {
        const float px = traj[3 * i], py = traj[3 * i + 1], pz = traj[3 * i + 2];
        if (m.hm && below_terrain(m, px, py, pz)) terr = min(terr, i);
        if (i >= first) continue;  // a later sample cannot lower this thread's first conflict
        const int64_t T = rq.depart_step + i;
        if (T < tbase || T >= tbase + a.tab.T_win) continue;
        int64_t row = T % a.tab.T_win;
        if (row < 0) row += a.tab.T_win;
        const int32_t* cs_row = iv.cstart + row * cst_row_len;
        const float4* items = iv.items + (size_t)row * a.tab.S_pad * 2;
        const int cx0 = cell_of(px - reach, iv.x0, iv.ncx), cx1 = cell_of(px + reach, iv.x0, iv.ncx);
        const int cy0 = cell_of(py - reach, iv.y0, iv.ncy), cy1 = cell_of(py + reach, iv.y0, iv.ncy);
        bool hit = false;
        for (int cy = cy0; cy <= cy1 + 1 && !hit; ++cy) {
            int b, e;
            if (cy <= cy1) {
                b = __ldcg(cs_row + cy * iv.ncx + cx0);
                e = __ldcg(cs_row + cy * iv.ncx + cx1 + 1);
            } else {  // the extra list
                b = __ldcg(cs_row + iv.ncell);
                e = b + __ldcg(iv.nextra + row);
            }
            for (int j = b; j < e; ++j) {
                const float4 Q = __ldcg(items + 2 * (size_t)j);
                if (!tag_visible(__float_as_int(Q.w), my_ord)) continue;
                float h2, dz;
                bool hin, vin;
                sep_pair(sk, px, py, pz, Q.x, Q.y, Q.z, h2, dz, hin, vin);
                if (hin && vin) {
                    hit = true;
                    break;
                }
            }
        }
        if (hit) first = i;
    }
    if (first != INT_MAX) atomicMin(&s_first, first);
    if (terr != INT_MAX) atomicMin(&s_terr, terr);
    // trajectory to the host, 12-byte samples as 4-byte words
    float* dst = a.pipe.h_traj + (size_t)r * a.cap * 3;
    for (int i = tid; i < 3 * n; i += NT) dst[i] = traj[i];
    const int32_t* obs = a.pipe.obs + (size_t)r * a.cap;
    int32_t* hobs = a.pipe.h_obs + (size_t)r * a.cap;
    for (int i = tid; i < n - 1; i += NT) hobs[i] = obs[i];
    __threadfence_system();
    __syncthreads();
    if (tid == 0) {
        SepOut so;
        so.first_conflict = s_first;
        so.first_terrain = s_terr;
        so.conflicts = 0ull;
        so.min_h_bits = 0x7f800000u;
        so.min_v_bits = 0x7f800000u;
        so.verdict = -1;
        so.pad = 0;
        a.pipe.sep[r] = so;
        PipeRecord* rec = a.pipe.rec + r;
        rec->ro = ro;
        rec->first_conflict = s_first == INT_MAX ? -1 : s_first;
        rec->first_terrain = s_terr == INT_MAX ? -1 : s_terr;
        rec->tail_pub = red[2];
        __threadfence_system();
        st_release_sys(a.pipe.done + r, token);
    }
    __syncthreads();
}

// Persistent pipelined launch (indexed mode, one CTA per work item): plans the items the
// host appends to the ring until it is told to stop, stays idle too long, or a wait expires.
template <bool GEN>
__device__ void pipe_loop(const RolloutArgs& a, unsigned char* smem) {
    const Layout L = make_layout(a.chunk, a.ring, a.icap);
    int* slot = reinterpret_cast<int*>(smem + L.misc);  // [0] ring position, [1] request, [2] token, [3] start
    long long* slot_tb = reinterpret_cast<long long*>(slot + 8);  // the item's window
    for (;;) {
        if (threadIdx.x == 0) {
            int r = 0, tok = 0, k0 = 0;
            long long tb = 0;
            const int w = pipe_take(a, &r, &tok, &k0, &tb);
            slot[0] = w;
            slot[1] = r;
            slot[2] = tok;
            slot[3] = k0;
            *slot_tb = tb;
        }
        __syncthreads();
        const int w = reinterpret_cast<volatile int*>(slot)[0];
        const int r = reinterpret_cast<volatile int*>(slot)[1];
        const int tok = reinterpret_cast<volatile int*>(slot)[2];
        const int k0 = reinterpret_cast<volatile int*>(slot)[3];
        const long long tb = *reinterpret_cast<volatile long long*>(slot_tb);
        __syncthreads();
        if (w < 0) break;
        if (k0 >= 0) plan_request<true, GEN>(a, r, smem, tb, k0);  // k0 < 0: the plan stands, only its check again
        pipe_finish(a, r, tok, slot + 4, tb);
    }
}

// One launch plans a set of requests. Without a work queue, cluster c plans request c.
// With a work queue (batch mode), each resident cluster pulls work items from a device
// counter until none are left, which balances requests of uneven horizon: the lead CTA
// takes the item and its peers read it from the lead's shared memory.
// IDX: the indexed-mode instance (cluster size 1; the pipelined mode runs only there);
// GEN: with the phase clock stamps.
template <bool IDX, bool GEN>
__global__ void __launch_bounds__(384, 1) rollout_kernel(const __grid_constant__ RolloutArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int cs = IDX ? 1 : a.cs;
    if constexpr (IDX) {
        if (a.pipe.on) {
            pipe_loop<GEN>(a, smem);
            return;
        }
    }
    if (a.queue == nullptr) {
        const int r = blockIdx.x / cs;
        if (r < a.n_req) plan_request<IDX, GEN>(a, r, smem, a.tab.t_base);  // uniform over the cluster
        return;
    }
    const Layout L = make_layout(a.chunk, a.ring, IDX ? a.icap : 0);
    int* next = reinterpret_cast<int*>(smem + L.misc);
    const int n = a.n_dev ? *a.n_dev : a.n_req;
    const bool lead = cs == 1 || cluster_rank() == 0;
    for (;;) {
        if (threadIdx.x == 0 && lead)  // after a device error, stop taking work
            *next = *reinterpret_cast<volatile int32_t*>(a.err) != 0 ? n : atomicAdd(a.queue, 1);
        int w;
        if (cs > 1) {
            cluster_barrier();
            w = ld_cluster_s32(dsmem_addr(smem_u32(next), 0));
            cluster_barrier();  // every CTA has read the item before the lead takes the next
        } else {
            __syncthreads();
            w = *reinterpret_cast<volatile int*>(next);
            __syncthreads();
        }
        if (w >= n) break;
        const int r = a.idx ? a.idx[w] : w;
        if (a.skip && a.skip[r]) continue;  // uniform over the cluster: every CTA read the same item
        plan_request<IDX, GEN>(a, r, smem, a.tab.t_base);
    }
}

size_t rollout_smem_bytes(int chunk, int depth, int icap) { return make_layout(chunk, depth, icap).total; }

cudaError_t prepare_rollout_kernel(size_t smem) {
    const void* fs[4] = {(const void*)rollout_kernel<true, false>, (const void*)rollout_kernel<false, false>,
                         (const void*)rollout_kernel<true, true>, (const void*)rollout_kernel<false, true>};
    for (const void* f : fs) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaFuncSetAttribute(fs[1], cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(fs[3], cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

int rollout_max_active_clusters_query(int cs, int threads, size_t smem);

int rollout_max_active_clusters(int cs, int threads, size_t smem) {
    // the answer depends only on the launch shape and the device: remember it per thread
    // (batched calls ask before every wave whose shape changed)
    struct Memo {
        int dev, cs, threads;
        size_t smem;
        int n;
    };
    thread_local Memo memo[16];
    thread_local int memo_n = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    for (int i = 0; i < memo_n; ++i)
        if (memo[i].dev == dev && memo[i].cs == cs && memo[i].threads == threads && memo[i].smem == smem)
            return memo[i].n;
    const int n = rollout_max_active_clusters_query(cs, threads, smem);
    if (n > 0) {
        memo[memo_n % 16] = Memo{dev, cs, threads, smem, n};
        memo_n = memo_n < 16 ? memo_n + 1 : 16;
    }
    return n;
}

template <bool IDX, bool GEN>
int rollout_max_active_clusters_of(int cs, int threads, size_t smem) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cs, 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, rollout_kernel<IDX, GEN>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

// Clusters of cs CTAs that fit at once. Every instance that may run that shape is asked (the
// indexed ones only for cluster size 1); the smallest answer holds for all of them.
int rollout_max_active_clusters_query(int cs, int threads, size_t smem) {
    int n = std::min(rollout_max_active_clusters_of<false, false>(cs, threads, smem),
                     rollout_max_active_clusters_of<false, true>(cs, threads, smem));
    if (cs == 1)
        n = std::min(n, std::min(rollout_max_active_clusters_of<true, false>(cs, threads, smem),
                                 rollout_max_active_clusters_of<true, true>(cs, threads, smem)));
    return n;
}

cudaError_t launch_rollout(const RolloutArgs& a, int threads, size_t smem, cudaStream_t s, int n_clusters) {
    if (a.indexed && a.cs != 1) return cudaErrorInvalidValue;  // the indexed instance has no cluster
    if (a.pipe.on && !a.indexed) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((n_clusters > 0 ? n_clusters : a.n_req) * a.cs), 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)a.cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // the general instance: phase stamps, trace, SUM combination or static wells
    const bool timed = a.phase != nullptr || a.trace != 0 || a.m.combine != 0 || a.m.n_static > 0;
    if (a.indexed)
        return timed ? cudaLaunchKernelEx(&cfg, rollout_kernel<true, true>, a)
                     : cudaLaunchKernelEx(&cfg, rollout_kernel<true, false>, a);
    return timed ? cudaLaunchKernelEx(&cfg, rollout_kernel<false, true>, a)
                 : cudaLaunchKernelEx(&cfg, rollout_kernel<false, false>, a);
}

}  // namespace fmdp
