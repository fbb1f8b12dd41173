// Persistent FastMDP rollout kernel (sm_103a).
//
// One thread-block cluster plans one request from departure to capture, horizon or
// dead end, without returning to the host (the paper's CPU loop of Fig. 3 runs nine
// kernels and a device-to-host copy per step; here the whole loop is one launch).
//
// Per step k (state s at time t = depart + k, successors at t + 1):
//   staging   slices t+1 (well positions) and t+2 (plan velocity) of this CTA's slot
//             partition arrive by TMA bulk copies into a 4-deep shared-memory ring; the
//             producer runs two steps ahead because the table does not depend on s;
//   cull      every slot whose wells cannot reach any successor is dropped by one
//             distance test (radius max_k R_k + |tau|max |v| + step + 1 m);
//   wells     near slots x actions x wells (Alg. 5-7, Table 3): lane a of a warp scores
//             action a; log2 of |r| gamma^d is max-reduced per action (Alg. 8 max);
//   exchange  per-action maxima are combined across the cluster through DSMEM;
//   combine   warp 0 of every CTA forms Q = goal - penalty - hard deck (Alg. 1, 8),
//             takes the argmax (Alg. 9, lowest index on ties) and advances the FP64
//             state exactly as the forward projection defines it (Alg. 3).
//
// Exactness: the state advance, box test, capture test and every threshold decision
// (well edge, terrain clearance) are evaluated in FP64 with explicitly rounded
// operations in the order the method defines them, so decisions match an FP64
// evaluation bit for bit; magnitudes of the well values are fp32 (relative error ~1e-6).
#include <cfloat>
#include <climits>

#include "fmdp_internal.cuh"

namespace fmdp {

namespace {

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
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t dsmem_addr(const void* local, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(local)), "r"(rank));
    return r;
}
__device__ __forceinline__ int dsmem_ld_s32(uint32_t addr) {
    int v;
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long dsmem_ld_u64(uint32_t addr) {
    unsigned long long v;
    asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(addr) : "memory");
    return v;
}

struct StepState {
    double s[3];      // current state (FP64)
    double e2;        // |goal - s|^2, FP64 in the method's order
    double cap2;      // (speed * dt)^2
    double step;      // speed * dt
    float s_hi[3], s_lo[3];  // s = s_hi + s_lo (fp32 pair) for fp32 plan offsets
    float G[3];       // goal - s, fp32
    float Gn;         // |G|
    int h;            // heading index (15-degree units relative to the initial bearing)
    int done;
    int status;
    int n_points;
    int near_ties;
    int steps;
    int abort_flag[2];  // this CTA's staging timed out in step k (indexed by k & 1)
    int cnt[2];       // near-list counters (double buffered by scan round)
    int ent_valid[kRing];
};

// Shared-memory carve-up (identical on host and device).
struct Layout {
    size_t ring, bars, st, tabs, keys, sums, sq, nl, total;
    int nl_cap;
};
__host__ __device__ inline Layout make_layout(int chunk, int threads) {
    Layout L;
    size_t o = 0;
    L.ring = o;
    o += (size_t)kRing * 3 * chunk * sizeof(float);
    o = (o + 15) & ~size_t(15);
    L.bars = o;
    o += kRing * sizeof(uint64_t);
    L.st = o;
    o += (sizeof(StepState) + 15) & ~size_t(15);
    L.tabs = o;  // Dx[24], Dy[24], dz64[32] doubles, then dx32[24], dy32[24], dz32[32] floats
    o += (24 + 24 + 32) * sizeof(double) + (24 + 24 + 32) * sizeof(float);
    o = (o + 15) & ~size_t(15);
    L.keys = o;
    o += 2 * kMaxActions * sizeof(int);
    o = (o + 15) & ~size_t(15);
    L.sums = o;
    o += 2 * kMaxActions * sizeof(unsigned long long);
    L.sq = o;
    o += kMaxStatic * 3 * sizeof(float);
    o = (o + 15) & ~size_t(15);
    L.nl_cap = 2 * threads;
    L.nl = o;
    o += (size_t)L.nl_cap * 7 * sizeof(float);
    L.total = (o + 127) & ~size_t(127);
    return L;
}

// cos / sin of k * 15 degrees from their surd forms (exact IEEE operations only).
__device__ void unit15(int k, double& ck, double& sk) {
    const double r2 = __dsqrt_rn(2.0), r3 = __dsqrt_rn(3.0), r6 = __dsqrt_rn(6.0);
    const double c15 = __ddiv_rn(__dadd_rn(r6, r2), 4.0), s15 = __ddiv_rn(__dsub_rn(r6, r2), 4.0);
    const int m = k % 6, quad = k / 6;
    double qc, qs;
    switch (m) {
        case 0: qc = 1.0; qs = 0.0; break;
        case 1: qc = c15; qs = s15; break;
        case 2: qc = __ddiv_rn(r3, 2.0); qs = 0.5; break;
        case 3: qc = __ddiv_rn(r2, 2.0); qs = __ddiv_rn(r2, 2.0); break;
        case 4: qc = 0.5; qs = __ddiv_rn(r3, 2.0); break;
        default: qc = s15; qs = c15; break;
    }
    if (quad == 0) { ck = qc; sk = qs; }
    else if (quad == 1) { ck = -qs; sk = qc; }
    else if (quad == 2) { ck = -qc; sk = -qs; }
    else { ck = qs; sk = -qc; }
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

__device__ __forceinline__ unsigned long long sum_term(float l, float ref) {
    const float t = exp2f(l - ref) * 1099511627776.0f;  // 2^40 fixed point
    return (unsigned long long)__float2ull_rn(t);
}

}  // namespace

__global__ void __launch_bounds__(512, 1) rollout_kernel(const __grid_constant__ RolloutArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const Model& m = a.m;
    const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31, warp = tid >> 5, NW = NT >> 5;
    const int cs = a.cs;
    const uint32_t rank = cs > 1 ? cluster_rank() : 0u;
    const int r = blockIdx.x / cs;
    if (r >= a.n_req) return;  // uniform over the cluster
    const fmdp_request req = a.reqs[r];
    const int A = m.A;
    const int chunk = a.chunk;
    const int c_begin = (int)rank * chunk;
    const int c_len = max(0, min(chunk, a.S_scan - c_begin));
    const Layout L = make_layout(chunk, NT);

    float* ring = reinterpret_cast<float*>(smem + L.ring);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bars);
    StepState* st = reinterpret_cast<StepState*>(smem + L.st);
    double* Dx = reinterpret_cast<double*>(smem + L.tabs);
    double* Dy = Dx + 24;
    double* Dz = Dy + 24;
    float* dx32 = reinterpret_cast<float*>(Dz + 32);
    float* dy32 = dx32 + 24;
    float* dz32 = dy32 + 24;
    int* keys = reinterpret_cast<int*>(smem + L.keys);                                   // [2][32]
    unsigned long long* sums = reinterpret_cast<unsigned long long*>(smem + L.sums);     // [2][32]
    float* sq = reinterpret_cast<float*>(smem + L.sq);                                   // [64][3]
    int* nl_slot = reinterpret_cast<int*>(smem + L.nl);
    float* nl_f = reinterpret_cast<float*>(nl_slot + L.nl_cap);  // 6 planes: qx qy qz vx vy vz
    const int NL = L.nl_cap;

    const bool lead = (rank == 0);
    float* traj = a.traj + (size_t)r * a.cap * 3;
    uint8_t* acts = a.acts + (size_t)r * a.cap;
    const int64_t t_lo = a.tab.t_base, t_hi = a.tab.t_base + a.tab.T_win;

    // ---- prologue: heading table (exact), action offsets, initial state
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
        Dx[tid] = __dmul_rn(step, C);
        Dy[tid] = __dmul_rn(step, S);
        dx32[tid] = (float)Dx[tid];
        dy32[tid] = (float)Dy[tid];
    }
    if (tid < kMaxActions) {
        const double dz = tid < A ? __dmul_rn(m.climb[tid], m.dt) : 0.0;
        Dz[tid] = dz;
        dz32[tid] = (float)dz;
        keys[tid] = keys[kMaxActions + tid] = float_key(-INFINITY);
        sums[tid] = sums[kMaxActions + tid] = 0ull;
    }
    if (tid == 0) {
        for (int e = 0; e < kRing; ++e) mbar_init(&bars[e], 1);
        mbar_fence_init();
        const double step = __dmul_rn(req.speed_mps, m.dt);
        st->step = step;
        st->cap2 = __dmul_rn(step, step);
        st->s[0] = req.ox; st->s[1] = req.oy; st->s[2] = req.oz;
        const double ex = __dsub_rn(req.gx, req.ox), ey = __dsub_rn(req.gy, req.oy), ez = __dsub_rn(req.gz, req.oz);
        st->e2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
        for (int i = 0; i < 3; ++i) {
            st->s_hi[i] = (float)st->s[i];
            st->s_lo[i] = (float)__dsub_rn(st->s[i], (double)st->s_hi[i]);
        }
        st->G[0] = (float)ex; st->G[1] = (float)ey; st->G[2] = (float)ez;
        st->Gn = sqrtf(st->G[0] * st->G[0] + st->G[1] * st->G[1] + st->G[2] * st->G[2]);
        st->h = 0;
        const bool captured = st->e2 <= st->cap2;
        st->done = captured || req.horizon <= 0;
        st->status = captured ? kStatusCaptured : FMDP_REJ_HORIZON;
        st->n_points = 1;
        st->near_ties = 0;
        st->steps = 0;
        st->abort_flag[0] = st->abort_flag[1] = 0;
        st->cnt[0] = st->cnt[1] = 0;
        if (lead) {
            traj[0] = (float)req.ox; traj[1] = (float)req.oy; traj[2] = (float)req.oz;
            if (a.trace && r == 0) {
                a.st_trace[0] = req.ox; a.st_trace[1] = req.oy; a.st_trace[2] = req.oz;
                a.hd_trace[0] = 0;
            }
        }
    }
    for (int w = tid; w < m.n_static; w += NT) {
        const double* c = m.statics + 6 * w;
        sq[3 * w] = (float)__dsub_rn(c[0], req.ox);
        sq[3 * w + 1] = (float)__dsub_rn(c[1], req.oy);
        sq[3 * w + 2] = (float)__dsub_rn(c[2], req.oz);
    }
    __syncthreads();

    // producer: slice j >= 1 (time depart + j) into ring entry (j - 1) % kRing; its mbarrier
    // phase parity is ((j - 1) / kRing) & 1
    const int64_t last_j = (int64_t)req.horizon + 1;
    auto entry_of = [](int64_t j) { return (int)((j - 1) % kRing); };
    auto parity_of = [](int64_t j) { return (uint32_t)(((j - 1) / kRing) & 1); };
    auto issue = [&](int64_t j) {
        const int e = entry_of(j);
        const int64_t T = req.depart_step + j;
        const bool valid = c_len > 0 && T >= t_lo && T < t_hi;
        st->ent_valid[e] = valid ? 1 : 0;
        if (valid) {
            int64_t row = T % a.tab.T_win;
            if (row < 0) row += a.tab.T_win;
            const size_t off = (size_t)row * a.tab.S_pad + c_begin;
            const uint32_t bytes = (uint32_t)c_len * 4u;
            float* dst = ring + (size_t)e * 3 * chunk;
            mbar_arrive_expect_tx(&bars[e], 3u * bytes);
            tma_bulk_load(dst, a.tab.X + off, bytes, &bars[e]);
            tma_bulk_load(dst + chunk, a.tab.Y + off, bytes, &bars[e]);
            tma_bulk_load(dst + 2 * chunk, a.tab.Z + off, bytes, &bars[e]);
        } else {
            mbar_arrive(&bars[e]);
        }
    };
    int64_t issued = 0;  // highest slice index issued (thread 0)
    int64_t waited = 0;  // highest slice index waited for (thread 0)
    if (tid == 0 && !st->done) {
        for (int64_t j = 1; j < kRing && j <= last_j; ++j) { issue(j); issued = j; }
    }

    // A staging wait that runs out (it never should) does not break the loop on its own:
    // the CTA flags it for this step, the flags of all CTAs are combined after the same
    // cluster barrier as the action values, and every CTA of the cluster then stops at the
    // same step, so the cluster barriers stay matched.
    int round = 0;
    bool stalled = false;
    for (int k = 0;; ++k) {
        if (tid == 0 && !st->done) {
            int timed_out = 0;
            if (!stalled) {
                const int64_t jn = (int64_t)k + kRing;
                if (jn <= last_j) { issue(jn); issued = jn; }
                const int64_t need = min((int64_t)k + 2, last_j);
                while (waited < need) {
                    const int64_t j = waited + 1;
                    if (!mbar_wait_bounded(&bars[entry_of(j)], parity_of(j))) {
                        timed_out = 1;
                        stalled = true;
                        atomicExch(a.err, FMDP_ERR_TIMEOUT);
                        for (int e = 0; e < kRing; ++e) st->ent_valid[e] = 0;
                        break;
                    }
                    waited = j;
                }
            } else {
                timed_out = 1;
            }
            st->abort_flag[k & 1] = timed_out;
        }
        __syncthreads();  // S1: state, ring entries and flags published
        if (st->done) break;

        const int e1 = entry_of(k + 1), e2 = entry_of(k + 2);
        const bool v1 = st->ent_valid[e1] != 0;
        const bool v2 = (k + 2 <= last_j) && st->ent_valid[e2] != 0;
        // acquire the async-proxy writes that the producer observed complete
        if (v1) mbar_test_wait(&bars[e1], parity_of(k + 1));
        if (v2) mbar_test_wait(&bars[e2], parity_of(k + 2));

        const int par = k & 1;
        const float shx = st->s_hi[0], shy = st->s_hi[1], shz = st->s_hi[2];
        const float slx = st->s_lo[0], sly = st->s_lo[1], slz = st->s_lo[2];
        const int h = st->h;
        const float dtf = (float)m.dt;
        const float stepf = (float)st->step;
        // cull radius without the plan's motion: max_k R_k + 1 m + largest successor offset
        float dzmax = 0.f;
        for (int i = 0; i < A; ++i) dzmax = fmaxf(dzmax, fabsf(dz32[i]));
        const float reach0 = m.reach_base + stepf + dzmax;

        // per-lane action constants
        int hn = 0;
        float dxa = 0.f, dya = 0.f, dza = 0.f;
        double DXa = 0.0, DYa = 0.0, DZa = 0.0;
        if (lane < A) {
            hn = ((h + m.dh[lane]) % 24 + 24) % 24;
            dxa = dx32[hn]; dya = dy32[hn]; dza = dz32[lane];
            DXa = Dx[hn]; DYa = Dy[hn]; DZa = Dz[lane];
        }
        float mloc = -INFINITY;
        unsigned long long sloc = 0ull;

        const float* X1 = ring + (size_t)e1 * 3 * chunk;
        const float* Y1 = X1 + chunk;
        const float* Z1 = Y1 + chunk;
        const float* X2 = ring + (size_t)e2 * 3 * chunk;
        const float* Y2 = X2 + chunk;
        const float* Z2 = Y2 + chunk;
        const int per_round = 2 * NT;
        const int scan_len = v1 ? c_len : 0;
        for (int base = 0; base < scan_len; base += per_round) {
            const int cpar = round & 1;
            // ---- cull
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int i = base + tid + u * NT;
                bool near = false;
                float qx = 0.f, qy = 0.f, qz = 0.f, vx = 0.f, vy = 0.f, vz = 0.f;
                if (i < scan_len) {
                    const float p1x = X1[i], p1y = Y1[i], p1z = Z1[i];
                    qx = (p1x - shx) - slx;
                    qy = (p1y - shy) - sly;
                    qz = (p1z - shz) - slz;
                    if (v2) {
                        const float p2x = X2[i];
                        if (p2x == p2x) {
                            vx = (p2x - p1x) / dtf;
                            vy = (Y2[i] - p1y) / dtf;
                            vz = (Z2[i] - p1z) / dtf;
                        }
                    }
                    const float vn = sqrtf(vx * vx + vy * vy + vz * vz);
                    const float reach = fmaf(m.tau_absmax, vn, reach0);
                    near = (qx * qx + qy * qy + qz * qz) < reach * reach;  // NaN: false
                }
                const unsigned mask = __ballot_sync(0xffffffffu, near);
                int pos0 = 0;
                if (lane == 0 && mask) pos0 = atomicAdd(&st->cnt[cpar], __popc(mask));
                pos0 = __shfl_sync(0xffffffffu, pos0, 0);
                if (near) {
                    const int pos = pos0 + __popc(mask & ((1u << lane) - 1u));
                    nl_slot[pos] = i;
                    nl_f[pos] = qx; nl_f[NL + pos] = qy; nl_f[2 * NL + pos] = qz;
                    nl_f[3 * NL + pos] = vx; nl_f[4 * NL + pos] = vy; nl_f[5 * NL + pos] = vz;
                }
            }
            __syncthreads();  // S2: near list complete
            const int n_near = st->cnt[cpar];
            if (tid == 0) st->cnt[cpar ^ 1] = 0;
            // ---- wells of near slots: warp per slot, lane per action
            for (int ei = warp; ei < n_near; ei += NW) {
                const float qx = nl_f[ei], qy = nl_f[NL + ei], qz = nl_f[2 * NL + ei];
                const float vx = nl_f[3 * NL + ei], vy = nl_f[4 * NL + ei], vz = nl_f[5 * NL + ei];
                if (lane < A) {
                    for (int w = 0; w < m.n_wells; ++w) {
                        const float tau = m.w_tau[w];
                        const float ex = dxa - fmaf(tau, vx, qx);
                        const float ey = dya - fmaf(tau, vy, qy);
                        const float ez = dza - fmaf(tau, vz, qz);
                        const float d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
                        const float R2 = m.w_R2[w], band = m.w_band[w];
                        if (d2 < R2 + band) {
                            bool inside = d2 < R2 - band;
                            if (!inside) {
                                const int i = nl_slot[ei];
                                const bool has2 = v2 && (X2[i] == X2[i]);
                                inside = well_inside_exact(m, st, DXa, DYa, DZa, X1[i], Y1[i], Z1[i],
                                                           has2 ? X2[i] : 0.f, has2 ? Y2[i] : 0.f,
                                                           has2 ? Z2[i] : 0.f, has2, w);
                            }
                            if (inside) {
                                const float l = fmaf(__fsqrt_rn(d2), m.w_lg[w], m.w_L[w]);
                                mloc = fmaxf(mloc, l);
                                if (m.combine) sloc += sum_term(l, m.sum_ref);
                            }
                        }
                    }
                }
            }
            ++round;
            __syncthreads();  // list consumed
        }
        // ---- static wells (restricted volumes / terrain peaks): CTA 0 of the cluster
        if (lead && m.n_static > 0 && lane < A) {
            for (int w = warp; w < m.n_static; w += NW) {
                const float ex = dxa - sq[3 * w], ey = dya - sq[3 * w + 1], ez = dza - sq[3 * w + 2];
                const float d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
                const float R2 = m.st_R2[w], band = m.st_band[w];
                if (d2 < R2 + band) {
                    bool inside = d2 < R2 - band;
                    if (!inside) inside = static_inside_exact(m, st, DXa, DYa, DZa, w);
                    if (inside) {
                        const float l = fmaf(__fsqrt_rn(d2), m.st_lg[w], m.st_L[w]);
                        mloc = fmaxf(mloc, l);
                        if (m.combine) sloc += sum_term(l, m.sum_ref);
                    }
                }
            }
        }
        if (lane < A) {
            if (mloc > -INFINITY) atomicMax(&keys[par * kMaxActions + lane], float_key(mloc));
            if (sloc) atomicAdd(&sums[par * kMaxActions + lane], sloc);
        }
        if (cs > 1) cluster_barrier(); else __syncthreads();  // S3: per-action partials complete

        // ---- combine, argmax, advance (warp 0 of every CTA, identical results)
        if (warp == 0) {
            const bool act = lane < A;
            int key = float_key(-INFINITY);
            unsigned long long ssum = 0ull;
            int any_abort = 0;
            if (lane < cs) {
                any_abort = cs > 1 ? dsmem_ld_s32(dsmem_addr(&st->abort_flag[par], lane)) : st->abort_flag[par];
            }
            any_abort = __any_sync(0xffffffffu, any_abort != 0);
            if (act) {
                if (cs > 1) {
                    for (int q = 0; q < cs; ++q) {
                        key = max(key, dsmem_ld_s32(dsmem_addr(&keys[par * kMaxActions + lane], q)));
                        if (m.combine) ssum += dsmem_ld_u64(dsmem_addr(&sums[par * kMaxActions + lane], q));
                    }
                } else {
                    key = keys[par * kMaxActions + lane];
                    ssum = sums[par * kMaxActions + lane];
                }
            }
            // penalty P of negative peaks (FP64 magnitude of the fp32 log-domain aggregate)
            double P = 0.0;
            if (m.combine) {
                P = (double)ssum * m.sum_scale;
            } else {
                const float Lp = key_float(key);
                if (Lp > -INFINITY) {
                    const float kf = floorf(Lp);
                    P = scale2((double)exp2f(Lp - kf), (int)kf);
                }
            }
            // successor (exact), validity (box)
            const double x = __dadd_rn(st->s[0], DXa), y = __dadd_rn(st->s[1], DYa), z = __dadd_rn(st->s[2], DZa);
            const bool valid = act && x >= m.box[0] && x <= m.box[3] && y >= m.box[1] && y <= m.box[4] &&
                               z >= m.box[2] && z <= m.box[5];
            // goal distance change Delta = |G - delta| - |G| in fp32 (G = goal - s)
            const float gX = st->G[0], gY = st->G[1], gZ = st->G[2], gN = st->Gn;
            const float fx = gX - dxa, fy = gY - dya, fz = gZ - dza;
            const float da = sqrtf(fx * fx + fy * fy + fz * fz);
            const float num = (dxa * dxa + dya * dya + dza * dza) - 2.0f * (gX * dxa + gY * dya + gZ * dza);
            const float den = da + gN;
            const float Dlt = den > 0.f ? num / den : 0.f;
            // hard deck: terrain clearance at the successor
            double V = 0.0;
            if (m.hm && act) {
                const float gxf = (float)__dsub_rn(x, m.box[0]) * m.hm_sx;
                const float gyf = (float)__dsub_rn(y, m.box[1]) * m.hm_sy;
                int ix = (int)floorf(gxf), iy = (int)floorf(gyf);
                ix = min(max(ix, 0), m.hm_nx - 2);
                iy = min(max(iy, 0), m.hm_ny - 2);
                const float ax = gxf - (float)ix, ay = gyf - (float)iy;
                const float* r0 = m.hm + (size_t)iy * m.hm_nx + ix;
                const float h00 = __ldg(r0), h10 = __ldg(r0 + 1), h01 = __ldg(r0 + m.hm_nx), h11 = __ldg(r0 + m.hm_nx + 1);
                const float hz = (1.f - ay) * ((1.f - ax) * h00 + ax * h10) + ay * ((1.f - ax) * h01 + ax * h11);
                const float c = (float)z - hz;
                const float clr = (float)m.clearance;
                if (fabsf(c - clr) < kClrBand) {
                    const double c64 = __dsub_rn(z, terrain64(m, x, y));
                    V = c64 < m.clearance ? __dsub_rn(m.deck, c64) : 0.0;
                } else if (c < clr) {
                    V = m.deck - (double)c;
                }
            }
            const double N = P + V;
            const unsigned pen = __ballot_sync(0xffffffffu, valid && N > 0.0);
            const bool full = a.trace || pen != 0u || !(m.goal_reward > 0.0);
            int best = 99, second = 99;
            bool tie = false;
            double Qa = -INFINITY;
            if (!full) {
                // all valid successors are free of penalties: Q = g is decreasing in the goal distance
                float kb = valid ? Dlt : INFINITY;
                int ib = valid ? lane : 99;
                for (int off = 16; off; off >>= 1) {
                    const float ok = __shfl_xor_sync(0xffffffffu, kb, off);
                    const int oi = __shfl_xor_sync(0xffffffffu, ib, off);
                    if (ok < kb || (ok == kb && oi < ib)) { kb = ok; ib = oi; }
                }
                best = ib;
                float k2 = (valid && lane != best) ? Dlt : INFINITY;
                int i2 = (valid && lane != best) ? lane : 99;
                for (int off = 16; off; off >>= 1) {
                    const float ok = __shfl_xor_sync(0xffffffffu, k2, off);
                    const int oi = __shfl_xor_sync(0xffffffffu, i2, off);
                    if (ok < k2 || (ok == k2 && oi < i2)) { k2 = ok; i2 = oi; }
                }
                second = i2;
                if (best < 99 && second < 99) {
                    const float gap = 1.0f - exp2f(-(k2 - kb) * fabsf(m.lg32));
                    tie = gap < (float)kTieRel;
                }
            } else {
                // full FP64 values: g = 2^(Lg0 + Delta * log2 gamma), Lg0 from the exact |goal - s|
                double Lg0 = 0.0;
                if (lane == 0) Lg0 = m.log2rg + __dsqrt_rn(st->e2) * m.lg64;
                Lg0 = __shfl_sync(0xffffffffu, Lg0, 0);
                double g = 0.0;
                if (m.goal_reward > 0.0) {
                    const double n0 = floor(Lg0);
                    const float phi = (float)(Lg0 - n0);
                    g = scale2((double)exp2f(fmaf(Dlt, m.lg32, phi)), (int)n0);
                }
                Qa = valid ? __dsub_rn(__dsub_rn(g, P), V) : -INFINITY;
                const double T = fmax(g, N);
                double qb = valid ? Qa : -INFINITY;
                int ib = valid ? lane : 99;
                for (int off = 16; off; off >>= 1) {
                    const double oq = __shfl_xor_sync(0xffffffffu, qb, off);
                    const int oi = __shfl_xor_sync(0xffffffffu, ib, off);
                    if (oq > qb || (oq == qb && oi < ib)) { qb = oq; ib = oi; }
                }
                best = ib;
                double q2 = (valid && lane != best) ? Qa : -INFINITY;
                int i2 = (valid && lane != best) ? lane : 99;
                for (int off = 16; off; off >>= 1) {
                    const double oq = __shfl_xor_sync(0xffffffffu, q2, off);
                    const int oi = __shfl_xor_sync(0xffffffffu, i2, off);
                    if (oq > q2 || (oq == q2 && oi < i2)) { q2 = oq; i2 = oi; }
                }
                second = i2;
                if (best < 99 && second < 99) {
                    const double T1 = __shfl_sync(0xffffffffu, T, best);
                    const double T2 = __shfl_sync(0xffffffffu, T, second);
                    const double sc = fmax(fmax(fabs(qb), fabs(q2)), fmax(T1, T2));
                    tie = (qb - q2) < kTieRel * sc;
                }
                if (a.trace && lead && r == 0 && act) a.q_trace[(size_t)k * A + lane] = Qa;
            }
            if (any_abort) {
                if (lane == 0) { st->done = 1; st->status = FMDP_REJ_NO_ACTION; st->steps = k; }
            } else if (best >= 99) {
                if (lane == 0) { st->done = 1; st->status = FMDP_REJ_NO_ACTION; st->steps = k; }
            } else {
                const double nx = __shfl_sync(0xffffffffu, x, best);
                const double ny = __shfl_sync(0xffffffffu, y, best);
                const double nz = __shfl_sync(0xffffffffu, z, best);
                const int nh = __shfl_sync(0xffffffffu, hn, best);
                if (lane == 0) {
                    st->s[0] = nx; st->s[1] = ny; st->s[2] = nz;
                    st->h = nh;
                    const double ex = __dsub_rn(req.gx, nx), ey = __dsub_rn(req.gy, ny), ez = __dsub_rn(req.gz, nz);
                    const double e2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
                    st->e2 = e2;
                    st->s_hi[0] = (float)nx; st->s_hi[1] = (float)ny; st->s_hi[2] = (float)nz;
                    st->s_lo[0] = (float)__dsub_rn(nx, (double)st->s_hi[0]);
                    st->s_lo[1] = (float)__dsub_rn(ny, (double)st->s_hi[1]);
                    st->s_lo[2] = (float)__dsub_rn(nz, (double)st->s_hi[2]);
                    const float Gx = (float)ex, Gy = (float)ey, Gz = (float)ez;
                    st->G[0] = Gx; st->G[1] = Gy; st->G[2] = Gz;
                    st->Gn = sqrtf(Gx * Gx + Gy * Gy + Gz * Gz);
                    const int np = st->n_points;
                    st->n_points = np + 1;
                    if (tie) st->near_ties += 1;
                    const bool captured = e2 <= st->cap2;
                    const bool last = (k + 1) >= req.horizon;
                    st->done = captured || last;
                    st->status = captured ? kStatusCaptured : FMDP_REJ_HORIZON;
                    st->steps = k + 1;
                    if (lead) {
                        traj[3 * np] = (float)nx; traj[3 * np + 1] = (float)ny; traj[3 * np + 2] = (float)nz;
                        acts[k] = (uint8_t)best;
                        if (a.trace && r == 0) {
                            a.st_trace[3 * np] = nx; a.st_trace[3 * np + 1] = ny; a.st_trace[3 * np + 2] = nz;
                            a.hd_trace[np] = nh;
                            a.tie_trace[k] = tie ? 1 : 0;
                        }
                    }
                }
                for (int w = lane; w < m.n_static; w += 32) {
                    const double* c = m.statics + 6 * w;
                    sq[3 * w] = (float)__dsub_rn(c[0], nx);
                    sq[3 * w + 1] = (float)__dsub_rn(c[1], ny);
                    sq[3 * w + 2] = (float)__dsub_rn(c[2], nz);
                }
            }
            if (act) {
                keys[(par ^ 1) * kMaxActions + lane] = float_key(-INFINITY);
                sums[(par ^ 1) * kMaxActions + lane] = 0ull;
            }
        }
    }

    // drain: every issued copy must land before the CTA exits
    if (tid == 0) {
        while (waited < issued) {
            const int64_t j = waited + 1;
            if (!mbar_wait_bounded(&bars[entry_of(j)], parity_of(j))) {
                atomicExch(a.err, FMDP_ERR_TIMEOUT);
                break;
            }
            waited = j;
        }
        if (lead) {
            RolloutOut o;
            o.n_points = st->n_points;
            o.status = st->status;
            o.near_ties = st->near_ties;
            o.steps = st->steps;
            a.out[r] = o;
        }
    }
    if (cs > 1) cluster_barrier();  // peers may still read this CTA's shared memory
}

size_t rollout_smem_bytes(int chunk, int threads) { return make_layout(chunk, threads).total; }

cudaError_t prepare_rollout_kernel(size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(rollout_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(rollout_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

int rollout_max_active_clusters(int cs, int threads, size_t smem) {
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
    if (cudaOccupancyMaxActiveClusters(&n, rollout_kernel, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t launch_rollout(const RolloutArgs& a, int threads, size_t smem, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(a.n_req * a.cs), 1, 1);
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
    return cudaLaunchKernelEx(&cfg, rollout_kernel, a);
}

}  // namespace fmdp
