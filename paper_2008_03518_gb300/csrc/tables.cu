// Plan-table kernels: separation check, FCFS admission and table maintenance (sm_103a).
//
// sep_check is the paper's terminal test applied to a finished trajectory (Sec. IV
// "Determine terminal state", Sec. V): every sample at time step t0 + k is compared with
// every known plan's sample at the same step; a pair is a conflict when the horizontal
// distance is below horiz_m and the vertical distance below vert_m, and a sample below
// the terrain surface is a terrain collision. The kernel streams each slice row once
// (coalesced float4 loads, 12 bytes per slot), so it is bound by HBM bandwidth.
#include <climits>

#include "fmdp_internal.cuh"

namespace fmdp {

namespace {

constexpr int kSepThreads = 256;
constexpr int kSepSlotsPerThread = 4;
constexpr int kSepSlotsPerCta = kSepThreads * kSepSlotsPerThread;

__device__ __forceinline__ int64_t ring_row(int64_t T, int32_t T_win) {
    int64_t r = T % T_win;
    return r < 0 ? r + T_win : r;
}

}  // namespace

__global__ void __launch_bounds__(kSepThreads) sepcheck_kernel(const __grid_constant__ SepArgs a) {
    if (a.n_dev && (int)blockIdx.z >= *a.n_dev) return;
    const int r = a.idx ? a.idx[blockIdx.z] : (int)blockIdx.z;
    const int k = blockIdx.x;
    const int n = a.rout ? a.rout[r].n_points : a.n_fixed;
    if (k >= n) return;
    const int64_t t0 = a.reqs ? a.reqs[r].depart_step : a.t0_fixed;
    const float* p = a.traj + ((size_t)r * a.cap + k) * 3;
    const float px = p[0], py = p[1], pz = p[2];
    SepOut* out = a.out + r;
    const Model& m = a.m;

    if (blockIdx.y == 0 && threadIdx.x == 0 && m.hm) {
        if ((double)pz < terrain64(m, (double)px, (double)py)) atomicMin(&out->first_terrain, k);
    }
    const int64_t T = t0 + k;
    if (T < a.tab.t_base || T >= a.tab.t_base + a.tab.T_win) return;
    const size_t rowoff = (size_t)ring_row(T, a.tab.T_win) * a.tab.S_pad;

    const float H = (float)m.sep_h, Vm = (float)m.sep_v;
    const float H2 = H * H;
    const float hband = 2.0f * H * kSepBand + kSepBand * kSepBand;
    const double H2d = __dmul_rn(m.sep_h, m.sep_h);

    int first = INT_MAX;
    unsigned cnt = 0;
    float minh = INFINITY, minv = INFINITY;
    const int s0 = (blockIdx.y * kSepThreads + threadIdx.x) * kSepSlotsPerThread;
    if (s0 < a.S_scan) {
        const float4 X4 = *reinterpret_cast<const float4*>(a.tab.X + rowoff + s0);
        const float4 Y4 = *reinterpret_cast<const float4*>(a.tab.Y + rowoff + s0);
        const float4 Z4 = *reinterpret_cast<const float4*>(a.tab.Z + rowoff + s0);
        const float qx[4] = {X4.x, X4.y, X4.z, X4.w};
        const float qy[4] = {Y4.x, Y4.y, Y4.z, Y4.w};
        const float qz[4] = {Z4.x, Z4.y, Z4.z, Z4.w};
#pragma unroll
        for (int u = 0; u < kSepSlotsPerThread; ++u) {
            const float dx = px - qx[u], dy = py - qy[u];
            const float dz = fabsf(pz - qz[u]);
            const float h2 = dx * dx + dy * dy;
            bool hin = h2 < H2;  // NaN (empty slot): false
            bool vin = dz < Vm;
            if (fabsf(h2 - H2) < hband) {
                const double ex = __dsub_rn((double)px, (double)qx[u]);
                const double ey = __dsub_rn((double)py, (double)qy[u]);
                hin = __dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)) < H2d;
            }
            if (fabsf(dz - Vm) < kSepBand) vin = fabs(__dsub_rn((double)pz, (double)qz[u])) < m.sep_v;
            if (vin) minh = fminf(minh, sqrtf(h2));
            if (hin) {
                minv = fminf(minv, dz);
                if (vin) { ++cnt; first = k; }
            }
        }
    }
    // warp reduction, then one atomic per warp and quantity
    for (int off = 16; off; off >>= 1) {
        first = min(first, __shfl_xor_sync(0xffffffffu, first, off));
        cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
        minh = fminf(minh, __shfl_xor_sync(0xffffffffu, minh, off));
        minv = fminf(minv, __shfl_xor_sync(0xffffffffu, minv, off));
    }
    if ((threadIdx.x & 31) == 0) {
        if (cnt) {
            atomicAdd(&out->conflicts, (unsigned long long)cnt);
            atomicMin(&out->first_conflict, first);
        }
        if (minh < INFINITY) atomicMin(&out->min_h_bits, __float_as_uint(minh));
        if (minv < INFINITY) atomicMin(&out->min_v_bits, __float_as_uint(minv));
    }
}

__global__ void sep_reset_kernel(SepOut* out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        SepOut o;
        o.first_conflict = INT_MAX;
        o.first_terrain = INT_MAX;
        o.conflicts = 0ull;
        o.min_h_bits = 0x7f800000u;
        o.min_v_bits = 0x7f800000u;
        o.verdict = -1;
        o.pad = 0;
        out[i] = o;
    }
}

// FCFS admission (Sec. V): the verdict of request r is decided on the device from its
// rollout status and separation check; an admitted trajectory is scattered into its
// slot column. In force mode, known plans are stored unconditionally.
__global__ void admit_kernel(const __grid_constant__ AdmitArgs a) {
    if (a.n_dev && (int)blockIdx.y >= *a.n_dev) return;
    const int r = a.idx ? a.idx[blockIdx.y] : (int)blockIdx.y;
    const int slot = a.slots[r];  // per request (index mode) or per work item (pointer-offset mode)
    int n;
    int64_t t0;
    size_t off;
    if (a.force) {
        n = a.counts[r];
        t0 = a.t0s[r];
        off = (size_t)a.offs[r];
    } else {
        const RolloutOut ro = a.rout[r];
        SepOut* so = a.sep + r;
        int verdict;
        if (ro.status != kStatusCaptured) verdict = ro.status;
        else if (so->first_conflict != INT_MAX) verdict = FMDP_REJ_CONFLICT;
        else if (so->first_terrain != INT_MAX) verdict = FMDP_REJ_TERRAIN;
        else verdict = FMDP_ADMITTED;
        if (blockIdx.x == 0 && threadIdx.x == 0) so->verdict = verdict;
        if (verdict != FMDP_ADMITTED) return;
        n = ro.n_points;
        t0 = a.reqs[r].depart_step;
        off = (size_t)r * a.cap;
    }
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const size_t row = (size_t)ring_row(t0 + k, a.tab.T_win) * a.tab.S_pad + slot;
        const float* p = a.traj + (off + k) * 3;
        a.tab.X[row] = p[0];
        a.tab.Y[row] = p[1];
        a.tab.Z[row] = p[2];
    }
}

__global__ void fill_nan_kernel(float* p, size_t n) {
    const float nanv = __int_as_float(0x7fc00000);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        p[i] = nanv;
}

cudaError_t launch_sepcheck(const SepArgs& a, int n_req, int max_points, cudaStream_t s) {
    if (n_req <= 0 || max_points <= 0) return cudaSuccess;
    const int tiles = a.S_scan > 0 ? (a.S_scan + kSepSlotsPerCta - 1) / kSepSlotsPerCta : 1;
    for (int r0 = 0; r0 < n_req; r0 += 65535) {
        SepArgs b = a;
        const int nr = min(65535, n_req - r0);
        if (a.idx) {
            b.idx = a.idx + r0;  // work items are mapped to requests; n_dev caps the total
            if (r0 > 0 && a.n_dev) return cudaErrorInvalidValue;
        } else {
            b.traj = a.traj + (size_t)r0 * a.cap * 3;
            if (a.rout) b.rout = a.rout + r0;
            if (a.reqs) b.reqs = a.reqs + r0;
            b.out = a.out + r0;
        }
        sepcheck_kernel<<<dim3((unsigned)max_points, (unsigned)tiles, (unsigned)nr), kSepThreads, 0, s>>>(b);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_sep_reset(SepOut* out, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    sep_reset_kernel<<<(n + 255) / 256, 256, 0, s>>>(out, n);
    return cudaGetLastError();
}

cudaError_t launch_admit(const AdmitArgs& a, int n_req, int max_points, cudaStream_t s) {
    if (n_req <= 0 || max_points <= 0) return cudaSuccess;
    const int bx = min((max_points + 255) / 256, 64);
    for (int r0 = 0; r0 < n_req; r0 += 65535) {
        AdmitArgs b = a;
        const int nr = min(65535, n_req - r0);
        if (a.idx) {
            if (r0 > 0) return cudaErrorInvalidValue;
            admit_kernel<<<dim3((unsigned)bx, (unsigned)nr), 256, 0, s>>>(b);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            continue;
        }
        b.slots = a.slots + r0;
        if (a.force) {
            b.t0s = a.t0s + r0;
            b.counts = a.counts + r0;
            b.offs = a.offs + r0;
        } else {
            b.traj = a.traj + (size_t)r0 * a.cap * 3;
            b.rout = a.rout + r0;
            b.reqs = a.reqs + r0;
            b.sep = a.sep + r0;
        }
        admit_kernel<<<dim3((unsigned)bx, (unsigned)nr), 256, 0, s>>>(b);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Influence of request j's speculative trajectory on request k's (j before k in arrival
// order). k's plan could differ from its speculative one only if some state of k lies
// within reach of a well of j one step later (|s_k(t) - p_j(t+1)| < max R + |tau|max |v_j|
// + successor offset + margin), and its verdict only if its origin conflicts with j. A
// conservative test: a false positive costs one more speculative round, never a result.
__global__ void __launch_bounds__(128) influence_kernel(const __grid_constant__ InfluenceArgs a) {
    const int n = *a.n_dev;
    const int w = blockIdx.x, v = blockIdx.y;  // k = item w, j = item v
    if (w >= n || v >= n) return;
    const int k = a.idx[w], j = a.idx[v];
    __shared__ int hit;
    if (threadIdx.x == 0) hit = 0;
    __syncthreads();
    if (j < k) {
        const int nk = a.rout[k].n_points, nj = a.rout[j].n_points;
        const int64_t tk = a.reqs[k].depart_step, tj = a.reqs[j].depart_step;
        const float rho = (float)(a.reqs[k].speed_mps * a.dt) + a.dzmax + 1.0f;
        const float* pk = a.traj + (size_t)k * a.cap * 3;
        const float* pj = a.traj + (size_t)j * a.cap * 3;
        // origin conflict (verdict only): j at k's departure step
        if (threadIdx.x == 0) {
            const int64_t i0 = tk - tj;
            if (i0 >= 0 && i0 < nj) {
                const float dx = pk[0] - pj[3 * i0], dy = pk[1] - pj[3 * i0 + 1], dz = pk[2] - pj[3 * i0 + 2];
                if (dx * dx + dy * dy < (a.sep_h + 1.f) * (a.sep_h + 1.f) && fabsf(dz) < a.sep_v + 1.f) hit = 1;
            }
        }
        // wells of j at t+1 against k's state at t, for every state of k
        for (int i = threadIdx.x; i < nk && !hit; i += blockDim.x) {
            const int64_t t1 = tk + i + 1 - tj;  // index of j's sample at t+1
            if (t1 < 0 || t1 >= nj) continue;
            const float* q1 = pj + 3 * t1;
            float vx = 0.f, vy = 0.f, vz = 0.f;
            if (t1 + 1 < nj) {
                vx = (q1[3] - q1[0]) / a.dt;
                vy = (q1[4] - q1[1]) / a.dt;
                vz = (q1[5] - q1[2]) / a.dt;
            }
            const float reach = a.reach_base + a.tau_absmax * sqrtf(vx * vx + vy * vy + vz * vz) + rho;
            const float dx = pk[3 * i] - q1[0], dy = pk[3 * i + 1] - q1[1], dz = pk[3 * i + 2] - q1[2];
            if (dx * dx + dy * dy + dz * dz < reach * reach) hit = 1;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) a.out[(size_t)w * a.n_cap + v] = (uint8_t)hit;
}

__global__ void sep_reset_idx_kernel(SepOut* out, const int32_t* idx, const int32_t* n_dev, int n_max) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= n_max || w >= *n_dev) return;
    SepOut o;
    o.first_conflict = INT_MAX;
    o.first_terrain = INT_MAX;
    o.conflicts = 0ull;
    o.min_h_bits = 0x7f800000u;
    o.min_v_bits = 0x7f800000u;
    o.verdict = -1;
    o.pad = 0;
    out[idx[w]] = o;
}

cudaError_t launch_influence(const InfluenceArgs& a, int n_max, int /*max_points*/, cudaStream_t s) {
    if (n_max <= 0) return cudaSuccess;
    influence_kernel<<<dim3((unsigned)n_max, (unsigned)n_max), 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sep_reset_idx(SepOut* out, const int32_t* idx, const int32_t* n_dev, int n_max, cudaStream_t s) {
    if (n_max <= 0) return cudaSuccess;
    sep_reset_idx_kernel<<<(n_max + 255) / 256, 256, 0, s>>>(out, idx, n_dev, n_max);
    return cudaGetLastError();
}

cudaError_t launch_fill_nan(float* p, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const size_t want = (n + 255) / 256;
    const size_t blocks = want < (size_t)(152 * 16) ? want : (size_t)(152 * 16);
    fill_nan_kernel<<<(unsigned)blocks, 256, 0, s>>>(p, n);
    return cudaGetLastError();
}

}  // namespace fmdp
