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
#include "sep_pair.cuh"

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

// Grid: x strides over the trajectory's samples (one block per sample when gridDim.x covers
// them all), y over 1024-slot tiles, z over requests.
__global__ void __launch_bounds__(kSepThreads) sepcheck_kernel(const __grid_constant__ SepArgs a) {
    if (a.n_dev && (int)blockIdx.z >= *a.n_dev) return;
    const int r = a.idx ? a.idx[blockIdx.z] : (int)blockIdx.z;
    const int n = a.rout ? a.rout[r].n_points : a.n_fixed;
    const int64_t t0 = a.reqs ? a.reqs[r].depart_step : a.t0_fixed;
    SepOut* out = a.out + r;
    const Model& m = a.m;
    const SepConsts sk = sep_consts(m.sep_h, m.sep_v);
    const int s0 = (blockIdx.y * kSepThreads + threadIdx.x) * kSepSlotsPerThread;

    // terrain collision (z below the surface): the first tile's blocks, one sample per
    // thread; fp32 outside a band around the surface, FP64 inside it
    if (blockIdx.y == 0 && m.hm) {
        int tfirst = INT_MAX;
        for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
            const float* p = a.traj + ((size_t)r * a.cap + k) * 3;
            const float c = p[2] - terrain32(m, p[0], p[1]);
            bool below = c < 0.f;
            if (fabsf(c) < kTerrBand) below = below_terrain_exact(m, p[0], p[1], p[2]);
            if (below) tfirst = min(tfirst, k);
        }
        for (int off = 16; off; off >>= 1) tfirst = min(tfirst, __shfl_xor_sync(0xffffffffu, tfirst, off));
        if ((threadIdx.x & 31) == 0 && tfirst != INT_MAX) atomicMin(&out->first_terrain, tfirst);
    }

    int first = INT_MAX;
    unsigned cnt = 0;
    float minh = INFINITY, minv = INFINITY;
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
    const float* p = a.traj + ((size_t)r * a.cap + k) * 3;
    const float px = p[0], py = p[1], pz = p[2];
    const int64_t T = t0 + k;
    if (T < a.tab.t_base || T >= a.tab.t_base + a.tab.T_win) continue;
    const size_t rowoff = (size_t)ring_row(T, a.tab.T_win) * a.tab.S_pad;
    if (s0 < a.S_scan) {
        const float4 X4 = *reinterpret_cast<const float4*>(a.tab.X + rowoff + s0);
        const float4 Y4 = *reinterpret_cast<const float4*>(a.tab.Y + rowoff + s0);
        const float4 Z4 = *reinterpret_cast<const float4*>(a.tab.Z + rowoff + s0);
        const float qx[4] = {X4.x, X4.y, X4.z, X4.w};
        const float qy[4] = {Y4.x, Y4.y, Y4.z, Y4.w};
        const float qz[4] = {Z4.x, Z4.y, Z4.z, Z4.w};
#pragma unroll
        for (int u = 0; u < kSepSlotsPerThread; ++u) {
            float h2, dz;
            bool hin, vin;
            sep_pair(sk, px, py, pz, qx[u], qy[u], qz[u], h2, dz, hin, vin);
            if (vin) minh = fminf(minh, sqrtf(h2));
            if (hin) {
                minv = fminf(minv, dz);
                if (vin) { ++cnt; first = min(first, k); }
            }
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
    if (a.err && *(volatile const int32_t*)a.err != 0) return;  // a call whose wait expired stores nothing
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
    if (a.slot_ord && blockIdx.x == 0 && threadIdx.x == 0) a.slot_ord[slot] = a.ord;
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

// Row-major separation check (batch waves). Each block gathers the work items' samples at
// its step into shared memory, one thread per sample, then streams the row's plan samples
// through shared memory in tiles; a thread keeps its sample's count, minima and conflict
// flag in registers (the minimum horizontal distance as a squared distance: the square
// root is monotone, so the root of the minimum is the minimum of the roots) and folds them
// into its request's report once at the end.
constexpr int kRowThreads = 256;
constexpr int kRowTile = 2048;

size_t sepcheck_rows_smem(int n_max) {
    return (size_t)kRowTile * (sizeof(float4) + sizeof(int)) + (size_t)n_max * (sizeof(float4) + 3 * sizeof(int)) +
           16;
}

__global__ void __launch_bounds__(kRowThreads) sepcheck_rows_kernel(const __grid_constant__ SepRowsArgs a) {
    extern __shared__ __align__(16) unsigned char srm[];
    float4* tile = reinterpret_cast<float4*>(srm);
    float4* pts = tile + kRowTile;
    int* pr = reinterpret_cast<int*>(pts + a.n_max);
    int* pk = pr + a.n_max;
    int* po = pk + a.n_max;       // ordinal of the sample's request (ordinal filter)
    int* tord = po + a.n_max;     // [kRowTile] ordinal of the tile's items' slots
    int* npts_s = tord + kRowTile;
    const int tid = threadIdx.x, NT = blockDim.x;
    const int32_t W = a.tab.T_win;
    const int64_t T = a.tab.t_base + a.row0 + blockIdx.x;
    int64_t row = T % W;
    if (row < 0) row += W;
    if (tid == 0) *npts_s = 0;
    __syncthreads();
    const int n = *a.n_dev;
    for (int w = tid; w < n; w += NT) {
        const int r = a.idx[w];
        if (a.skip && a.skip[r]) continue;
        const int64_t d = a.reqs[r].depart_step;
        const int np = a.rout[r].n_points;
        if (T >= d && T < d + np) {
            const int q = atomicAdd(npts_s, 1);
            const int k = (int)(T - d);
            const float* p = a.traj + ((size_t)r * a.cap + k) * 3;
            pts[q] = make_float4(p[0], p[1], p[2], 0.f);
            pr[q] = r;
            pk[q] = k;
            po[q] = a.slot_ord ? a.req_ord[r] : 0;
        }
    }
    __syncthreads();
    const int npts = *npts_s;
    if (npts == 0) return;
    const Model& m = a.m;
    const SepConsts sk = sep_consts(m.sep_h, m.sep_v);
    // terrain collision of each sample (fp32 outside a band, FP64 inside)
    if (m.hm) {
        for (int q = tid; q < npts; q += NT) {
            const float4 P = pts[q];
            const float c = P.z - terrain32(m, P.x, P.y);
            bool below = c < 0.f;
            if (fabsf(c) < kTerrBand) below = below_terrain_exact(m, P.x, P.y, P.z);
            if (below) atomicMin(&a.out[pr[q]].first_terrain, pk[q]);
        }
    }
    // plan samples of the row: index items (one per finite sample) or the table planes
    int nslots;
    const float4* it = nullptr;
    if (a.items) {
        const int32_t* cs_row = a.cstart + row * (int64_t)(a.ncell + 1);
        nslots = cs_row[a.ncell] + a.nextra[row];
        it = a.items + (size_t)row * a.tab.S_pad * 2;
    } else {
        nslots = a.S_scan;
    }
    const size_t poff = (size_t)row * a.tab.S_pad;
    // thread t: sample pg + t % P of the current group of P samples, slots of group t / P
    // (G = NT / P groups share out each tile); lanes of a warp read the same slot
    for (int pg = 0; pg < npts; pg += NT) {
        const int P = min(NT, npts - pg);
        const int G = NT / P;
        const int q = pg + tid % P, g = tid / P;
        const bool act = g < G;
        const float4 P4 = act ? pts[q] : make_float4(0.f, 0.f, 0.f, 0.f);
        const int my_ord = act ? po[q] : 0;
        const bool filt = a.slot_ord != nullptr && it != nullptr;
        unsigned cnt = 0;
        float minh2 = INFINITY, minv = INFINITY;
        for (int s0 = 0; s0 < nslots; s0 += kRowTile) {
            const int tn = min(kRowTile, nslots - s0);
            __syncthreads();
            for (int j = tid; j < tn; j += NT) {
                if (it) {
                    const float4 Q = it[2 * (size_t)(s0 + j)];
                    tile[j] = Q;
                    if (filt) {  // the ordinal of the item's plan: a stored plan's slot ordinal, a
                                 // tentative plan's own; a withdrawn item is never counted
                        const int tag = __float_as_int(Q.w);
                        tord[j] = tag >= 0 ? ((unsigned)tag < (unsigned)a.tab.S_pad ? a.slot_ord[tag] : INT_MIN)
                                           : (tag == kTagDead ? INT_MAX : -tag - 2);
                    }
                } else {
                    const size_t o = poff + s0 + j;
                    tile[j] = make_float4(a.tab.X[o], a.tab.Y[o], a.tab.Z[o], 0.f);
                }
            }
            __syncthreads();
            if (act) {
#pragma unroll 4
                for (int j = g; j < tn; j += G) {
                    const float4 Q = tile[j];
                    if (filt && tord[j] >= my_ord) continue;  // admitted after this request
                    float h2, dz;
                    bool hin, vin;
                    sep_pair(sk, P4.x, P4.y, P4.z, Q.x, Q.y, Q.z, h2, dz, hin, vin);
                    if (vin) minh2 = fminf(minh2, h2);
                    if (hin) {
                        minv = fminf(minv, dz);
                        cnt += vin ? 1u : 0u;
                    }
                }
            }
        }
        if (act) {
            SepOut* o = a.out + pr[q];
            if (cnt) {
                atomicAdd(&o->conflicts, (unsigned long long)cnt);
                atomicMin(&o->first_conflict, pk[q]);
            }
            if (minh2 < INFINITY) atomicMin(&o->min_h_bits, __float_as_uint(sqrtf(minh2)));
            if (minv < INFINITY) atomicMin(&o->min_v_bits, __float_as_uint(minv));
        }
    }
}

cudaError_t prepare_sepcheck_rows(size_t smem) {
    return cudaFuncSetAttribute(sepcheck_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_sepcheck_rows(const SepRowsArgs& a, cudaStream_t s) {
    const int32_t rows = a.nrows > 0 ? a.nrows : a.tab.T_win;
    if (a.row0 < 0 || a.row0 + rows > a.tab.T_win) return cudaErrorInvalidValue;
    sepcheck_rows_kernel<<<(unsigned)rows, kRowThreads, sepcheck_rows_smem(a.n_max), s>>>(a);
    return cudaGetLastError();
}

// Minimum separations of each request of a batch to the requests admitted before it in the
// same batch (at common steps), folded into its separation report. A request's plan and
// verdict are final once no earlier admission influences it, but its minimum distances
// to plans far away still see every earlier admission, as a sequential run would.
__global__ void __launch_bounds__(256) batch_minsep_kernel(const __grid_constant__ MinSepArgs a) {
    if ((int)blockIdx.x >= a.n) return;
    const int k = a.k0 + (int)blockIdx.x;
    const SepConsts sk = sep_consts(a.sep_h, a.sep_v);
    const int nk = a.rout[k].n_points;
    const int64_t tk = a.reqs[k].depart_step;
    const float* pk = a.traj + (size_t)k * a.cap * 3;
    float minh = INFINITY, minv = INFINITY;
    for (int q = 0; q < a.n_adm; ++q) {
        const int j = a.adm[q];
        if (j >= k) break;  // admitted requests in arrival order
        const int nj = a.rout[j].n_points;
        const int64_t tj = a.reqs[j].depart_step;
        const float* pj = a.traj + (size_t)j * a.cap * 3;
        const int64_t lo = max(tk, tj), hi = min(tk + nk, tj + nj);
        for (int64_t t = lo + threadIdx.x; t < hi; t += blockDim.x) {
            const float* p = pk + 3 * (t - tk);
            const float* q3 = pj + 3 * (t - tj);
            float h2, dz;
            bool hin, vin;
            sep_pair(sk, p[0], p[1], p[2], q3[0], q3[1], q3[2], h2, dz, hin, vin);
            if (vin) minh = fminf(minh, sqrtf(h2));
            if (hin) minv = fminf(minv, dz);
        }
    }
    for (int off = 16; off; off >>= 1) {
        minh = fminf(minh, __shfl_xor_sync(0xffffffffu, minh, off));
        minv = fminf(minv, __shfl_xor_sync(0xffffffffu, minv, off));
    }
    if ((threadIdx.x & 31) == 0) {
        if (minh < INFINITY) atomicMin(&a.out[k].min_h_bits, __float_as_uint(minh));
        if (minv < INFINITY) atomicMin(&a.out[k].min_v_bits, __float_as_uint(minv));
    }
}

cudaError_t launch_batch_minsep(const MinSepArgs& a, cudaStream_t s) {
    if (a.n <= 0 || a.n_adm <= 0) return cudaSuccess;
    batch_minsep_kernel<<<a.n, 256, 0, s>>>(a);
    return cudaGetLastError();
}

// Influence of request j's speculative trajectory on request k's (j before k in arrival
// order). With j stored as a plan, k's rollout could choose differently only at a step
// whose state lies within reach of one of j's wells one step later: well w is centred at
// c_w = p_j(t+1) + tau_w v_j with radius R_w (Table 3), and it adds an exact zero to the
// value of every successor when |s_k(t) - c_w| >= R_w + successor offset + 1 m. k's
// verdict could change only where the two trajectories come within the separation minima
// (+1 m) at the same step. In learned FCFS a proposal at state s(t) reads the plan samples
// of step t+1 within the feature radius, so j may also change k's proposal where
// |s(t) - p_j(t+1)| < radius + 1 m along the proposal's path: the stored trajectory when the
// judge accepted it (no FastMDP rollout ran, so its wells do not matter), else the
// proposal's own path (j can only add conflicts to an unchanged proposal, so a rejected one
// stays rejected unless its features change; the stored FastMDP plan keeps the wells test).
// A false positive costs one more speculative round, never a result.
__global__ void __launch_bounds__(128) influence_kernel(const __grid_constant__ InfluenceArgs a) {
    const int n = *a.n_dev;
    const int w = blockIdx.x, v = blockIdx.y;  // k = item w, j = item v
    if (w >= n || v >= n) return;
    const int k = a.idx[w], j = a.idx[v];
    __shared__ int hit;
    if (threadIdx.x == 0) hit = 0;
    __syncthreads();
    const int nk = j < k ? a.rout[k].n_points : 0, nj = j < k ? a.rout[j].n_points : 0;
    const int64_t tk = a.reqs[k].depart_step, tj = a.reqs[j].depart_step;
    const bool acc = a.accepted && a.accepted[k] != 0;  // stored trajectory = the accepted proposal
    if (nk > 0 && nj > 0 && tk < tj + nj && tj < tk + nk + (a.W - 1)) {  // lifetimes overlap (k sees W ahead)
        const float rho = (float)(a.reqs[k].speed_mps * a.dt) + a.dzmax + 1.0f;
        const float* pk = a.traj + (size_t)k * a.cap * 3;
        const float* pj = a.traj + (size_t)j * a.cap * 3;
        const float H = a.sep_h + 1.f, V = a.sep_v + 1.f;
        for (int i = threadIdx.x; i < nk && !hit; i += blockDim.x) {
            const float sx = pk[3 * i], sy = pk[3 * i + 1], sz = pk[3 * i + 2];
            // separation of the two trajectories at the same step (k's verdict)
            const int64_t t0 = tk + i - tj;
            if (t0 >= 0 && t0 < nj) {
                const float dx = sx - pj[3 * t0], dy = sy - pj[3 * t0 + 1], dz = sz - pj[3 * t0 + 2];
                if (dx * dx + dy * dy < H * H && fabsf(dz) < V) hit = 1;
            }
            // wells of j one to W steps later against k's state (k's action choice at this
            // step: sub-step jj of an action lies within jj successor offsets of the state)
            for (int jj = 1; jj <= a.W; ++jj) {
                const int64_t t1 = t0 + jj;
                if (t1 < 0 || t1 >= nj) continue;
                const float* q1 = pj + 3 * t1;
                float vx = 0.f, vy = 0.f, vz = 0.f;
                if (t1 + 1 < nj) {
                    vx = (q1[3] - q1[0]) / a.dt;
                    vy = (q1[4] - q1[1]) / a.dt;
                    vz = (q1[5] - q1[2]) / a.dt;
                }
                const float rj = rho * (float)jj;
                if (acc) {
                    // the accepted proposal: its features (below), not FastMDP's wells
                } else if (a.n_wells > 0) {
                    for (int w = 0; w < a.n_wells; ++w) {
                        const float r = a.w_R[w] + 1.f + rj;
                        const float dx = sx - (q1[0] + a.w_tau[w] * vx), dy = sy - (q1[1] + a.w_tau[w] * vy),
                                    dz = sz - (q1[2] + a.w_tau[w] * vz);
                        if (dx * dx + dy * dy + dz * dz < r * r) hit = 1;
                    }
                } else {
                    const float reach = a.reach_base + a.tau_absmax * sqrtf(vx * vx + vy * vy + vz * vz) + rj;
                    const float dx = sx - q1[0], dy = sy - q1[1], dz = sz - q1[2];
                    if (dx * dx + dy * dy + dz * dz < reach * reach) hit = 1;
                }
                if (acc && a.feat_r > 0.f && jj == 1) {
                    const float dx = sx - q1[0], dy = sy - q1[1], dz = sz - q1[2];
                    if (dx * dx + dy * dy + dz * dz < a.feat_r * a.feat_r) hit = 1;
                }
            }
        }
    }
    const int np = (j < k && a.traj_p && !a.accepted[k]) ? a.rout_p[k].n_points : 0;
    if (np > 0 && nj > 0 && tk < tj + nj && tj < tk + np) {  // the rejected proposal's path
        const float* pk = a.traj_p + (size_t)k * a.cap * 3;
        const float* pj = a.traj + (size_t)j * a.cap * 3;
        for (int i = threadIdx.x; i < np && !hit; i += blockDim.x) {
            const int64_t t1 = tk + i - tj + 1;
            if (t1 < 0 || t1 >= nj) continue;
            const float dx = pk[3 * i] - pj[3 * t1], dy = pk[3 * i + 1] - pj[3 * t1 + 1],
                        dz = pk[3 * i + 2] - pj[3 * t1 + 2];
            if (dx * dx + dy * dy + dz * dz < a.feat_r * a.feat_r) hit = 1;
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

// Copies the samples of n plans out of the table planes into one packed [sum counts][3]
// array (plan i's samples at offs[i]): grid x strides over samples, y over plans.
__global__ void gather_plans_kernel(const float* X, const float* Y, const float* Z, int32_t S_pad, int32_t T_win,
                                    const int32_t* slots, const int64_t* t0s, const int32_t* counts,
                                    const int64_t* offs, float* out) {
    const int p = blockIdx.y;
    const int32_t n = counts[p], slot = slots[p];
    const int64_t t0 = t0s[p], off = offs[p];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        int64_t row = (t0 + k) % T_win;
        if (row < 0) row += T_win;
        const size_t at = (size_t)row * S_pad + slot;
        float* o = out + 3 * (size_t)(off + k);
        o[0] = X[at];
        o[1] = Y[at];
        o[2] = Z[at];
    }
}

cudaError_t launch_gather_plans(const float* X, const float* Y, const float* Z, int32_t S_pad, int32_t T_win,
                                const int32_t* slots, const int64_t* t0s, const int32_t* counts, const int64_t* offs,
                                float* out, int n_plans, int max_count, cudaStream_t s) {
    if (n_plans <= 0 || max_count <= 0) return cudaSuccess;
    const int bx = min((max_count + 255) / 256, 16);
    for (int p0 = 0; p0 < n_plans; p0 += 65535) {
        const int np = min(65535, n_plans - p0);
        gather_plans_kernel<<<dim3((unsigned)bx, (unsigned)np), 256, 0, s>>>(X, Y, Z, S_pad, T_win, slots + p0, t0s + p0,
                                                                            counts + p0, offs + p0, out);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Loads the table kernels now, for the reason given at preload_index_kernels.
cudaError_t preload_table_kernels() {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, sepcheck_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, sep_reset_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, admit_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, fill_nan_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, sepcheck_rows_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, batch_minsep_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, influence_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, sep_reset_idx_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, gather_plans_kernel);
    return e;
}

cudaError_t launch_fill_nan(float* p, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const size_t want = (n + 255) / 256;
    const size_t blocks = want < (size_t)(152 * 16) ? want : (size_t)(152 * 16);
    fill_nan_kernel<<<(unsigned)blocks, 256, 0, s>>>(p, n);
    return cudaGetLastError();
}

}  // namespace fmdp
