// Spatial index of the plan table (sm_103a).
//
// The rollout's value function (Alg. 1, Sec. III) only gains a term from a known plan
// whose well (radius R_k around the plan's position at the next step, offset along its
// velocity by tau_k) reaches one of the successor states; every other plan adds an exact
// zero. The index lets a rollout step read only the plans near its state: for every ring
// row (one time step) the row's samples are grouped by the 2-D cell of their position, in
// compressed-row form, each item carrying the slot's samples at the row's step and the
// next one (its velocity). Items that move faster than a bound go to an extra list that
// every query scans, as do items appended after the row was built; a row whose extra list
// grows past a limit is rebuilt.
#include <climits>

#include <mutex>

#include "fmdp_internal.cuh"

namespace fmdp {

namespace {

constexpr int kBuildThreads = 512;

__device__ __forceinline__ int64_t ring_of(int64_t T, int32_t W) {
    int64_t r = T % W;
    return r < 0 ? r + W : r;
}

__device__ __forceinline__ int clamp_cell(float v, float o, float inv, int n) {
    const float f = floorf((v - o) * inv);
    return f < 0.f ? 0 : (f > (float)(n - 1) ? n - 1 : (int)f);
}

// cell of an item, or ncell (the extra list) when it moves faster than vmax; the velocity
// is formed exactly as the rollout forms it
__device__ __forceinline__ int item_class(const IndexArgs& a, float x1, float y1, float z1, float x2, float y2,
                                          float z2) {
    if (x2 == x2) {
        const float vx = (x2 - x1) * a.inv_dt, vy = (y2 - y1) * a.inv_dt, vz = (z2 - z1) * a.inv_dt;
        if (!(vx * vx + vy * vy + vz * vz <= a.vmax * a.vmax)) return a.ncell;
    }
    return clamp_cell(y1, a.y0, a.inv_cell, a.ncy) * a.ncx + clamp_cell(x1, a.x0, a.inv_cell, a.ncx);
}

// in-place exclusive scan of v[0 .. n) by one block; returns the total
__device__ int block_exclusive_scan(int* v, int n, int* warp_sums) {
    const int tid = threadIdx.x, NT = blockDim.x;
    const int per = (n + NT - 1) / NT;
    const int lo = min(n, tid * per), hi = min(n, lo + per);
    int local = 0;
    for (int i = lo; i < hi; ++i) local += v[i];
    // inclusive scan of the per-thread sums
    int x = local;
    const int lane = tid & 31, w = tid >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = lane < (NT >> 5) ? warp_sums[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < (NT >> 5)) warp_sums[lane] = s;  // inclusive per warp
    }
    __syncthreads();
    const int before = x - local + (w > 0 ? warp_sums[w - 1] : 0);
    const int total = warp_sums[(NT >> 5) - 1];
    __syncthreads();
    int run = before;
    for (int i = lo; i < hi; ++i) {
        const int c = v[i];
        v[i] = run;
        run += c;
    }
    __syncthreads();
    return total;
}

}  // namespace

// One block per row: count items per class, scan, scatter. Item order within a cell is not
// fixed; the rollout's combine of per-plan terms (max, or a sum in integer fixed point)
// does not depend on it.
__global__ void __launch_bounds__(kBuildThreads) index_build_kernel(const __grid_constant__ IndexArgs a, int64_t T0,
                                                                     int dirty_only) {
    extern __shared__ int ism[];
    const int32_t W = a.tab.T_win;
    const int64_t T = T0 + blockIdx.x;
    const int64_t row = ring_of(T, W);
    if (dirty_only && a.dirty[row] == 0) return;
    const int nc1 = a.ncell + 1;
    int* cnt = ism;             // [nc1]
    int* warp_sums = ism + nc1;  // [32]
    const int tid = threadIdx.x, NT = blockDim.x;
    for (int i = tid; i < nc1; i += NT) cnt[i] = 0;
    __syncthreads();
    const int S = a.tab.S_pad;
    const size_t o1 = (size_t)row * S;
    const bool has_next = T + 1 < a.tab.t_base + W;  // the next step lies in the window
    const size_t o2 = (size_t)ring_of(T + 1, W) * S;
    const float nanv = __int_as_float(0x7fc00000);
    for (int s = tid; s < S; s += NT) {
        const float x1 = a.tab.X[o1 + s];
        if (x1 != x1) continue;
        const float y1 = a.tab.Y[o1 + s], z1 = a.tab.Z[o1 + s];
        const float x2 = has_next ? a.tab.X[o2 + s] : nanv;
        const float y2 = has_next ? a.tab.Y[o2 + s] : nanv, z2 = has_next ? a.tab.Z[o2 + s] : nanv;
        atomicAdd(&cnt[item_class(a, x1, y1, z1, x2, y2, z2)], 1);
    }
    __syncthreads();
    const int n_extra = cnt[a.ncell];
    __syncthreads();
    block_exclusive_scan(cnt, nc1, warp_sums);
    int32_t* cs_row = a.cstart + row * (int64_t)nc1;
    for (int i = tid; i < nc1; i += NT) cs_row[i] = cnt[i];
    if (tid == 0) {
        a.nextra[row] = n_extra;
        a.nres[row] = n_extra;
        a.dirty[row] = 0;
    }
    __syncthreads();
    float4* it = a.items + (size_t)row * S * 2;
    for (int s = tid; s < S; s += NT) {
        const float x1 = a.tab.X[o1 + s];
        if (x1 != x1) continue;
        const float y1 = a.tab.Y[o1 + s], z1 = a.tab.Z[o1 + s];
        const float x2 = has_next ? a.tab.X[o2 + s] : nanv;
        const float y2 = has_next ? a.tab.Y[o2 + s] : nanv, z2 = has_next ? a.tab.Z[o2 + s] : nanv;
        const int pos = atomicAdd(&cnt[item_class(a, x1, y1, z1, x2, y2, z2)], 1);
        it[2 * pos] = make_float4(x1, y1, z1, __int_as_float(s));
        it[2 * pos + 1] = make_float4(x2, y2, z2, 0.f);
    }
}

// Grid: x strides over samples, y over trajectories. Each slot has at most one sample per
// row, and a stored trajectory occupies a slot that had none in its rows when they were
// last built, so a row never holds more than S_pad items.
__global__ void index_append_kernel(const __grid_constant__ IndexAppendArgs a) {
    const IndexArgs& ix = a.ix;
    int n, slot;
    int64_t t0;
    const float* base;
    if (a.force) {
        const int r = blockIdx.y;
        slot = a.slots[r];
        n = a.counts[r];
        t0 = a.t0s[r];
        base = a.traj + (size_t)a.offs[r] * 3;
    } else {
        if (a.n_dev && (int)blockIdx.y >= *a.n_dev) return;
        const int r = a.idx ? a.idx[blockIdx.y] : (int)blockIdx.y;
        if (!a.tentative && a.sep[r].verdict != FMDP_ADMITTED) return;
        slot = a.tentative ? 0 : a.slots[r];
        n = a.rout[r].n_points;
        t0 = a.reqs[r].depart_step;
        base = a.traj + (size_t)r * a.cap * 3;
    }
    const int32_t W = ix.tab.T_win;
    const int S = ix.tab.S_pad;
    const float nanv = __int_as_float(0x7fc00000);
    const bool tent = a.tentative != 0;
    const int32_t tag = tent ? tentative_tag(a.tent_ord) : slot;
    int32_t* tpos = tent ? a.tpos + (size_t)(a.idx ? a.idx[blockIdx.y] : (int)blockIdx.y) * a.cap : nullptr;
    const int k0 = tent ? a.first : 0;
    for (int k = k0 + blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int64_t T = t0 + k;
        if (tpos) tpos[k] = -1;
        if (T < ix.tab.t_base || T >= ix.tab.t_base + W) continue;
        const int64_t row = ring_of(T, W);
        const float* p = base + 3 * (size_t)k;
        const bool has_next = k + 1 < n && T + 1 < ix.tab.t_base + W;
        const int pos = atomicAdd(&ix.nres[row], 1);
        const int at = ix.cstart[row * (int64_t)(ix.ncell + 1) + ix.ncell] + pos;
        if (at < S) {
            float4* it = ix.items + (size_t)row * S * 2;
            it[2 * at] = make_float4(p[0], p[1], p[2], __int_as_float(tag));
            it[2 * at + 1] = has_next ? make_float4(p[3], p[4], p[5], 0.f) : make_float4(nanv, nanv, nanv, 0.f);
            if (tpos) tpos[k] = at;
        } else {
            atomicSub(&ix.nres[row], 1);  // cannot happen (see above); rebuild the row instead
            ix.dirty[row] = 1;
        }
        if (pos + 1 > ix.extra_limit) ix.dirty[row] = 1;
    }
}

// nextra = nres for every row: the items appended by earlier launches on this stream
// become visible to readers (stream order: those launches have completed).
__global__ void index_publish_kernel(int32_t* nextra, const int32_t* nres, int32_t n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) nextra[i] = nres[i];
}

cudaError_t launch_index_publish(const IndexArgs& a, cudaStream_t s) {
    const int n = a.tab.T_win;
    if (n <= 0) return cudaSuccess;
    index_publish_kernel<<<(n + 255) / 256, 256, 0, s>>>(a.nextra, a.nres, n);
    return cudaGetLastError();
}

__global__ void index_withdraw_kernel(const __grid_constant__ IndexArgs ix, const int32_t* tpos, int64_t t0,
                                      int32_t n) {
    const int32_t W = ix.tab.T_win;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int64_t T = t0 + k;
        const int32_t at = tpos[k];
        if (at < 0 || T < ix.tab.t_base || T >= ix.tab.t_base + W) continue;
        const int64_t row = ring_of(T, W);
        float* w = reinterpret_cast<float*>(ix.items + ((size_t)row * ix.tab.S_pad + at) * 2) + 3;
        *w = __int_as_float(kTagDead);
    }
}

cudaError_t launch_index_withdraw(const IndexArgs& a, const int32_t* tpos, int64_t t0, int32_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    index_withdraw_kernel<<<(n + 255) / 256, 256, 0, s>>>(a, tpos, t0, n);
    return cudaGetLastError();
}

__global__ void store_release_kernel(int32_t* p, int32_t v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

cudaError_t launch_store_release(int32_t* p, int32_t v, cudaStream_t s) {
    store_release_kernel<<<1, 1, 0, s>>>(p, v);
    return cudaGetLastError();
}

// Loads the index kernels now. Under lazy module loading a kernel's code is loaded at its first
// launch, and that load waits for the kernels running at the time; the pipelined mode launches
// these kernels beside a persistent rollout launch that runs until the host stops it.
cudaError_t preload_index_kernels() {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, index_build_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, index_append_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, index_publish_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, index_withdraw_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, store_release_kernel);
    return e;
}

size_t index_build_smem(int ncell) { return (size_t)(ncell + 1 + 32) * sizeof(int); }

// The attribute belongs to the kernel, not to a context: every scheduler of the process
// shares it, so it only ever grows (a later scheduler with a smaller grid must not shrink
// what an earlier one launches with).
cudaError_t prepare_index_kernels(size_t smem) {
    static std::mutex mu;
    static size_t granted = 0;
    std::lock_guard<std::mutex> lock(mu);
    if (smem <= granted) return cudaSuccess;
    const cudaError_t e =
        cudaFuncSetAttribute(index_build_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) granted = smem;
    return e;
}

cudaError_t launch_index_build(const IndexArgs& a, int64_t T0, int32_t n, int dirty_only, size_t smem,
                               cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    index_build_kernel<<<(unsigned)n, kBuildThreads, smem, s>>>(a, T0, dirty_only);
    return cudaGetLastError();
}

cudaError_t launch_index_append(const IndexAppendArgs& a, int n_items, int max_points, cudaStream_t s) {
    if (n_items <= 0 || max_points <= 0) return cudaSuccess;
    const int bx = min((max_points + 255) / 256, 16);
    for (int r0 = 0; r0 < n_items; r0 += 65535) {
        if (r0 > 0 && (a.idx || a.n_dev)) return cudaErrorInvalidValue;
        IndexAppendArgs b = a;
        const int nr = min(65535, n_items - r0);
        if (a.force) {
            b.t0s = a.t0s + r0;
            b.counts = a.counts + r0;
            b.offs = a.offs + r0;
        }
        index_append_kernel<<<dim3((unsigned)bx, (unsigned)nr), 256, 0, s>>>(b);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace fmdp
