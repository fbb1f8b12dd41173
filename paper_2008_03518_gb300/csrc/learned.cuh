// Learned proposal (no counterpart in the paper): a small MLP trained on FastMDP's action
// choices (Alg. 1, Sec. III) proposes a whole trajectory, which the separation check and a
// path-cost bound then judge; plain FastMDP is the fallback.
#pragma once

#include <cuda_bf16.h>

#include "fmdp_internal.cuh"

namespace fmdp {

constexpr int kFeat = 128;        // network inputs
constexpr int kHid = 256;         // hidden width (four hidden layers)
constexpr int kOut = 25;          // action logits
constexpr int kOutPad = 32;       // logits padded to four 8-wide tiles
constexpr int kLayers = 5;
constexpr int kSectors = 20;      // 10 azimuth sectors x (above, below)
constexpr int kOwn = 8;
constexpr float kRF = 1000.0f;    // metres: sectors see plan samples this close
constexpr int kChunkK = 64;       // weight rows per staged chunk (policy kernel)
constexpr int kChunkPad = 72;     // bf16 per staged row: 64 + 8 (bank-conflict-free reads)

__host__ __device__ constexpr int layer_in(int l) { return l == 0 ? kFeat : kHid; }
__host__ __device__ constexpr int layer_out(int l) { return l == kLayers - 1 ? kOut : kHid; }
__host__ __device__ constexpr int layer_out_pad(int l) { return l == kLayers - 1 ? kOutPad : kHid; }
// fp32 master parameters: per layer W (in x out, row-major) then b (out)
__host__ __device__ inline size_t param_offset_W(int l) {
    size_t o = 0;
    for (int i = 0; i < l; ++i) o += (size_t)layer_in(i) * layer_out(i) + layer_out(i);
    return o;
}
__host__ __device__ inline size_t param_offset_b(int l) { return param_offset_W(l) + (size_t)layer_in(l) * layer_out(l); }
__host__ __device__ inline size_t n_params_total() { return param_offset_W(kLayers); }
// policy weights: per layer, chunks of kChunkK input rows, each [out_pad][kChunkPad] bf16
// (out-major, the chunk's inputs contiguous: the column layout of the mma B operand)
__host__ __device__ inline size_t wp_chunk_elems(int l) { return (size_t)layer_out_pad(l) * kChunkPad; }
__host__ __device__ inline size_t wp_layer_offset(int l) {
    size_t o = 0;
    for (int i = 0; i < l; ++i) o += (size_t)(layer_in(i) / kChunkK) * wp_chunk_elems(i);
    return o;
}
__host__ __device__ inline size_t wp_total() { return wp_layer_offset(kLayers); }

// Features of one state, computed by one warp into out[kFeat] (shared memory). s: position;
// (hc, hs): heading cos / sin; T1: the step of the plan samples to read (the next step);
// skey: kSectors words of scratch in shared memory. The order of reading and of the
// index's items does not change the result: each sector keeps its minimum of (squared
// distance, a hash of the sample's coordinates).
__device__ __forceinline__ uint32_t sample_hash(float x, float y, float z) {
    return __float_as_uint(x) ^ (__float_as_uint(y) * 2654435761u) ^ (__float_as_uint(z) * 40503u);
}
__device__ __forceinline__ float clampf(float v, float lo, float hi) { return fminf(fmaxf(v, lo), hi); }

__device__ inline void warp_features(const Model& m, const IndexView& iv, const TableView& tab, int64_t T1, float sx,
                                     float sy, float sz, float hc, float hs, float speed, float gx, float gy, float gz,
                                     float inv_dt, float* out, unsigned long long* skey) {
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < kFeat; i += 32) out[i] = 0.f;
    if (lane < kSectors) skey[lane] = ~0ull;
    if (lane == 0) {
        const float z0 = (float)m.box[2], z1 = (float)m.box[5];
        out[0] = (sz - z0) / (z1 - z0);
        const float clr = m.hm ? sz - terrain32(m, sx, sy) : sz - z0;
        out[1] = clampf(clr / 200.f, -1.f, 4.f);
        const float Gx = gx - sx, Gy = gy - sy, Gz = gz - sz;
        const float gf = Gx * hc + Gy * hs, gl = -Gx * hs + Gy * hc;
        const float gh = sqrtf(gf * gf + gl * gl);
        out[2] = clampf(gf / 5000.f, -4.f, 4.f);
        out[3] = clampf(gl / 5000.f, -4.f, 4.f);
        out[4] = clampf(Gz / 200.f, -4.f, 4.f);
        out[5] = fminf(gh / 20000.f, 4.f);
        out[6] = gh > 0.f ? gf / gh : 1.f;
        out[7] = gh > 0.f ? gl / gh : 0.f;
    }
    __syncwarp();
    if (T1 < tab.t_base || T1 >= tab.t_base + tab.T_win) return;
    int64_t row = T1 % tab.T_win;
    if (row < 0) row += tab.T_win;
    const int32_t* cs_row = iv.cstart + row * (int64_t)(iv.ncell + 1);
    const float4* it = iv.items + (size_t)row * tab.S_pad * 2;
    auto cell_of = [&](float v, float o, int n) {
        const float f = floorf((v - o) * iv.inv_cell);
        return f < 0.f ? 0 : (f > (float)(n - 1) ? n - 1 : (int)f);
    };
    const int cx0 = cell_of(sx - kRF, iv.x0, iv.ncx), cx1 = cell_of(sx + kRF, iv.x0, iv.ncx);
    const int cy0 = cell_of(sy - kRF, iv.y0, iv.ncy), cy1 = cell_of(sy + kRF, iv.y0, iv.ncy);
    const float R2 = kRF * kRF;
    const unsigned full = 0xffffffffu;
    auto sector_of = [&](float rf, float rl, float rz) {
        const float az = atan2f(rl, rf);  // [-pi, pi]
        int k = (int)floorf((az + 3.14159265358979f) * (10.f / 6.28318530717959f));
        k = min(max(k, 0), 9);
        return k + (rz >= 0.f ? 10 : 0);
    };
    // The query's ranges: its cell rows (cells cx0..cx1 of a row are contiguous), then the
    // extra list. They are taken 16 at a time; lanes 2q and 2q + 1 load range q's bounds
    // together, and the lanes then share out the group's items as one flat list.
    const int nrows = cy1 - cy0 + 1;
    auto visit = [&](auto&& fn) {
        for (int q0 = 0; q0 <= nrows; q0 += 16) {
            const int q = q0 + (lane >> 1);
            int v = 0;
            if (q < nrows) {
                v = cs_row[(cy0 + q) * iv.ncx + ((lane & 1) ? cx1 + 1 : cx0)];
            } else if (q == nrows) {
                v = (lane & 1) ? cs_row[iv.ncell] + iv.nextra[row] : cs_row[iv.ncell];
            }
            int beg[16], start[17];
            start[0] = 0;
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int b = __shfl_sync(full, v, 2 * k), e = __shfl_sync(full, v, 2 * k + 1);
                beg[k] = b;
                start[k + 1] = start[k] + (q0 + k <= nrows ? max(0, e - b) : 0);
            }
            const int total = start[16];
            for (int j = lane; j < total; j += 32) {
                // the range holding flat item j: the last k whose start is at or before j
                int i = beg[0] + j;
#pragma unroll
                for (int k = 1; k < 16; ++k)
                    if (j >= start[k]) i = beg[k] + (j - start[k]);
                fn(i);
            }
        }
    };
    // sector feature of the nearest sample P1 (and the same plan's next sample P2)
    auto emit = [&](float4 P1, float4 P2, float d2, int sec) {
        const float rx = P1.x - sx, ry = P1.y - sy, rz = P1.z - sz;
        const float rf = rx * hc + ry * hs, rl = -rx * hs + ry * hc;
        float vx = 0.f, vy = 0.f, vz = 0.f;
        if (P2.x == P2.x) {
            vx = (P2.x - P1.x) * inv_dt;
            vy = (P2.y - P1.y) * inv_dt;
            vz = (P2.z - P1.z) * inv_dt;
        }
        const float vf = vx * hc + vy * hs, vl = -vx * hs + vy * hc;
        const float w = 1.f - sqrtf(d2) / kRF;
        float* o = out + kOwn + 6 * sec;
        o[0] = rf * (1.f / 500.f) * w;
        o[1] = rl * (1.f / 500.f) * w;
        o[2] = rz * (1.f / 500.f) * w;
        o[3] = (vf - speed) * (1.f / 50.f) * w;
        o[4] = vl * (1.f / 50.f) * w;
        o[5] = vz * (1.f / 50.f) * w;
    };
    // key of sample P1: (squared distance, position hash), all-ones beyond R_F
    auto key_of = [&](float4 P1, float& d2, int& sec) {
        const float rx = P1.x - sx, ry = P1.y - sy, rz = P1.z - sz;
        d2 = rx * rx + ry * ry + rz * rz;
        if (!(d2 < R2)) return ~0ull;
        sec = sector_of(rx * hc + ry * hs, -rx * hs + ry * hc, rz);
        return ((unsigned long long)__float_as_uint(d2) << 32) | sample_hash(P1.x, P1.y, P1.z);
    };
    // pass 1: every sector's least key; a lane keeps its first two in-range samples
    int ci0 = -1, ci1 = -1, cs0 = 0, cs1 = 0;
    float cd0 = 0.f, cd1 = 0.f;
    unsigned long long ck0 = 0, ck1 = 0;
    float4 cp0 = make_float4(0.f, 0.f, 0.f, 0.f), cp1 = cp0;
    bool over = false;
    visit([&](int i) {
        const float4 P1 = it[2 * (size_t)i];
        float d2;
        int sec;
        const unsigned long long key = key_of(P1, d2, sec);
        if (key == ~0ull) return;
        atomicMin(&skey[sec], key);
        if (ci0 < 0) {
            ci0 = i, cs0 = sec, cd0 = d2, ck0 = key, cp0 = P1;
        } else if (ci1 < 0) {
            ci1 = i, cs1 = sec, cd1 = d2, ck1 = key, cp1 = P1;
        } else {
            over = true;
        }
    });
    __syncwarp();
    // pass 2: the sector winners write their features
    if (!__any_sync(full, over)) {
        if (ci0 >= 0 && ck0 == skey[cs0]) emit(cp0, it[2 * (size_t)ci0 + 1], cd0, cs0);
        if (ci1 >= 0 && ck1 == skey[cs1]) emit(cp1, it[2 * (size_t)ci1 + 1], cd1, cs1);
    } else {
        visit([&](int i) {
            const float4 P1 = it[2 * (size_t)i];
            float d2;
            int sec;
            const unsigned long long key = key_of(P1, d2, sec);
            if (key != ~0ull && key == skey[sec]) emit(P1, it[2 * (size_t)i + 1], d2, sec);
        });
    }
    __syncwarp();
}

// fp32 cos / sin of the heading with index h (15 degree steps) turned from the bearing
// (c0, s0): the features' heading frame
__device__ __forceinline__ void heading_cs(float c0, float s0, int h, float& hc, float& hs) {
    const float a = (float)h * (3.14159265358979f / 12.f);
    float sk, ck;
    sincosf(a, &sk, &ck);
    hc = c0 * ck - s0 * sk;
    hs = s0 * ck + c0 * sk;
}

// ---- device entry points (learned.cu)
struct CollectArgs {
    Model m;
    TableView tab;
    IndexView iv;
    const float* traj;          // [n][cap][3]
    const uint8_t* acts;        // [n][cap]
    int32_t cap;
    const RolloutOut* rout;
    const fmdp_request* reqs;
    const int64_t* row0;        // [n]: first training row of request r
    __nv_bfloat16* X;           // [rows][kFeat]
    uint8_t* y;                 // [rows]
    int32_t n;
};
cudaError_t launch_collect(const CollectArgs& a, cudaStream_t s);

// C[M x N] (fp32, row stride ldc) = op(A) op(B) (+ C when accumulate): A(i, k) at
// A[i * sa_i + k * sa_k], B(k, j) at B[k * sb_k + j * sb_j], both bf16.
cudaError_t launch_gemm_bf16(int M, int N, int K, const __nv_bfloat16* A, long sa_i, long sa_k,
                             const __nv_bfloat16* B, long sb_k, long sb_j, float* C, int ldc, int accumulate,
                             cudaStream_t s);
// H (bf16) = act(Z + b): relu for hidden layers
cudaError_t launch_bias_act(const float* Z, const float* b, __nv_bfloat16* H, int M, int N, int ldz, int ldh, int relu,
                            cudaStream_t s);
// mean softmax cross-entropy: loss added to *loss, dZ (bf16, ld) = (softmax - onehot) / M
cudaError_t launch_softmax_ce(const float* Z, int ldz, const float* bias, const uint8_t* y, int M, int n_valid,
                              __nv_bfloat16* dZ, int lddz, float* dZf, float* loss, cudaStream_t s);
// dZ (bf16 and fp32) = dH * (H > 0)
cudaError_t launch_relu_bwd(const float* dH, const __nv_bfloat16* H, int M, int N, __nv_bfloat16* dZ, float* dZf,
                            cudaStream_t s);
cudaError_t launch_colsum(const float* G, int M, int N, int ld, float* out, cudaStream_t s);
cudaError_t launch_gather_rows(const __nv_bfloat16* X, const int32_t* idx, int M, __nv_bfloat16* out,
                               const uint8_t* y, uint8_t* y_out, cudaStream_t s);
// Adam on the fp32 master parameters, then the bf16 copies (training layout W[in][out],
// and the policy's chunk layout)
cudaError_t launch_adam(float* p, const float* g, float* m1, float* m2, size_t n, float lr, float b1, float b2,
                        float eps, int t, cudaStream_t s);
cudaError_t launch_export_weights(const float* p, __nv_bfloat16* Wt, __nv_bfloat16* Wp, cudaStream_t s);

// Policy rollouts: each CTA carries kPolicyRows requests in lock step (one matrix row each)
// and refills a finished row from the work queue.
constexpr int kPolicyRows = 32;
constexpr int kWBufs = 4;       // weight chunk buffers: three chunks stream while one is used
constexpr int kPolicyThreads = 256;
struct PolicyArgs {
    Model m;
    TableView tab;
    IndexView iv;
    const __nv_bfloat16* Wp;  // chunked bf16 weights
    const float* params;      // fp32 master parameters (biases)
    const fmdp_request* reqs;
    const int32_t* idx;       // work items -> requests (nullptr: identity)
    int32_t n_items;
    const int32_t* n_dev;     // number of work items on the device (nullptr: n_items)
    int32_t* queue;           // work counter
    int32_t cap;
    float* traj;              // [n][cap][3]
    uint8_t* acts;            // [n][cap]
    RolloutOut* out;          // [n]
    int32_t* err;
    int32_t rows;             // requests per CTA: 16 or 32
    // 1: stop a proposal at the judge's step bound (a longer one would be rejected anyway)
    int32_t step_bound;
    double slack, climb_step;
};
// rows per CTA for n work items on n_sm multiprocessors: 32 when that still gives every
// multiprocessor a CTA, else 16
inline int policy_rows_for(int n, int n_sm) { return (n + 31) / 32 >= n_sm ? 32 : 16; }
size_t policy_smem_bytes();
cudaError_t prepare_policy_kernel();
cudaError_t launch_policy(const PolicyArgs& a, int n_ctas, cudaStream_t s);

// Judge: a proposal is accepted when it reaches the goal, passes the separation and
// terrain checks, and takes at most (1 + slack) times the fewest steps any trajectory
// needs to reach the goal (which bounds its cost gap to FastMDP's by the same factor).
// Accepted proposals are copied over the request's FastMDP buffers and flagged.
struct JudgeArgs {
    const fmdp_request* reqs;
    const int32_t* idx;
    const int32_t* n_dev;
    int32_t n;
    const float* traj_p;
    const uint8_t* acts_p;
    const RolloutOut* rout_p;
    const SepOut* sep_p;
    float* traj;              // nullptr: decide only, copy nothing
    uint8_t* acts;
    RolloutOut* rout;
    SepOut* sep;
    int32_t* accepted;        // [n]
    int32_t cap;
    double dt, slack;
    double climb_step;        // largest |climb| x dt of the action set
};
cudaError_t launch_judge(const JudgeArgs& a, int max_points, cudaStream_t s);

}  // namespace fmdp
