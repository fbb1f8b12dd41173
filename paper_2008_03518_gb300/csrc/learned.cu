// Learned proposal kernels (sm_103a): training-set collection from FastMDP rollouts, the
// bf16 tensor-core GEMM and element-wise steps of training, and policy rollouts that run
// many requests in lock step through the MLP (mma.sync m16n8k16, weights staged by bulk
// copy). The network, its inputs and its loss are stated in plain FP64 in the oracle.
#include <climits>

#include "learned.cuh"

namespace fmdp {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ void bar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void bar_expect(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool bar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait (about a second of SM cycles); false on timeout
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!bar_try(bar, parity))
        if (clock64() - t0 > (1ll << 31)) return false;
    return true;
}
__device__ __forceinline__ void bar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

}  // namespace

// ------------------------------------------------------------------ training-set collection

// One block per request: headings from the recorded actions, then one warp per step. The
// heading recurrence runs in chunks of kHeadChunk steps (one shared array per chunk), so a
// rollout of any length writes one row per step: exactly the n_points - 1 rows the host
// counted for it.
constexpr int kHeadChunk = 2048;
__global__ void __launch_bounds__(256) collect_kernel(const __grid_constant__ CollectArgs a) {
    __shared__ float feat[8][kFeat];
    __shared__ unsigned long long skey[8][kSectors];
    __shared__ int8_t head[kHeadChunk];
    __shared__ int h_carry;
    const int r = blockIdx.x;
    if (r >= a.n) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const fmdp_request req = a.reqs[r];
    const int np = a.rout[r].n_points;
    const int steps = max(np - 1, 0);
    const uint8_t* act = a.acts + (size_t)r * a.cap;
    const float dx = (float)(req.gx - req.ox), dy = (float)(req.gy - req.oy);
    const float L = sqrtf(dx * dx + dy * dy);
    const float c0 = L > 0.f ? dx / L : 1.f, s0 = L > 0.f ? dy / L : 0.f;
    const float inv_dt = (float)(1.0 / a.m.dt);
    if (threadIdx.x == 0) h_carry = 0;
    for (int k0 = 0; k0 < steps; k0 += kHeadChunk) {
        const int k1 = min(steps, k0 + kHeadChunk);
        __syncthreads();  // the previous chunk's headings are no longer read
        if (threadIdx.x == 0) {
            int h = h_carry;
            for (int k = k0; k < k1; ++k) {
                head[k - k0] = (int8_t)h;
                h += a.m.dh[act[k]];
                h += h < 0 ? 24 : 0;
                h -= h >= 24 ? 24 : 0;
            }
            h_carry = h;
        }
        __syncthreads();
        for (int k = k0 + warp; k < k1; k += 8) {
            const float* p = a.traj + ((size_t)r * a.cap + k) * 3;
            float hc, hs;
            heading_cs(c0, s0, head[k - k0], hc, hs);
            warp_features(a.m, a.iv, a.tab, req.depart_step + k + 1, p[0], p[1], p[2], hc, hs,
                          (float)req.speed_mps, (float)req.gx, (float)req.gy, (float)req.gz, inv_dt, feat[warp],
                          skey[warp]);
            const size_t row = (size_t)a.row0[r] + k;
            for (int i = lane; i < kFeat; i += 32) a.X[row * kFeat + i] = __float2bfloat16_rn(feat[warp][i]);
            if (lane == 0) a.y[row] = act[k];
            __syncwarp();
        }
    }
}

cudaError_t launch_collect(const CollectArgs& a, cudaStream_t s) {
    if (a.n <= 0) return cudaSuccess;
    collect_kernel<<<a.n, 256, 0, s>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ training kernels

// 64 x 64 output tile per block, 4 warps of 32 x 32, K in steps of 32 through shared memory.
__global__ void __launch_bounds__(128) gemm_bf16_kernel(int M, int N, int K, const __nv_bfloat16* A, long sai,
                                                        long sak, const __nv_bfloat16* B, long sbk, long sbj,
                                                        float* C, int ldc, int accumulate) {
    __shared__ __align__(16) __nv_bfloat16 As[64][40];
    __shared__ __align__(16) __nv_bfloat16 Bs[64][40];  // [n][k]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, t = lane & 3;
    const int bm = blockIdx.y * 64, bn = blockIdx.x * 64;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
    const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
    for (int k0 = 0; k0 < K; k0 += 32) {
        for (int e = tid; e < 64 * 32; e += 128) {
            const int i = e >> 5, k = e & 31, gi = bm + i, gk = k0 + k;
            As[i][k] = (gi < M && gk < K) ? A[gi * sai + gk * sak] : zero;
            const int gj = bn + i;
            Bs[i][k] = (gj < N && gk < K) ? B[gk * sbk + gj * sbj] : zero;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 32; kk += 16) {
            uint32_t af[2][4], bf[4][2];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const int r0 = wm + mt * 16 + g;
                af[mt][0] = ld32(&As[r0][kk + 2 * t]);
                af[mt][1] = ld32(&As[r0 + 8][kk + 2 * t]);
                af[mt][2] = ld32(&As[r0][kk + 8 + 2 * t]);
                af[mt][3] = ld32(&As[r0 + 8][kk + 8 + 2 * t]);
            }
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int c0 = wn + nt * 8 + g;
                bf[nt][0] = ld32(&Bs[c0][kk + 2 * t]);
                bf[nt][1] = ld32(&Bs[c0][kk + 8 + 2 * t]);
            }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[mt][nt], af[mt], bf[nt]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r = bm + wm + mt * 16 + g + (q >= 2 ? 8 : 0);
                const int c = bn + wn + nt * 8 + 2 * t + (q & 1);
                if (r < M && c < N) {
                    float v = acc[mt][nt][q];
                    if (accumulate) v += C[(size_t)r * ldc + c];
                    C[(size_t)r * ldc + c] = v;
                }
            }
}

cudaError_t launch_gemm_bf16(int M, int N, int K, const __nv_bfloat16* A, long sa_i, long sa_k,
                             const __nv_bfloat16* B, long sb_k, long sb_j, float* C, int ldc, int accumulate,
                             cudaStream_t s) {
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    gemm_bf16_kernel<<<dim3((N + 63) / 64, (M + 63) / 64), 128, 0, s>>>(M, N, K, A, sa_i, sa_k, B, sb_k, sb_j, C,
                                                                        ldc, accumulate);
    return cudaGetLastError();
}

__global__ void bias_act_kernel(const float* Z, const float* b, __nv_bfloat16* H, int M, int N, int ldz, int ldh,
                                int relu) {
    const size_t n = (size_t)M * N;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / N), j = (int)(e % N);
        float v = Z[(size_t)i * ldz + j] + b[j];
        if (relu) v = fmaxf(v, 0.f);
        H[(size_t)i * ldh + j] = __float2bfloat16_rn(v);
    }
}
cudaError_t launch_bias_act(const float* Z, const float* b, __nv_bfloat16* H, int M, int N, int ldz, int ldh, int relu,
                            cudaStream_t s) {
    bias_act_kernel<<<592, 256, 0, s>>>(Z, b, H, M, N, ldz, ldh, relu);
    return cudaGetLastError();
}

// one warp per row (logits of at most 32 actions, lanes = actions)
__global__ void softmax_ce_kernel(const float* Z, int ldz, const float* bias, const uint8_t* y, int M, int n_valid,
                                  __nv_bfloat16* dZ, int lddz, float* dZf, float* loss) {
    const int lane = threadIdx.x & 31;
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= M) return;
    const float z = lane < n_valid ? Z[(size_t)row * ldz + lane] + bias[lane] : -INFINITY;
    float mx = z;
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
    const float e = lane < n_valid ? expf(z - mx) : 0.f;
    float sum = e;
    for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(kFull, sum, o);
    const float p = e / sum;
    const int lab = y[row];
    const float gval = (p - (lane == lab ? 1.f : 0.f)) / (float)M;
    if (lane < lddz) {
        dZ[(size_t)row * lddz + lane] = __float2bfloat16_rn(lane < n_valid ? gval : 0.f);
        dZf[(size_t)row * lddz + lane] = lane < n_valid ? gval : 0.f;
    }
    if (lane == lab) atomicAdd(loss, -(logf(p)) / (float)M);
}
cudaError_t launch_softmax_ce(const float* Z, int ldz, const float* bias, const uint8_t* y, int M, int n_valid,
                              __nv_bfloat16* dZ, int lddz, float* dZf, float* loss, cudaStream_t s) {
    softmax_ce_kernel<<<(M * 32 + 255) / 256, 256, 0, s>>>(Z, ldz, bias, y, M, n_valid, dZ, lddz, dZf, loss);
    return cudaGetLastError();
}

__global__ void relu_bwd_kernel(const float* dH, const __nv_bfloat16* H, int M, int N, __nv_bfloat16* dZ, float* dZf) {
    const size_t n = (size_t)M * N;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const float v = __bfloat162float(H[e]) > 0.f ? dH[e] : 0.f;
        dZ[e] = __float2bfloat16_rn(v);
        dZf[e] = v;
    }
}
cudaError_t launch_relu_bwd(const float* dH, const __nv_bfloat16* H, int M, int N, __nv_bfloat16* dZ, float* dZf,
                            cudaStream_t s) {
    relu_bwd_kernel<<<592, 256, 0, s>>>(dH, H, M, N, dZ, dZf);
    return cudaGetLastError();
}

// column sums of G (M x N): one thread per column
__global__ void colsum_kernel(const float* G, int M, int N, int ld, float* out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    float s = 0.f;
    for (int i = 0; i < M; ++i) s += G[(size_t)i * ld + j];
    out[j] = s;
}
cudaError_t launch_colsum(const float* G, int M, int N, int ld, float* out, cudaStream_t s) {
    colsum_kernel<<<(N + 127) / 128, 128, 0, s>>>(G, M, N, ld, out);
    return cudaGetLastError();
}

__global__ void gather_rows_kernel(const __nv_bfloat16* X, const int32_t* idx, int M, __nv_bfloat16* out,
                                   const uint8_t* y, uint8_t* y_out) {
    const int row = blockIdx.x;
    if (row >= M) return;
    const int src = idx[row];
    for (int i = threadIdx.x; i < kFeat; i += blockDim.x) out[(size_t)row * kFeat + i] = X[(size_t)src * kFeat + i];
    if (threadIdx.x == 0) y_out[row] = y[src];
}
cudaError_t launch_gather_rows(const __nv_bfloat16* X, const int32_t* idx, int M, __nv_bfloat16* out,
                               const uint8_t* y, uint8_t* y_out, cudaStream_t s) {
    if (M <= 0) return cudaSuccess;
    gather_rows_kernel<<<M, 128, 0, s>>>(X, idx, M, out, y, y_out);
    return cudaGetLastError();
}

__global__ void adam_kernel(float* p, const float* g, float* m1, float* m2, size_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float a = b1 * m1[i] + (1.f - b1) * gi;
        const float v = b2 * m2[i] + (1.f - b2) * gi * gi;
        m1[i] = a;
        m2[i] = v;
        p[i] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
    }
}
cudaError_t launch_adam(float* p, const float* g, float* m1, float* m2, size_t n, float lr, float b1, float b2,
                        float eps, int t, cudaStream_t s) {
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    adam_kernel<<<592, 256, 0, s>>>(p, g, m1, m2, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

// bf16 copies of the weights: Wt[l] = W_l (in x out_pad, row-major, zero padded) for
// training, and the policy's chunked layout
__global__ void export_kernel(const float* p, __nv_bfloat16* Wt, __nv_bfloat16* Wp) {
    size_t o_t = 0;
    for (int l = 0; l < kLayers; ++l) {
        const int in = layer_in(l), out = layer_out(l), op = layer_out_pad(l);
        const float* W = p + param_offset_W(l);
        __nv_bfloat16* wp = Wp + wp_layer_offset(l);
        const size_t n = (size_t)in * op;
        for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
            const int i = (int)(e / op), j = (int)(e % op);
            const __nv_bfloat16 v = __float2bfloat16_rn(j < out ? W[(size_t)i * out + j] : 0.f);
            Wt[o_t + e] = v;
            const int ch = i / kChunkK, kl = i % kChunkK;
            wp[(size_t)ch * wp_chunk_elems(l) + (size_t)j * kChunkPad + kl] = v;
        }
        // row padding of the chunked layout
        const size_t npad = (size_t)(in / kChunkK) * op * (kChunkPad - kChunkK);
        for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < npad; e += (size_t)gridDim.x * blockDim.x) {
            const size_t rowi = e / (kChunkPad - kChunkK), q = e % (kChunkPad - kChunkK);
            wp[rowi * kChunkPad + kChunkK + q] = __float2bfloat16_rn(0.f);
        }
        o_t += n;
    }
}
cudaError_t launch_export_weights(const float* p, __nv_bfloat16* Wt, __nv_bfloat16* Wp, cudaStream_t s) {
    export_kernel<<<296, 256, 0, s>>>(p, Wt, Wp);
    return cudaGetLastError();
}

// Largest step count the judge accepts for request q: (1 + slack) times the fewest steps
// that can reach the capture ball (radius one step): horizontal motion is exactly one step
// per step, vertical motion at most the largest climb.
__device__ __noinline__ double judge_step_bound(const fmdp_request& q, double dt, double climb_step, double slack) {
    const double step = q.speed_mps * dt;
    const double dh = sqrt((q.gx - q.ox) * (q.gx - q.ox) + (q.gy - q.oy) * (q.gy - q.oy));
    const double dz = fabs(q.gz - q.oz);
    double kmin = fmax(0.0, ceil(dh / step - 1.0));
    if (climb_step > 0.0) kmin = fmax(kmin, ceil((dz - step) / climb_step));
    return floor((1.0 + slack) * kmin + 1e-9);
}

// ------------------------------------------------------------------ policy rollouts

namespace {

constexpr int kActPad = kHid + 8;  // bf16 per activation row (bank-conflict-free fragment reads)

struct PolicyRow {
    double s[3];
    double c0, s0, step, cap2;
    double gx, gy, gz;          // the request's goal, kept so a step reads no request
    int64_t t1;                 // time step of the next sample
    float speed;
    int32_t horizon;
    int32_t req, k, h, status;  // req < 0: empty
};

struct PolicyLayout {
    size_t act, wbuf, logits, feat, skey, rows, cks, bias, climb, dh, choice, bars, misc, total;
};
__host__ __device__ inline PolicyLayout policy_layout() {
    PolicyLayout L;
    size_t o = 0;
    auto al = [&](size_t a) { o = (o + a - 1) & ~(a - 1); };
    L.act = o;
    o += (size_t)2 * kPolicyRows * kActPad * sizeof(__nv_bfloat16);
    al(128);
    L.wbuf = o;
    o += (size_t)kWBufs * kHid * kChunkPad * sizeof(__nv_bfloat16);
    al(16);
    L.logits = o;
    o += (size_t)kPolicyRows * kOutPad * sizeof(float);
    L.feat = o;
    o += (size_t)(kPolicyThreads / 32) * kFeat * sizeof(float);
    al(16);
    L.skey = o;
    o += (size_t)(kPolicyThreads / 32) * kSectors * sizeof(unsigned long long);
    al(16);
    L.rows = o;
    o += (size_t)kPolicyRows * sizeof(PolicyRow);
    al(16);
    L.cks = o;  // cos, sin of 15 degree steps (FP64)
    o += 48 * sizeof(double);
    L.climb = o;  // climb x dt per action (FP64)
    o += kMaxActions * sizeof(double);
    L.bias = o;  // every layer's bias (fp32), in parameter order
    o += (size_t)((kLayers - 1) * kHid + kOutPad) * sizeof(float);
    L.dh = o;
    o += kMaxActions * sizeof(int);
    al(16);
    L.choice = o;
    o += kPolicyRows * sizeof(int);
    al(16);
    L.bars = o;
    o += kWBufs * sizeof(uint64_t);
    L.misc = o;
    o += 16;
    L.total = (o + 127) & ~size_t(127);
    return L;
}

}  // namespace

size_t policy_smem_bytes() { return policy_layout().total; }

__global__ void __launch_bounds__(kPolicyThreads, 1) policy_kernel(const __grid_constant__ PolicyArgs a) {
    extern __shared__ __align__(128) unsigned char psm[];
    const PolicyLayout L = policy_layout();
    __nv_bfloat16* act = reinterpret_cast<__nv_bfloat16*>(psm + L.act);
    __nv_bfloat16* wbuf = reinterpret_cast<__nv_bfloat16*>(psm + L.wbuf);
    float* logits = reinterpret_cast<float*>(psm + L.logits);
    float* feat = reinterpret_cast<float*>(psm + L.feat);
    unsigned long long* skey = reinterpret_cast<unsigned long long*>(psm + L.skey);
    PolicyRow* rows = reinterpret_cast<PolicyRow*>(psm + L.rows);
    double* cks = reinterpret_cast<double*>(psm + L.cks);
    int* choice = reinterpret_cast<int*>(psm + L.choice);
    uint64_t* bars = reinterpret_cast<uint64_t*>(psm + L.bars);
    int* misc = reinterpret_cast<int*>(psm + L.misc);
    double* climb_dt = reinterpret_cast<double*>(psm + L.climb);
    float* bias_s = reinterpret_cast<float*>(psm + L.bias);
    int* dh_s = reinterpret_cast<int*>(psm + L.dh);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, NWp = kPolicyThreads / 32;
    const int g = lane >> 2, t = lane & 3;
    const Model& m = a.m;
    const int A = m.A;
    const int G = a.rows;    // rows carried by this CTA (a multiple of 16, at most kPolicyRows)
    const int MT = G >> 4;   // 16-row tiles
    const float inv_dt = (float)(1.0 / m.dt);
    if (tid < 24) unit15(tid, cks[2 * tid], cks[2 * tid + 1]);
    if (tid < kPolicyRows) rows[tid].req = -1;
    if (tid < kMaxActions) {
        climb_dt[tid] = tid < A ? __dmul_rn(m.climb[tid], m.dt) : 0.0;
        dh_s[tid] = tid < A ? m.dh[tid] : 0;
    }
    for (int l = 0, o = 0; l < kLayers; o += layer_out(l), ++l)
        for (int j = tid; j < layer_out(l); j += kPolicyThreads) bias_s[o + j] = a.params[param_offset_b(l) + j];
    if (tid == 0) {
        for (int b = 0; b < kWBufs; ++b) bar_init(&bars[b]);
        misc[0] = 0;
        misc[1] = 1;  // 1 while the queue may hold work
    }
    __syncthreads();
    // weight chunks are numbered across steps (cg); chunk cg uses buffer cg % kWBufs and is
    // that buffer's (cg / kWBufs)-th fill
    long long cg = 0;
    // the weight stream of one step: chunk c of layer l_of(c)
    constexpr int kChunks = kFeat / kChunkK + (kLayers - 1) * (kHid / kChunkK);
    auto chunk_layer = [&](int c, int& l, int& kc) {
        l = 0;
        kc = c;
        while (kc >= layer_in(l) / kChunkK) {
            kc -= layer_in(l) / kChunkK;
            ++l;
        }
    };
    auto issue_chunk = [&](long long q) {  // thread 0: global chunk q
        int l, kc;
        chunk_layer((int)(q % kChunks), l, kc);
        const int b = (int)(q % kWBufs);
        const uint32_t bytes = (uint32_t)(wp_chunk_elems(l) * sizeof(__nv_bfloat16));
        bar_expect(&bars[b], bytes);
        bulk_load(wbuf + (size_t)b * kHid * kChunkPad, a.Wp + wp_layer_offset(l) + (size_t)kc * wp_chunk_elems(l),
                  bytes, &bars[b]);
    };
    bool failed = false;
    if (tid == 0)
        for (int q = 0; q < kWBufs - 1; ++q) issue_chunk(q);
    for (;;) {
        // ---- refill empty rows from the work queue (one thread per row)
        if (tid < G && rows[tid].req < 0 && misc[1]) {
            const int w = atomicAdd(a.queue, 1);
            if (w < (a.n_dev ? *a.n_dev : a.n_items)) {
                const int r = a.idx ? a.idx[w] : w;
                const fmdp_request q = a.reqs[r];
                PolicyRow& R = rows[tid];
                R.req = r;
                R.k = 0;
                R.h = 0;
                R.s[0] = q.ox;
                R.s[1] = q.oy;
                R.s[2] = q.oz;
                const double dx = __dsub_rn(q.gx, q.ox), dy = __dsub_rn(q.gy, q.oy);
                const double Lh = __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
                R.c0 = Lh > 0.0 ? __ddiv_rn(dx, Lh) : 1.0;
                R.s0 = Lh > 0.0 ? __ddiv_rn(dy, Lh) : 0.0;
                R.step = __dmul_rn(q.speed_mps, m.dt);
                R.cap2 = __dmul_rn(R.step, R.step);
                R.gx = q.gx;
                R.gy = q.gy;
                R.gz = q.gz;
                R.t1 = q.depart_step + 1;
                R.speed = (float)q.speed_mps;
                R.horizon = q.horizon;
                if (a.step_bound) {  // the judge rejects anything longer: stop there
                    const double b = judge_step_bound(q, m.dt, a.climb_step, a.slack);
                    if (b < (double)R.horizon) R.horizon = (int32_t)fmax(b, 0.0);
                }
                float* tr = a.traj + (size_t)r * a.cap * 3;
                tr[0] = (float)q.ox;
                tr[1] = (float)q.oy;
                tr[2] = (float)q.oz;
                R.status = -1;
                const double ex = __dsub_rn(q.gx, q.ox), ey = __dsub_rn(q.gy, q.oy), ez = __dsub_rn(q.gz, q.oz);
                const bool cap0 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez)) <= R.cap2;
                if (cap0 || R.horizon <= 0) {  // done before the first step
                    RolloutOut o;
                    o.n_points = 1;
                    o.status = cap0 ? kStatusCaptured : FMDP_REJ_HORIZON;
                    o.near_ties = 0;
                    o.steps = 0;
                    a.out[r] = o;
                    R.req = -1;  // the row pulls again next round
                }
            } else {
                misc[1] = 0;
            }
        }
        __syncthreads();
        int any = 0;
        for (int i = lane; i < G; i += 32) any |= rows[i].req >= 0;
        any = __any_sync(kFull, any);
        const int more = misc[1];
        __syncthreads();
        if (!any && !more) break;
        if (!any) continue;
        if (failed) break;
        // ---- features of every active row (one warp per row) into act[0]
        for (int rr = warp; rr < G; rr += NWp) {
            __nv_bfloat16* xr = act + (size_t)rr * kActPad;
            const PolicyRow R = rows[rr];
            if (R.req < 0) {
                for (int i = lane; i < kFeat; i += 32) xr[i] = __float2bfloat16_rn(0.f);
                continue;
            }
            float hc, hs;
            heading_cs((float)R.c0, (float)R.s0, R.h, hc, hs);
            warp_features(m, a.iv, a.tab, R.t1 + R.k, (float)R.s[0], (float)R.s[1], (float)R.s[2], hc, hs, R.speed,
                          (float)R.gx, (float)R.gy, (float)R.gz, inv_dt, feat + warp * kFeat, skey + warp * kSectors);
            for (int i = lane; i < kFeat; i += 32) xr[i] = __float2bfloat16_rn(feat[warp * kFeat + i]);
            __syncwarp();
        }
        __syncthreads();
        // ---- the MLP: layer by layer, weights streamed chunk by chunk
        for (int l = 0; l < kLayers && !failed; ++l) {
            const __nv_bfloat16* xin = act + (size_t)(l & 1) * kPolicyRows * kActPad;
            __nv_bfloat16* xout = act + (size_t)((l + 1) & 1) * kPolicyRows * kActPad;
            const bool last = l == kLayers - 1;
            float acc[4][4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
            const int nk = layer_in(l) / kChunkK;
            for (int kc = 0; kc < nk; ++kc, ++cg) {
                const int buf = (int)(cg % kWBufs);
                if (!bar_wait(&bars[buf], (uint32_t)((cg / kWBufs) & 1))) {
                    failed = true;
                    if (tid == 0) atomicExch(a.err, FMDP_ERR_TIMEOUT);
                }
                // the buffer of chunk cg - 1 is free (all threads passed its end barrier)
                if (tid == 0 && !failed) issue_chunk(cg + kWBufs - 1);
                const __nv_bfloat16* wb = wbuf + (size_t)buf * kHid * kChunkPad;
                if (!failed) {
                    if (!last) {
                        // warp: columns [32 warp, 32 warp + 32), all rows
#pragma unroll
                        for (int kk = 0; kk < kChunkK; kk += 16) {
                            uint32_t af[4][4], bf[4][2];
#pragma unroll
                            for (int mt = 0; mt < 4; ++mt) {
                                if (mt >= MT) break;
                                const __nv_bfloat16* r0 = xin + (size_t)(mt * 16 + g) * kActPad + kc * kChunkK + kk;
                                af[mt][0] = ld32(r0 + 2 * t);
                                af[mt][1] = ld32(r0 + 8 * kActPad + 2 * t);
                                af[mt][2] = ld32(r0 + 8 + 2 * t);
                                af[mt][3] = ld32(r0 + 8 * kActPad + 8 + 2 * t);
                            }
#pragma unroll
                            for (int nt = 0; nt < 4; ++nt) {
                                const __nv_bfloat16* b0 = wb + (size_t)(warp * 32 + nt * 8 + g) * kChunkPad + kk;
                                bf[nt][0] = ld32(b0 + 2 * t);
                                bf[nt][1] = ld32(b0 + 8 + 2 * t);
                            }
#pragma unroll
                            for (int mt = 0; mt < 4; ++mt)
#pragma unroll
                                for (int nt = 0; nt < 4; ++nt)
                                    if (mt < MT) mma_bf16(acc[mt][nt], af[mt], bf[nt]);
                        }
                    } else if (warp < MT) {
                        // last layer: warp takes rows [16 warp, 16 warp + 16), all 32 columns
#pragma unroll
                        for (int kk = 0; kk < kChunkK; kk += 16) {
                            uint32_t af[4], bf[4][2];
                            const __nv_bfloat16* r0 = xin + (size_t)(warp * 16 + g) * kActPad + kc * kChunkK + kk;
                            af[0] = ld32(r0 + 2 * t);
                            af[1] = ld32(r0 + 8 * kActPad + 2 * t);
                            af[2] = ld32(r0 + 8 + 2 * t);
                            af[3] = ld32(r0 + 8 * kActPad + 8 + 2 * t);
#pragma unroll
                            for (int nt = 0; nt < 4; ++nt) {
                                const __nv_bfloat16* b0 = wb + (size_t)(nt * 8 + g) * kChunkPad + kk;
                                bf[nt][0] = ld32(b0 + 2 * t);
                                bf[nt][1] = ld32(b0 + 8 + 2 * t);
                            }
#pragma unroll
                            for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[0][nt], af, bf[nt]);
                        }
                    }
                }
                // the chunk's buffer is free again; a timed-out wait anywhere stops every thread
                failed = __syncthreads_or(failed ? 1 : 0) != 0;
            }
            // epilogue: bias (+ ReLU) into the next activation buffer, or the logits
            const float* bias = bias_s + l * kHid;
            if (!last) {
#pragma unroll
                for (int mt = 0; mt < 4; ++mt)
#pragma unroll
                    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            if (mt >= MT) continue;
                            const int r = mt * 16 + g + (q >= 2 ? 8 : 0);
                            const int col = warp * 32 + nt * 8 + 2 * t + (q & 1);
                            xout[(size_t)r * kActPad + col] = __float2bfloat16_rn(fmaxf(acc[mt][nt][q] + bias[col], 0.f));
                        }
            } else if (warp < MT) {
#pragma unroll
                for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int r = warp * 16 + g + (q >= 2 ? 8 : 0);
                        const int col = nt * 8 + 2 * t + (q & 1);
                        logits[r * kOutPad + col] = col < kOut ? acc[0][nt][q] + bias[col] : -INFINITY;
                    }
            }
            __syncthreads();
        }
        if (failed) break;
        // ---- argmax over the actions that keep the successor inside the box (one warp per row)
        for (int rr = warp; rr < G; rr += NWp) {
            const PolicyRow R = rows[rr];
            if (R.req < 0) continue;
            float v = -INFINITY;
            if (lane < A) {
                int hn = R.h + dh_s[lane];
                hn += hn < 0 ? 24 : 0;
                hn -= hn >= 24 ? 24 : 0;
                const float C = (float)R.c0 * (float)cks[2 * hn] - (float)R.s0 * (float)cks[2 * hn + 1];
                const float S = (float)R.s0 * (float)cks[2 * hn] + (float)R.c0 * (float)cks[2 * hn + 1];
                const float x = (float)R.s[0] + (float)R.step * C, y = (float)R.s[1] + (float)R.step * S;
                const float z = (float)R.s[2] + (float)climb_dt[lane];
                const float mg = 1.0f;  // metres kept from the box faces
                const bool inside = x > (float)m.box[0] + mg && x < (float)m.box[3] - mg && y > (float)m.box[1] + mg &&
                                    y < (float)m.box[4] - mg && z > (float)m.box[2] + mg && z < (float)m.box[5] - mg;
                v = inside ? logits[rr * kOutPad + lane] : -INFINITY;
            }
            float mx = v;
            for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
            const unsigned bm = __ballot_sync(kFull, v == mx && mx > -INFINITY);
            if (lane == 0) choice[rr] = bm ? __ffs(bm) - 1 : -1;
        }
        __syncthreads();
        // ---- exact FP64 advance of the chosen action (FastMDP's successor rule, Alg. 1)
        if (tid < G && rows[tid].req >= 0) {
            PolicyRow& R = rows[tid];
            const int ch = choice[tid];
            bool done = false;
            if (ch < 0) {
                R.status = FMDP_REJ_NO_ACTION;
                done = true;
            } else {
                int hn = R.h + dh_s[ch];
                hn += hn < 0 ? 24 : 0;
                hn -= hn >= 24 ? 24 : 0;
                const double C = __dsub_rn(__dmul_rn(R.c0, cks[2 * hn]), __dmul_rn(R.s0, cks[2 * hn + 1]));
                const double S = __dadd_rn(__dmul_rn(R.s0, cks[2 * hn]), __dmul_rn(R.c0, cks[2 * hn + 1]));
                R.s[0] = __dadd_rn(R.s[0], __dmul_rn(R.step, C));
                R.s[1] = __dadd_rn(R.s[1], __dmul_rn(R.step, S));
                R.s[2] = __dadd_rn(R.s[2], climb_dt[ch]);
                R.h = hn;
                a.acts[(size_t)R.req * a.cap + R.k] = (uint8_t)ch;
                R.k += 1;
                float* tr = a.traj + ((size_t)R.req * a.cap + R.k) * 3;
                tr[0] = (float)R.s[0];
                tr[1] = (float)R.s[1];
                tr[2] = (float)R.s[2];
                const double ex = __dsub_rn(R.gx, R.s[0]), ey = __dsub_rn(R.gy, R.s[1]), ez = __dsub_rn(R.gz, R.s[2]);
                if (__dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez)) <= R.cap2) {
                    R.status = kStatusCaptured;
                    done = true;
                } else if (R.k >= R.horizon) {
                    R.status = FMDP_REJ_HORIZON;
                    done = true;
                }
            }
            if (done) {
                RolloutOut o;
                o.n_points = R.k + 1;
                o.status = R.status;
                o.near_ties = 0;
                o.steps = R.k;
                a.out[R.req] = o;
                R.req = -1;
            }
        }
        __syncthreads();
    }
    // the chunks issued for a next step that never came: wait for them before leaving
    __syncthreads();
    if (tid == 0) {
        if (!failed)
            for (long long q = cg; q < cg + kWBufs - 1; ++q) bar_wait(&bars[q % kWBufs], (uint32_t)((q / kWBufs) & 1));
        for (int b = 0; b < kWBufs; ++b) bar_inval(&bars[b]);
    }
}

cudaError_t prepare_policy_kernel() {
    return cudaFuncSetAttribute(policy_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)policy_smem_bytes());
}

cudaError_t launch_policy(const PolicyArgs& a, int n_ctas, cudaStream_t s) {
    if (a.n_items <= 0 || n_ctas <= 0) return cudaSuccess;
    policy_kernel<<<n_ctas, kPolicyThreads, policy_smem_bytes(), s>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ judge

__global__ void judge_kernel(const __grid_constant__ JudgeArgs a) {
    const int w = blockIdx.x;
    if (w >= a.n || (a.n_dev && w >= *a.n_dev)) return;
    const int r = a.idx ? a.idx[w] : w;
    __shared__ int ok_s;
    const RolloutOut rp = a.rout_p[r];
    if (threadIdx.x == 0) {
        const fmdp_request q = a.reqs[r];
        const SepOut sp = a.sep_p[r];
        const bool ok = rp.status == kStatusCaptured && sp.first_conflict == INT_MAX && sp.first_terrain == INT_MAX &&
                        (double)rp.steps <= judge_step_bound(q, a.dt, a.climb_step, a.slack);
        ok_s = ok ? 1 : 0;
        a.accepted[r] = ok_s;
        if (ok && a.traj) {
            a.rout[r] = rp;
            a.sep[r] = sp;
        }
    }
    __syncthreads();
    if (!ok_s || !a.traj) return;
    const int np = rp.n_points;
    for (int k = threadIdx.x; k < np; k += blockDim.x) {
        const size_t o = ((size_t)r * a.cap + k) * 3;
        a.traj[o] = a.traj_p[o];
        a.traj[o + 1] = a.traj_p[o + 1];
        a.traj[o + 2] = a.traj_p[o + 2];
        if (k + 1 < np) a.acts[(size_t)r * a.cap + k] = a.acts_p[(size_t)r * a.cap + k];
    }
}

cudaError_t launch_judge(const JudgeArgs& a, int max_points, cudaStream_t s) {
    if (a.n <= 0) return cudaSuccess;
    judge_kernel<<<a.n, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace fmdp
