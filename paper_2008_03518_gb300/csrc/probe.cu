// Throughput probes of the units the well scan uses (measurement support): FP32 FMA and the
// MUFU reciprocal square root and exp2, each as eight independent dependency chains per
// thread over every SM, timed with CUDA events. The SM clock is read from clock64 over the
// FMA probe. The bench divides the well scan's counted operations by these rates.
#include <vector>

#include "fmdp_internal.cuh"

namespace fmdp {

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 4;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kProbeThreads) ffma_probe(float* sink, long long* cycles, int iters, float a,
                                                            float b) {
    float x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = 1e-7f * threadIdx.x + (float)i;
    const long long c0 = clock64();
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = fmaf(x[i], a, b);
    const long long c1 = clock64();
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    if (s == -1.2345f) sink[blockIdx.x] = s;  // never true: keeps the chains live
    if (threadIdx.x == 0) cycles[blockIdx.x] = c1 - c0;
}

template <int OP>
__global__ void __launch_bounds__(kProbeThreads) mufu_probe(float* sink, int iters) {
    float x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = 1.0f + 1e-7f * threadIdx.x + 0.125f * (float)i;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < kChains; ++i) {
            if (OP == 0)
                asm volatile("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(x[i]));
            else
                asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(x[i]));
        }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    if (s == -1.2345f) sink[blockIdx.x] = s;
}

}  // namespace

cudaError_t probe_peaks(int n_sm, cudaStream_t s, fmdp_peaks* out) {
    const int blocks = n_sm * kProbeBlocksPerSm;
    const double threads = (double)blocks * kProbeThreads;
    float* sink = nullptr;
    long long* cyc = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&sink, blocks * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&cyc, blocks * sizeof(long long));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    auto timed = [&](auto&& launch, float& ms) {
        launch();  // warm-up
        cudaEventRecord(e0, s);
        launch();
        cudaEventRecord(e1, s);
        cudaError_t r = cudaGetLastError();
        if (r == cudaSuccess) r = cudaEventSynchronize(e1);
        if (r == cudaSuccess) r = cudaEventElapsedTime(&ms, e0, e1);
        return r;
    };
    const int it_fma = 1 << 16, it_mufu = 1 << 13;
    float ms_fma = 0.f, ms_rsq = 0.f, ms_ex2 = 0.f;
    if (e == cudaSuccess)
        e = timed([&] { ffma_probe<<<blocks, kProbeThreads, 0, s>>>(sink, cyc, it_fma, 0.9999f, 1e-7f); }, ms_fma);
    std::vector<long long> h(blocks, 0);
    if (e == cudaSuccess) e = cudaMemcpy(h.data(), cyc, blocks * sizeof(long long), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = timed([&] { mufu_probe<0><<<blocks, kProbeThreads, 0, s>>>(sink, it_mufu); }, ms_rsq);
    if (e == cudaSuccess)
        e = timed([&] { mufu_probe<1><<<blocks, kProbeThreads, 0, s>>>(sink, it_mufu); }, ms_ex2);
    if (e == cudaSuccess) {
        long long mx = 0;
        for (long long v : h) mx = v > mx ? v : mx;
        out->fp32_tflops = 2.0 * kChains * it_fma * threads / (ms_fma * 1e-3) / 1e12;
        out->mufu_rsqrt_tops = (double)kChains * it_mufu * threads / (ms_rsq * 1e-3) / 1e12;
        out->mufu_ex2_tops = (double)kChains * it_mufu * threads / (ms_ex2 * 1e-3) / 1e12;
        out->sm_mhz = ms_fma > 0.f ? (double)mx / (ms_fma * 1e-3) / 1e6 : 0.0;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (cyc) cudaFree(cyc);
    return e;
}

}  // namespace fmdp
