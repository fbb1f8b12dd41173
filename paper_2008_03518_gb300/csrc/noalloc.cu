// Allocation-free separation check: fmdp_sep_check_noalloc.
//
// The regular fmdp_sep_check stages the caller's trajectory and the kernel's atomic
// accumulators in device buffers that the library allocates and grows on demand. This
// entry point uses one fixed scratch array instead, declared below at file scope, so a
// call allocates nothing. The array lives in the library image: every GPU that loads the
// library holds it until the process exits, and all calls on a device share it.
//
// In host code the name g_noalloc_scratch is a host-side stand-in, not a device address,
// so the device address is looked up once per device (cudaGetSymbolAddress, with that
// device current) on the first call and cached. With lazy module loading the driver also
// places the array in device memory at that first lookup, so the first call on a device
// is the set-up call; it should run at start-up, before any stream capture.
#include <cstdio>
#include <cstring>
#include <climits>
#include <mutex>

#include "fmdp_internal.cuh"

namespace fmdp {
namespace {

struct NoAllocScratch {
    SepOut acc;                             // accumulators of the check (cleared per call)
    float xyz[3 * FMDP_NOALLOC_MAX_POINTS]; // staged trajectory samples
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

constexpr int kMaxDevices = 128;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t scratch_address(NoAllocScratch** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<NoAllocScratch*>(g_scratch_addr[dev]);
    return cudaSuccess;
}

fmdp_status fail(fmdp_ctx* ctx, fmdp_status code, const char* what, cudaError_t e = cudaSuccess) {
    char buf[256];
    if (e != cudaSuccess) std::snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    else std::snprintf(buf, sizeof buf, "%s", what);
    ctx_set_error(ctx, buf);
    return code;
}

}  // namespace
}  // namespace fmdp

using namespace fmdp;

extern "C" fmdp_status fmdp_sep_check_noalloc(fmdp_ctx* ctx, int64_t t0_step, const float* xyz, int32_t n,
                                              fmdp_sep_report* out) {
    if (!ctx) return FMDP_ERR_ARG;
    if (!xyz || !out || n < 1) return fail(ctx, FMDP_ERR_ARG, "null trajectory or report, or n < 1");
    if (n > FMDP_NOALLOC_MAX_POINTS)
        return fail(ctx, FMDP_ERR_ARG, "n exceeds FMDP_NOALLOC_MAX_POINTS (16384 samples per call)");
    SepView v;
    ctx_sep_view(ctx, &v);
    NoAllocScratch* d = nullptr;
    cudaError_t e = scratch_address(&d);
    if (e != cudaSuccess) return fail(ctx, FMDP_ERR_CUDA, "scratch address lookup", e);
    e = cudaMemcpyAsync(d->xyz, xyz, (size_t)n * 3 * sizeof(float), cudaMemcpyHostToDevice, v.stream);
    if (e != cudaSuccess) return fail(ctx, FMDP_ERR_CUDA, "trajectory upload", e);
    e = launch_sep_reset(&d->acc, 1, v.stream);  // the array keeps the previous call's contents
    if (e != cudaSuccess) return fail(ctx, FMDP_ERR_CUDA, "accumulator reset", e);
    SepArgs sa{};
    sa.m = v.m;
    sa.tab = v.tab;
    sa.S_scan = v.S_scan;
    sa.cap = n;
    sa.traj = d->xyz;
    sa.rout = nullptr;
    sa.reqs = nullptr;
    sa.t0_fixed = t0_step;
    sa.n_fixed = n;
    sa.out = &d->acc;
    e = launch_sepcheck(sa, 1, n, v.stream);
    if (e != cudaSuccess) return fail(ctx, FMDP_ERR_CUDA, "separation-check launch", e);
    SepOut so;
    e = cudaMemcpyAsync(&so, &d->acc, sizeof so, cudaMemcpyDeviceToHost, v.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(v.stream);
    if (e != cudaSuccess) return fail(ctx, FMDP_ERR_CUDA, "report download", e);
    out->first_conflict_step = so.first_conflict == INT_MAX ? -1 : so.first_conflict;
    out->first_terrain_step = so.first_terrain == INT_MAX ? -1 : so.first_terrain;
    out->conflicts = (int64_t)so.conflicts;
    float mh, mv;
    std::memcpy(&mh, &so.min_h_bits, 4);
    std::memcpy(&mv, &so.min_v_bits, 4);
    out->min_sep_h = mh;
    out->min_sep_v = mv;
    ctx_set_error(ctx, "");
    return FMDP_OK;
}
