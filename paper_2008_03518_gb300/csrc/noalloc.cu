// Allocation-free separation check: fmdp_sep_check_noalloc.
//
// The regular fmdp_sep_check stages the caller's trajectory and the kernel's atomic
// accumulators in device buffers that the library allocates and grows on demand. This
// entry point uses one fixed scratch array instead, declared below at file scope, so a
// call allocates nothing. The array lives in the library image: every GPU that loads the
// library holds it until the process exits, and all calls on a device share it.
//
// In host code the name g_noalloc_scratch is a host-side stand-in, not a device address.
// The device address is looked up with cudaGetSymbolAddress, with the context's device
// current, by the context's first call of this entry point, and kept in the context (so it
// lives and dies with the context). With lazy module loading the driver also places the
// array in device memory at that first lookup, so a context's first call is its set-up
// call; it should run at start-up, before any stream capture.
//
// Like every other entry point, the call runs on the context's device whichever device the
// caller has current (the caller's device is restored on return), reports errors through
// the context's status and message, and is counted in fmdp_stats as a separation-check
// launch.
#include <climits>
#include <cstring>

#include "host.cuh"

namespace fmdp {
namespace {

struct NoAllocScratch {
    SepOut acc;                              // accumulators of the check (cleared per call)
    float xyz[3 * FMDP_NOALLOC_MAX_POINTS];  // staged trajectory samples
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

}  // namespace
}  // namespace fmdp

extern "C" fmdp_status fmdp_sep_check_noalloc(fmdp_ctx* c, int64_t t0_step, const float* xyz, int32_t n,
                                              fmdp_sep_report* out) {
    if (!c) return FMDP_ERR_ARG;
    return guard(c, [&] {
        require(xyz && out && n >= 1, FMDP_ERR_ARG, "null trajectory or report, or n < 1");
        require(n <= FMDP_NOALLOC_MAX_POINTS, FMDP_ERR_ARG,
                "n exceeds FMDP_NOALLOC_MAX_POINTS (16384 samples per call)");
        if (!c->noalloc_scratch) {  // set-up: the array's address on the context's device
            void* p = nullptr;
            CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
            c->noalloc_scratch = p;
        }
        NoAllocScratch* d = static_cast<NoAllocScratch*>(c->noalloc_scratch);
        const int32_t S_scan = round_up(c->book.S_hw, 32);
        CK(cudaMemcpyAsync(d->xyz, xyz, (size_t)n * 3 * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        LAUNCH(c, launch_sep_reset(&d->acc, 1, c->stream));  // the array keeps the last call's contents
        SepArgs sa{};
        sa.m = c->model;
        sa.tab = table_view(c);
        sa.S_scan = S_scan;
        sa.cap = n;
        sa.traj = d->xyz;
        sa.rout = nullptr;
        sa.reqs = nullptr;
        sa.t0_fixed = t0_step;
        sa.n_fixed = n;
        sa.out = &d->acc;
        {
            KernelTimer t(c, 1);
            LAUNCH(c, launch_sepcheck(sa, 1, n, c->stream));
            t.stop();
        }
        SepOut so;
        CK(cudaMemcpyAsync(&so, &d->acc, sizeof so, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        if (c->profiling) collect_timers(c);
        c->stats.sep_pairs += (int64_t)n * S_scan;
        out->first_conflict_step = so.first_conflict == INT_MAX ? -1 : so.first_conflict;
        out->first_terrain_step = so.first_terrain == INT_MAX ? -1 : so.first_terrain;
        out->conflicts = (int64_t)so.conflicts;
        float mh, mv;
        std::memcpy(&mh, &so.min_h_bits, 4);
        std::memcpy(&mv, &so.min_v_bits, 4);
        out->min_sep_h = mh;
        out->min_sep_v = mv;
    });
}
