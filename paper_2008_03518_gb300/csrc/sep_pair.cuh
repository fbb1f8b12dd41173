// Separation test of one pair of samples (Sec. V: a conflict is a pair closer than the
// horizontal minimum and the vertical minimum at the same step), shared by every kernel
// that measures a pair, so that they all decide it the same way.
#pragma once

#include "fmdp_internal.cuh"

namespace fmdp {

// Separation minima of one sample pair with explicit rounding (no contraction), so that
// every kernel that measures the same pair gets the same bits. Thresholds in the band
// around H^2 and V are decided again in FP64 from the same fp32 inputs.
//
// Width of the bands, with u = 2^-24 (fp32 round to nearest): dx = fl(px - qx) is the exact
// difference ex times (1 + d), |d| <= u, whatever the magnitudes (one rounding of an exact
// real), so h2 = fl(dx^2 + fl(dy^2)) lies within a factor (1 +- u)^4 of E = ex^2 + ey^2,
// and H2 = fl(fl(sep_h)^2) within (1 +- u)^3 of S = sep_h^2; the FP64 decision rounds E and
// S by a few 2^-53 at most. If |h2 - H2| >= 16 u H2, E and S therefore differ by more than
// 8 u S in the same direction, and the FP64 decision agrees with the fp32 one. Likewise
// |dz| and Vm = fl(sep_v) are within a factor 1 +- u of |ez| and sep_v, so 16 u Vm
// suffices vertically. A floor of 2^-100 keeps the bands positive for zero minima.
struct SepConsts {
    float H2, Vm, hband, vband;
    double H2d, Vd;
};
static __device__ __forceinline__ SepConsts sep_consts(double sep_h, double sep_v) {
    SepConsts k;
    const float H = (float)sep_h;
    k.H2 = __fmul_rn(H, H);
    k.Vm = (float)sep_v;
    k.hband = fmaxf(__fmul_rn(k.H2, 0x1p-20f), 0x1p-100f);
    k.vband = fmaxf(__fmul_rn(k.Vm, 0x1p-20f), 0x1p-100f);
    k.H2d = __dmul_rn(sep_h, sep_h);
    k.Vd = sep_v;
    return k;
}
// FP64 decisions inside the bands, kept out of line: inlined, the compiler may evaluate
// them for every pair (predicated), and FP64 runs at a small fraction of the FP32 rate here
static __device__ __noinline__ bool hin_exact(float px, float py, float qx, float qy, double H2d) {
    const double ex = __dsub_rn((double)px, (double)qx);
    const double ey = __dsub_rn((double)py, (double)qy);
    return __dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)) < H2d;
}
static __device__ __noinline__ bool vin_exact(float pz, float qz, double Vd) {
    return fabs(__dsub_rn((double)pz, (double)qz)) < Vd;
}
static __device__ __noinline__ bool below_terrain_exact(const Model& m, float x, float y, float z) {
    return (double)z < terrain64(m, (double)x, (double)y);
}

// h2: squared horizontal distance, dz: |vertical distance|; hin / vin: inside the minima
static __device__ __forceinline__ void sep_pair(const SepConsts& k, float px, float py, float pz, float qx, float qy,
                                         float qz, float& h2, float& dz, bool& hin, bool& vin) {
    const float dx = __fsub_rn(px, qx), dy = __fsub_rn(py, qy);
    dz = fabsf(__fsub_rn(pz, qz));
    h2 = __fmaf_rn(dx, dx, __fmul_rn(dy, dy));
    hin = h2 < k.H2;  // NaN (empty slot): false
    vin = dz < k.Vm;
    if (fabsf(h2 - k.H2) < k.hband) hin = hin_exact(px, py, qx, qy, k.H2d);
    if (fabsf(dz - k.Vm) < k.vband) vin = vin_exact(pz, qz, k.Vd);
}

// Terrain collision of one sample: fp32 outside a band around the surface, FP64 inside it.
static __device__ __forceinline__ bool below_terrain(const Model& m, float x, float y, float z) {
    const float c = z - terrain32(m, x, y);
    bool below = c < 0.f;
    if (fabsf(c) < kTerrBand) below = below_terrain_exact(m, x, y, z);
    return below;
}

}  // namespace fmdp
