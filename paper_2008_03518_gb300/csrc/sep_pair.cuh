// Separation test of one pair of samples (Sec. V: a conflict is a pair closer than the
// horizontal minimum and the vertical minimum at the same step), shared by every kernel
// that measures a pair, so that they all decide it the same way.
#pragma once

#include "fmdp_internal.cuh"

namespace fmdp {

// Separation minima of one sample pair with explicit rounding (no contraction), so that
// every kernel that measures the same pair gets the same bits. Thresholds in the band
// around H^2 and V are decided again in FP64 from the same fp32 inputs.
struct SepConsts {
    float H2, Vm, hband;
    double H2d, Vd;
};
static __device__ __forceinline__ SepConsts sep_consts(double sep_h, double sep_v) {
    SepConsts k;
    const float H = (float)sep_h;
    k.H2 = __fmul_rn(H, H);
    k.Vm = (float)sep_v;
    k.hband = 2.0f * H * kSepBand + kSepBand * kSepBand;
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
    if (fabsf(dz - k.Vm) < kSepBand) vin = vin_exact(pz, qz, k.Vd);
}

// Terrain collision of one sample: fp32 outside a band around the surface, FP64 inside it.
static __device__ __forceinline__ bool below_terrain(const Model& m, float x, float y, float z) {
    const float c = z - terrain32(m, x, y);
    bool below = c < 0.f;
    if (fabsf(c) < kTerrBand) below = below_terrain_exact(m, x, y, z);
    return below;
}

}  // namespace fmdp
