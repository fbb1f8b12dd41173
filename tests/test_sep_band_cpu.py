"""The separation test's FP64 re-decision bands (csrc/sep_pair.cuh), checked on the host.

Every kernel decides a pair of fp32 samples in fp32 (dx = fl(px - qx), h2 = fma(dx, dx,
fl(dy * dy)), |dz| = |fl(pz - qz)|) and decides again in FP64, from the same fp32 inputs as
the oracle does, only when h2 lies within 16 fp32 ulps of H^2 = fl(fl(sep_h)^2) or |dz|
within 16 ulps of V = fl(sep_v). The rounding bound behind that width says the fp32 and
FP64 decisions agree outside the bands. Here numpy's IEEE fp32 arithmetic reproduces the
kernels' steps (the fused multiply-add as an exact float64 product plus a float64 sum,
rounded once more to fp32) on pairs placed within a few ulps to a few metres of the minima,
at coordinates from metres to hundreds of kilometres, and for minima that fp32 does not
represent exactly. Outside the bands every decision must match the FP64 one; inside them
(where the kernels use FP64) disagreements may occur, and the bands must stay narrow.
"""
import numpy as np
import pytest

F = np.float32


def kernel_bands(sep_h, sep_v):
    H = F(sep_h)
    H2 = F(H * H)
    Vm = F(sep_v)
    hband = max(F(H2 * F(2.0 ** -20)), F(2.0 ** -100))
    vband = max(F(Vm * F(2.0 ** -20)), F(2.0 ** -100))
    return H2, Vm, hband, vband


def pairs(rng, n, scale, sep_h, sep_v):
    """Pairs near the separation minima: horizontal distance sep_h (1 + d) with d from 1e-9
    to 1e-2, vertical distance sep_v (1 + d') likewise, at coordinates around `scale`."""
    px = (rng.uniform(-1, 1, n) * scale).astype(F)
    py = (rng.uniform(-1, 1, n) * scale).astype(F)
    pz = (rng.uniform(0, 1, n) * min(scale, 2e4)).astype(F)
    a = rng.uniform(0, 2 * np.pi, n)
    rel = np.exp(rng.uniform(np.log(1e-9), np.log(1e-2), n)) * rng.choice([-1.0, 1.0], n)
    relz = np.exp(rng.uniform(np.log(1e-9), np.log(1e-2), n)) * rng.choice([-1.0, 1.0], n)
    r = sep_h * (1.0 + rel)
    qx = (px.astype(np.float64) + r * np.cos(a)).astype(F)
    qy = (py.astype(np.float64) + r * np.sin(a)).astype(F)
    qz = (pz.astype(np.float64) + rng.choice([-1.0, 1.0], n) * sep_v * (1.0 + relz)).astype(F)
    return px, py, pz, qx, qy, qz


def decide(px, py, pz, qx, qy, qz, sep_h, sep_v, band_scale=1.0):
    """fp32 and FP64 decisions of each pair, band membership, and each pair's relative
    distance from the minima on the exact side."""
    H2, Vm, hband, vband = kernel_bands(sep_h, sep_v)
    hband, vband = F(hband * band_scale), F(vband * band_scale)
    dx = (px - qx).astype(F)
    dy = (py - qy).astype(F)
    m = (dy * dy).astype(F)
    h2 = (dx.astype(np.float64) * dx.astype(np.float64) + m.astype(np.float64)).astype(F)
    dz = np.abs((pz - qz).astype(F))
    hin32, vin32 = h2 < H2, dz < Vm
    in_hband = np.abs((h2 - H2).astype(F)) < hband
    in_vband = np.abs((dz - Vm).astype(F)) < vband
    # FP64 decisions from the same fp32 inputs, in the oracle's order (no contraction)
    ex = px.astype(np.float64) - qx.astype(np.float64)
    ey = py.astype(np.float64) - qy.astype(np.float64)
    hin64 = ex * ex + ey * ey < sep_h * sep_h
    vin64 = np.abs(pz.astype(np.float64) - qz.astype(np.float64)) < sep_v
    rel_h = np.abs((ex * ex + ey * ey) / (sep_h * sep_h) - 1.0)
    rel_v = np.abs(np.abs(pz.astype(np.float64) - qz.astype(np.float64)) / sep_v - 1.0)
    return hin32, vin32, in_hband, in_vband, hin64, vin64, rel_h, rel_v


@pytest.mark.parametrize("sep_h,sep_v", [(150.0, 30.0), (152.4, 30.48), (1852.0 / 3.0, 1000.0 / 3.0), (5.0, 1.0)])
@pytest.mark.parametrize("scale", [1e1, 3e4, 4e5])
def test_fp32_decisions_outside_the_bands_equal_fp64(sep_h, sep_v, scale):
    rng = np.random.default_rng(int(scale) + int(sep_h * 1000))
    hin32, vin32, in_hband, in_vband, hin64, vin64, rel_h, rel_v = decide(
        *pairs(rng, 400_000, scale, sep_h, sep_v), sep_h, sep_v)
    out_h, out_v = ~in_hband, ~in_vband
    assert np.array_equal(hin32[out_h], hin64[out_h])
    assert np.array_equal(vin32[out_v], vin64[out_v])
    # both sides of each minimum are sampled, some pairs fall inside the bands, and the bands
    # are narrow: a pair in one lies within about 16 fp32 ulps of the minimum (plus the
    # roundings of its own arithmetic), 40 x 2^-24 relative at most
    assert hin64.any() and (~hin64).any() and vin64.any() and (~vin64).any()
    assert in_hband.any() and in_vband.any()
    assert rel_h[in_hband].max() < 40 * 2.0 ** -24 and rel_v[in_vband].max() < 40 * 2.0 ** -24


def test_the_bands_are_needed():
    """Next to the minima the fp32 decision alone disagrees with FP64 (only inside the
    bands), and bands of one ulp instead of sixteen would let such pairs through."""
    rng = np.random.default_rng(7)
    hin32, vin32, in_hband, in_vband, hin64, vin64, _, _ = decide(*pairs(rng, 400_000, 4e5, 150.0, 30.0), 150.0, 30.0)
    wrong = (hin32 != hin64) | (vin32 != vin64)
    assert wrong.any()
    assert not (hin32 != hin64)[~in_hband].any() and not (vin32 != vin64)[~in_vband].any()
    hin32, vin32, in_hband, in_vband, hin64, vin64, _, _ = decide(*pairs(rng, 400_000, 4e5, 150.0, 30.0), 150.0, 30.0,
                                                                  band_scale=1.0 / 16)
    assert (hin32 != hin64)[~in_hband].any() or (vin32 != vin64)[~in_vband].any()
