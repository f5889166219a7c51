"""The margin behind the list build's settled hits (reading 20, extended).

On plans with the fixed-point list build, pass 1 takes separations as floats
relative to the item's first particle: each coordinate is the 32-bit
fixed-point difference to that particle, rounded to FP32 and scaled, and the
pair separation is the difference of two such floats.  A hit whose squared
separation there is below (H_i - delta)^2 is accepted without the exact test
on the fixed-point words (delta = 4e-6 of the largest box side).  These tests
emulate both computations in numpy at the worst magnitudes the plan allows
(offsets up to half the box) and check that they differ by far less than
delta, so the shortcut never accepts a pair the exact test would reject."""
import numpy as np

TWO32 = 4294967296.0


def _fixed(x, box):
    """X = round(x 2^32 / L) mod 2^32 per coordinate, as uint32."""
    k = np.rint(x * (TWO32 / box)).astype(np.int64)
    return (k & 0xFFFFFFFF).astype(np.uint32)


def _sep(xa, xb, unit):
    """FP32 of the signed fixed-point difference, times the FP32 unit."""
    d = (xa.astype(np.int64) - xb.astype(np.int64)) & 0xFFFFFFFF
    d = np.where(d >= 2 ** 31, d - 2 ** 32, d).astype(np.int32)
    return d.astype(np.float32) * unit


def _r2(dx, fused):
    if fused:       # the three products and sums rounded once (an upper bound on FMA's care)
        return (dx.astype(np.float64) ** 2).sum(axis=1).astype(np.float32)
    return (dx[:, 0] * dx[:, 0] + dx[:, 1] * dx[:, 1]) + dx[:, 2] * dx[:, 2]


def _case(seed, box, n=200_000):
    rng = np.random.Generator(np.random.PCG64(seed))
    box = np.asarray(box, np.float64)
    unit = (box / TWO32).astype(np.float32)
    delta = np.float32(4e-6 * box.max())
    ref = rng.random((n, 3)) * box
    # supports from 1e-4 to 4e-2 of the box; partners near r = H_i - delta
    H = np.exp(rng.uniform(np.log(1e-4), np.log(4e-2), n)) * box.max()
    # own particle as far from the reference as the plan allows: the item's
    # extent plus the support stays below half the box
    xi = ref + (rng.random((n, 3)) - 0.5) * 0.999 * (box - 2.0 * H[:, None])
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    r = H - float(delta) * rng.uniform(-2.0, 3.0, n)
    xj = xi + u * np.maximum(r, 0.0)[:, None]
    R, Xi, Xj = _fixed(ref, box), _fixed(xi % box, box), _fixed(xj % box, box)
    o0 = _sep(Xi, R, unit)
    r0 = _sep(Xj, R, unit)
    rel = (o0 - r0).astype(np.float32)
    fix = _sep(Xi, Xj, unit)
    Hf = H.astype(np.float32)
    return rel, fix, Hf, delta


def test_relative_floats_stay_far_inside_the_margin():
    for seed, box in ((11, (1.0, 1.0, 1.0)), (12, (1.0, 0.7, 1.3)), (13, (250.0, 250.0, 250.0))):
        rel, fix, _, delta = _case(seed, box)
        err = np.max(np.abs(rel.astype(np.float64) - fix.astype(np.float64)))
        assert err < delta / 8, (box, err, delta)


def test_settled_hits_are_inside_the_support_on_the_fixed_point_words():
    for seed, box in ((21, (1.0, 1.0, 1.0)), (22, (1.0, 0.7, 1.3))):
        rel, fix, Hf, delta = _case(seed, box)
        Hs = np.maximum(Hf - delta, np.float32(0.0)).astype(np.float32)
        for fused in (False, True):
            sure = _r2(rel, fused) < Hs * Hs
            inside = _r2(fix, fused) < Hf * Hf
            assert sure.sum() > 1000          # the band is actually exercised
            assert np.all(inside[sure]), (box, fused)
        # pairs just outside the margin are left to the exact test, not dropped
        near = (_r2(rel, False) >= Hs * Hs) & (_r2(fix, False) < Hf * Hf)
        assert near.sum() > 100
