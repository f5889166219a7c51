"""The synthetic inputs reproduce the statistics the paper states for its
workloads (Sec. 3.4)."""
import numpy as np

from paper_2606_23891_b300 import ics


def test_gresho_cell_occupancy_matches_the_paper():
    # Gresho256: 256^3 particles; min / max / mean / median particles per
    # cell 55 / 73 / 64 / 64 (Sec. 3.4).  Cells of four lattice spacings.
    x = ics.jittered_lattice(256, 0.52, 3)
    c = np.floor(x * 64).astype(np.int64).clip(0, 63)
    cnt = np.bincount(c[:, 0] + 64 * (c[:, 1] + 64 * c[:, 2]), minlength=64 ** 3)
    assert (cnt.min(), cnt.max(), cnt.mean(), np.median(cnt)) == (55, 73, 64.0, 64.0)


def test_gresho_fields_are_the_vortex():
    f = ics.gresho(n_side=32)
    r = np.hypot(f["x"][:, 0] - 0.5, f["x"][:, 1] - 0.5)
    vphi = np.hypot(f["v"][:, 0], f["v"][:, 1])
    np.testing.assert_allclose(vphi, ics.gresho_vphi(r), atol=1e-6)
    # rotation is counter-clockwise about the z axis and has no z component
    assert np.all(f["v"][:, 2] == 0)
    lz = (f["x"][:, 0] - 0.5) * f["v"][:, 1] - (f["x"][:, 1] - 0.5) * f["v"][:, 0]
    assert np.all(lz >= -1e-7)
    # pressure is continuous at r = 0.2 and 0.4 and balances the rotation:
    # dP/dr = rho v_phi^2 / r
    for r0 in (0.2, 0.4):
        p = ics.gresho_pressure(np.array([r0 - 1e-9, r0 + 1e-9]))
        assert abs(p[0] - p[1]) < 1e-7
    rr = np.array([0.05, 0.1, 0.25, 0.3, 0.35, 0.45])
    e = 1e-6
    dp = (ics.gresho_pressure(rr + e) - ics.gresho_pressure(rr - e)) / (2 * e)
    np.testing.assert_allclose(dp, ics.gresho_vphi(rr) ** 2 / rr, atol=1e-5)
    np.testing.assert_allclose(f["mass"].astype(np.float64).sum(), 1.0, rtol=1e-6)


def test_generators_are_seeded():
    a = ics.jittered_lattice(8, 0.3, 5)
    b = ics.jittered_lattice(8, 0.3, 5)
    c = ics.jittered_lattice(8, 0.3, 6)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.min() >= 0.0 and a.max() < 1.0


def test_lognormal_recipe():
    """Clustered set: equal masses, positions in the box, a wide spread of
    smoothing lengths with neighbour counts near the target (scipy KD-tree
    count), and reproducible draws."""
    from scipy.spatial import cKDTree
    f = ics.lognormal(n_side=32, seed=21)
    n = 32 ** 3
    assert f["x"].shape == (n, 3)
    assert np.all((f["x"] >= 0) & (f["x"] < 1))
    assert np.all(f["mass"] == np.float32(1.0 / n))
    H = 1.825742 * f["h"].astype(np.float64)
    assert H.max() / H.min() > 5
    assert H.max() < 0.5
    cnt = cKDTree(f["x"], boxsize=1.0).query_ball_point(f["x"], H, return_length=True) - 1
    assert 40 < np.median(cnt) < 56
    assert cnt.min() >= 4
    g = ics.lognormal(n_side=32, seed=21)
    for k in ("x", "v", "h", "u", "alpha_visc"):
        np.testing.assert_array_equal(f[k], g[k])
