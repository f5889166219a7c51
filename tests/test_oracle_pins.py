"""Pins of the CPU oracle against facts it does not compute itself: closed
forms, library routines, conservation laws and finite differences.  Each test
is chosen so that a plausible slip in the oracle (a dropped term, a sign, a
wrong index or factor) fails it."""
import ctypes as C
import math

import numpy as np
import pytest
from scipy import integrate
from scipy.spatial import cKDTree

import oracle
from paper_2606_23891_b300 import ics


# ---------------------------------------------------------------- kernel ---
@pytest.mark.parametrize("H", [0.37, 1.0, 2.5])
def test_kernel_volume_integral_is_one(H):
    f = lambda r: 4.0 * math.pi * r * r * oracle.W(r, H)
    val = integrate.quad(f, 0.0, 0.5 * H, epsabs=1e-14, epsrel=1e-13)[0] + \
        integrate.quad(f, 0.5 * H, H, epsabs=1e-14, epsrel=1e-13)[0]
    assert abs(val - 1.0) < 1e-10


def test_kernel_shape_and_continuity():
    L = oracle.lib()
    assert L.oracle_w(0.0) == 1.0
    assert L.oracle_w(1.0) == 0.0 and L.oracle_w(1.7) == 0.0
    for q0 in (0.5, 1.0):
        for fn in (L.oracle_w, L.oracle_dw):
            assert abs(fn(q0 - 1e-12) - fn(q0 + 1e-12)) < 1e-9
    assert L.oracle_dw(0.0) == 0.0          # smooth at the origin
    assert oracle.W(2.0, 2.0) == 0.0


@pytest.mark.parametrize("q", [0.05, 0.3, 0.49, 0.51, 0.75, 0.97])
def test_kernel_derivatives_match_finite_differences(q):
    H = 0.8
    r = q * H
    e = 1e-6
    fd_r = (oracle.W(r + e, H) - oracle.W(r - e, H)) / (2 * e)
    fd_H = (oracle.W(r, H + e) - oracle.W(r, H - e)) / (2 * e)
    assert abs(oracle.dWdr(r, H) - fd_r) <= 1e-6 * max(1.0, abs(fd_r))
    assert abs(oracle.dWdH(r, H) - fd_H) <= 1e-6 * max(1.0, abs(fd_H))


# ------------------------------------------------------- neighbour search ---
def _random_box(n, seed, hmin=0.06, hmax=0.09):
    rng = np.random.Generator(np.random.PCG64(seed))
    f = ics.empty_fields(n)
    f["x"][:] = rng.uniform(0.0, 1.0, (n, 3))
    f["v"][:] = rng.uniform(-1, 1, (n, 3)).astype(np.float32)
    f["mass"][:] = rng.uniform(0.5, 1.5, n).astype(np.float32) / n
    f["h"][:] = rng.uniform(hmin, hmax, n).astype(np.float32)
    f["u"][:] = rng.uniform(0.5, 2.0, n).astype(np.float32)
    f["alpha_visc"][:] = rng.uniform(0.1, 1.0, n).astype(np.float32)
    f["alpha_diff"][:] = rng.uniform(0.0, 0.5, n).astype(np.float32)
    f["id"][:] = np.arange(n)
    return f


def test_neighbour_counts_match_periodic_kdtree():
    f = _random_box(600, seed=11)
    P = oracle.params()
    H = oracle.KERNEL_GAMMA * f["h"].astype(np.float64)
    tree = cKDTree(f["x"], boxsize=1.0)
    for i in range(0, 600, 7):
        _, pairs = oracle.density(f, P, [i])
        ref = len(tree.query_ball_point(f["x"][i], H[i])) - 1
        assert pairs == ref
        # force loop: r < max(H_i, H_j)
        cand = tree.query_ball_point(f["x"][i], H.max())
        d = f["x"][cand] - f["x"][i]
        d -= np.rint(d)
        r = np.sqrt((d * d).sum(1))
        ref_f = int(((r < np.maximum(H[i], H[cand])) & (np.array(cand) != i)).sum())
        g = {k: np.ones(600) for k in ("rho", "f_gradh", "pressure",
                                        "soundspeed", "balsara")}
        _, pf = oracle.force(f, P, g, [i])
        assert pf == ref_f


# ---------------------------------------------------------------- density ---
def test_perfect_lattice_density_is_the_lattice_sum():
    n_side = 10
    f = ics.uniform_lattice(n_side=n_side, jitter=0.0)
    f["h"][:] = np.float32(1.7 / n_side)
    P = oracle.params()
    sel = [0, 137, 999]
    raw, _ = oracle.density(f, P, sel)
    gh = oracle.ghost(f, P, raw, sel)
    H = oracle.KERNEL_GAMMA * float(f["h"][0])
    dx = 1.0 / n_side
    m = float(f["mass"][0])
    kmax = int(math.ceil(H / dx))
    rho = 0.0
    wc = 0.0
    for a in range(-kmax, kmax + 1):
        for b in range(-kmax, kmax + 1):
            for c in range(-kmax, kmax + 1):
                r = dx * math.sqrt(a * a + b * b + c * c)
                if r < H:
                    rho += m * oracle.W(r, H)
                    wc += 4.0 / 3.0 * math.pi * H ** 3 * oracle.W(r, H)
    np.testing.assert_allclose(gh[:, 0], rho, rtol=1e-12)
    np.testing.assert_allclose(gh[:, 2], wc, rtol=1e-12)
    assert abs(rho - 1.0) < 0.05          # a lattice is a fair density estimate


def test_grad_h_factor_follows_h_of_rho():
    # Omega = 1 - (dh/drho)(d rho/dh) with h = eta (m/rho)^(1/3): both
    # derivatives taken numerically, independently of the oracle's ghost
    f = ics.perturb(ics.uniform_lattice(n_side=9, jitter=0.3, seed=5), seed=6,
                    h_amp=0.1)
    P = oracle.params()
    for i in (7, 300):
        raw, _ = oracle.density(f, P, [i])
        g0 = oracle.ghost(f, P, raw, [i])[0]
        rho, h, m = g0[0], float(f["h"][i]), float(f["mass"][i])
        vals, hs = [], []
        for s in (1.0 - 1e-3, 1.0 + 1e-3):
            g = {k: v.copy() for k, v in f.items()}
            g["h"][i] = np.float32(h * s)
            r2, _ = oracle.density(g, P, [i])
            vals.append(oracle.ghost(g, P, r2, [i])[0][0])
            hs.append(float(g["h"][i]))
        drho_dh = (vals[1] - vals[0]) / (hs[1] - hs[0])
        eta = h / (m / rho) ** (1.0 / 3.0)
        e = 1e-6 * rho
        dh_drho = (eta * (m / (rho + e)) ** (1 / 3) - eta * (m / (rho - e)) ** (1 / 3)) / (2 * e)
        omega = 1.0 - dh_drho * drho_dh
        assert abs(g0[8] - 1.0 / omega) < 1e-5


def test_h_derivatives_match_finite_differences_in_h():
    f = ics.perturb(ics.uniform_lattice(n_side=9, jitter=0.3, seed=5), seed=6,
                    h_amp=0.1)
    P = oracle.params()
    for i in (3, 200, 511):
        raw, _ = oracle.density(f, P, [i])
        g0 = oracle.ghost(f, P, raw, [i])[0]
        vals = []
        Hs = []
        for s in (1.0 - 1e-3, 1.0 + 1e-3):
            g = {k: v.copy() for k, v in f.items()}
            g["h"][i] = np.float32(f["h"][i] * s)
            r2, _ = oracle.density(g, P, [i])
            vals.append(oracle.ghost(g, P, r2, [i])[0])
            Hs.append(oracle.KERNEL_GAMMA * float(g["h"][i]))
        dH = Hs[1] - Hs[0]
        fd_rho = (vals[1][0] - vals[0][0]) / dH
        fd_wc = (vals[1][2] - vals[0][2]) / dH
        scale = 3.0 * g0[0] / Hs[0]
        assert abs(g0[1] - fd_rho) < 1e-5 * scale
        assert abs(g0[3] - fd_wc) < 1e-5 * abs(fd_wc)


def _lattice_with_velocity(n_side, vfun):
    f = ics.uniform_lattice(n_side=n_side, jitter=0.0)
    f["v"][:] = vfun(f["x"]).astype(np.float32)
    return f


def test_div_and_curl_of_sinusoidal_fields():
    n_side = 40
    A = 0.1
    k = 2 * math.pi
    # v = (A sin kx, 0, 0): div v = A k cos kx
    f = _lattice_with_velocity(n_side, lambda x: np.stack(
        [A * np.sin(k * x[:, 0]), 0 * x[:, 0], 0 * x[:, 0]], 1))
    P = oracle.params()
    sel = np.array([0, 5, 13, 27, 1000, 20000, 41111])
    raw, _ = oracle.density(f, P, sel)
    gh = oracle.ghost(f, P, raw, sel)
    ref = A * k * np.cos(k * f["x"][sel, 0])
    assert np.max(np.abs(gh[:, 4] - ref)) < 0.03 * A * k
    assert np.max(np.abs(gh[:, 5:8])) < 1e-6 * A * k
    # v = (-A sin ky, A sin kx, 0): curl_z = A k (cos kx + cos ky), div = 0
    f = _lattice_with_velocity(n_side, lambda x: np.stack(
        [-A * np.sin(k * x[:, 1]), A * np.sin(k * x[:, 0]), 0 * x[:, 0]], 1))
    raw, _ = oracle.density(f, P, sel)
    gh = oracle.ghost(f, P, raw, sel)
    ref = A * k * (np.cos(k * f["x"][sel, 0]) + np.cos(k * f["x"][sel, 1]))
    assert np.max(np.abs(gh[:, 7] - ref)) < 0.03 * 2 * A * k
    assert np.max(np.abs(gh[:, 4])) < 1e-6 * A * k
    # v = A (sin ky, sin kz, sin kx): curl v = -A k (cos kz, cos kx, cos ky)
    f = _lattice_with_velocity(n_side, lambda x: A * np.stack(
        [np.sin(k * x[:, 1]), np.sin(k * x[:, 2]), np.sin(k * x[:, 0])], 1))
    raw, _ = oracle.density(f, P, sel)
    gh = oracle.ghost(f, P, raw, sel)
    xs = f["x"][sel]
    ref = -A * k * np.stack([np.cos(k * xs[:, 2]), np.cos(k * xs[:, 0]),
                             np.cos(k * xs[:, 1])], 1)
    assert np.max(np.abs(gh[:, 5:8] - ref)) < 0.03 * A * k


def test_balsara_switch_separates_shear_from_compression():
    n_side = 40
    A, k = 0.1, 2 * math.pi
    P = oracle.params()
    sel = np.array([0, 5, 13, 27, 1000, 20000])
    shear = _lattice_with_velocity(n_side, lambda x: np.stack(
        [A * np.sin(k * x[:, 1]), 0 * x[:, 0], 0 * x[:, 0]], 1))
    comp = _lattice_with_velocity(n_side, lambda x: np.stack(
        [A * np.sin(k * x[:, 0]), 0 * x[:, 0], 0 * x[:, 0]], 1))
    for f in (shear, comp):
        f["alpha_visc"][:] = 1.0
    os_ = oracle.chain(shear, P, sel)
    oc = oracle.chain(comp, P, sel)
    assert np.all(os_["balsara"] < 1e-4)
    far = np.abs(np.cos(k * comp["x"][sel, 0])) > 0.3
    assert np.all(oc["balsara"][far] > 0.95)
    # equal divergence and curl magnitudes: B = 1/2 (up to eps c/h)
    mixed = _lattice_with_velocity(n_side, lambda x: A * np.stack(
        [np.sin(k * x[:, 0]), np.sin(k * x[:, 0]), 0 * x[:, 0]], 1))
    om = oracle.chain(mixed, P, sel)
    assert np.all(np.abs(om["balsara"][far] - 0.5) < 0.01)
    # pure shear: the switch removes viscous heating, and the pressure work
    # vanishes with div v, so du/dt ~ 0 although the flow is sheared
    assert np.max(np.abs(os_["u_dt"])) < 1e-3 * A * k * os_["pressure"].max()


# --------------------------------------------------------------- gradient ---
def test_gradient_closed_forms():
    f = ics.uniform_lattice(n_side=8, jitter=0.2, seed=3, u0=2.0)
    P = oracle.params()
    out = oracle.chain(f, P)
    c = math.sqrt(oracle.GAMMA * (oracle.GAMMA - 1.0) * 2.0)
    np.testing.assert_allclose(out["v_sig_grad"], 2 * c, rtol=1e-14)
    np.testing.assert_allclose(out["soundspeed"], c, rtol=1e-14)
    assert np.max(np.abs(out["laplace_u"])) == 0.0
    np.testing.assert_allclose(out["pressure"], (oracle.GAMMA - 1) * out["rho"] * 2.0,
                               rtol=1e-14)


def test_laplacian_of_sinusoidal_energy():
    n_side = 40
    f = ics.uniform_lattice(n_side=n_side, jitter=0.0)
    A = 0.05
    k = 2 * math.pi
    f["u"][:] = (1.0 + A * np.sin(k * f["x"][:, 0])).astype(np.float32)
    P = oracle.params()
    sel = np.array([3, 17, 29, 33000])
    out = oracle.chain(f, P, sel)
    ref = -A * k * k * np.sin(k * f["x"][sel, 0])
    assert np.max(np.abs(out["laplace_u"] - ref)) < 0.03 * A * k * k


def test_signal_velocity_sees_approach_speed():
    # two particle streams approaching along x: v_sig = 2c + beta |v_ij . rhat|
    f = ics.uniform_lattice(n_side=8, jitter=0.0)
    f["v"][:, 0] = np.where(f["x"][:, 0] < 0.5, 1.0, -1.0).astype(np.float32)
    P = oracle.params()
    out = oracle.chain(f, P)
    c = math.sqrt(oracle.GAMMA * (oracle.GAMMA - 1.0))
    # a particle at the interface sees an on-axis neighbour closing at speed 2
    assert abs(out["v_sig_grad"].max() - (2 * c + 3.0 * 2.0)) < 1e-12
    assert abs(out["v_sig"].max() - (2 * c + 3.0 * 2.0)) < 1e-12
    assert abs(out["v_sig"].min() - 2 * c) < 1e-12       # receding side


# ------------------------------------------------------------------ force ---
def test_force_vanishes_on_a_static_uniform_lattice():
    f = ics.uniform_lattice(n_side=8, jitter=0.0)
    P = oracle.params()
    out = oracle.chain(f, P)
    term = out["pressure"].max() / out["rho"].max() ** 2 * abs(
        oracle.dWdr(0.5 * oracle.KERNEL_GAMMA * float(f["h"][0]),
                    oracle.KERNEL_GAMMA * float(f["h"][0]))) * float(f["mass"][0])
    assert np.max(np.abs(out["a"])) < 1e-10 * term
    assert np.max(np.abs(out["u_dt"])) < 1e-10 * term


@pytest.fixture(scope="module")
def turbulent():
    f = ics.perturb(ics.uniform_lattice(n_side=10, jitter=0.35, seed=21,
                                        alpha_visc=1.0), seed=22, v_amp=0.5,
                    u_amp=0.3, alpha_diff=0.6, h_amp=0.12)
    rng = np.random.Generator(np.random.PCG64(23))
    f["alpha_visc"][:] = rng.uniform(0.2, 2.0, f["alpha_visc"].shape).astype(np.float32)
    P = oracle.params()
    return f, P, oracle.chain(f, P)


def test_force_conserves_momentum(turbulent):
    f, P, out = turbulent
    m = f["mass"].astype(np.float64)
    tot = (m[:, None] * out["a"]).sum(0)
    scale = (m[:, None] * np.abs(out["a"])).sum(0)
    assert np.all(np.abs(tot) < 1e-12 * scale)


def test_force_conserves_energy(turbulent):
    f, P, out = turbulent
    m = f["mass"].astype(np.float64)
    v = f["v"].astype(np.float64)
    kin = (m * (v * out["a"]).sum(1))
    th = m * out["u_dt"]
    assert abs(kin.sum() + th.sum()) < 1e-12 * (np.abs(kin).sum() + np.abs(th).sum())
    assert np.abs(th).sum() > 0 and np.abs(kin).sum() > 0


def test_conduction_alone_conserves_thermal_energy():
    f = ics.perturb(ics.uniform_lattice(n_side=9, jitter=0.3, seed=31), seed=32,
                    u_amp=0.5, alpha_diff=0.8, h_amp=0.1)
    f["alpha_visc"][:] = 0.0
    P = oracle.params()
    out = oracle.chain(f, P)
    m = f["mass"].astype(np.float64)
    # with v = 0 only conduction changes u: total thermal energy is constant
    th = m * out["u_dt"]
    assert np.abs(th).sum() > 0
    assert abs(th.sum()) < 1e-12 * np.abs(th).sum()
    # heat flows from hot to cold: the u-weighted rate is negative
    assert (th * f["u"]).sum() < 0.0


def test_dh_dt_equals_h_f_div_v_over_three(turbulent):
    f, P, out = turbulent
    h = f["h"].astype(np.float64)
    ref = h / 3.0 * out["f_gradh"] * out["div_v"]
    np.testing.assert_allclose(out["h_dt"], ref, rtol=1e-10,
                               atol=1e-12 * np.abs(ref).max())


def test_inactive_particles_are_not_updated():
    f = ics.perturb(ics.uniform_lattice(n_side=8, jitter=0.3, seed=41), seed=42,
                    v_amp=0.3)
    f["time_bin"][::2] = 3
    P = oracle.params(active_bin=2)
    out = oracle.chain(f, P)
    assert np.all(out["a"][::2] == 0.0) and np.all(out["v_sig"][::2] == 0.0)
    assert np.all(out["v_sig"][1::2] > 0.0)


# ---------------------------------------------------- cells, tasks, shifts ---
def test_tasks_cover_every_interacting_pair_exactly_once():
    f = _random_box(1500, seed=51, hmin=0.04, hmax=0.07)
    g = oracle.grid(f)
    assert g is not None
    nc, perm, cs = g
    H = oracle.KERNEL_GAMMA * f["h"].astype(np.float64)
    assert np.all(1.0 / nc >= H.max())
    ci, cj, sh = oracle.tasks(nc, cs)
    cell_of = np.empty(1500, np.int64)
    for c in range(len(cs) - 1):
        cell_of[perm[cs[c]:cs[c + 1]]] = c
    # the permutation is the stable sort of the particles' cells
    assert np.all(np.diff(cell_of[perm]) >= 0)
    tree = cKDTree(f["x"], boxsize=1.0)
    ref = set()
    for i, j in tree.query_pairs(H.max()):
        d = f["x"][i] - f["x"][j]
        d -= np.rint(d)
        if np.sqrt((d * d).sum()) < max(H[i], H[j]):
            ref.add((min(i, j), max(i, j)))
    seen = {}
    x = f["x"]
    for t in range(len(ci)):
        a = perm[cs[ci[t]]:cs[ci[t] + 1]]
        if cj[t] < 0:
            for p in range(len(a)):
                for q in range(p + 1, len(a)):
                    i, j = a[p], a[q]
                    d = x[i] - x[j]
                    r = math.sqrt((d * d).sum())
                    if r < max(H[i], H[j]):
                        k = (min(i, j), max(i, j))
                        seen[k] = seen.get(k, 0) + 1
            continue
        b = perm[cs[cj[t]]:cs[cj[t] + 1]]
        xb = x[b] + sh[t].astype(np.float64)
        for p, i in enumerate(a):
            d = x[i] - xb
            r = np.sqrt((d * d).sum(1))
            for q in np.nonzero(r < np.maximum(H[i], H[b]))[0]:
                k = (min(i, b[q]), max(i, b[q]))
                seen[k] = seen.get(k, 0) + 1
    assert set(seen) == ref
    assert all(v == 1 for v in seen.values())


def test_grid_rejects_supports_too_large_for_three_cells():
    f = _random_box(200, seed=61, hmin=0.2, hmax=0.25)
    assert oracle.grid(f) is None


def test_bundles_respect_the_slot_budget():
    f = ics.uniform_lattice(n_side=12, jitter=0.45, seed=71)
    nc, perm, cs = oracle.grid(f)
    ci, cj, sh = oracle.tasks(nc, cs)
    cnt = np.diff(cs)
    slots = cnt[ci] + np.where(cj >= 0, cnt[np.maximum(cj, 0)], 0)
    for budget in (0, 1, 500, 4000):
        bs = oracle.bundles(ci, cj, cs, budget)
        assert bs[0] == 0 and bs[-1] == len(ci) and np.all(np.diff(bs) >= 1)
        for b in range(len(bs) - 1):
            s = slots[bs[b]:bs[b + 1]].sum()
            assert budget <= 0 or s <= budget or bs[b + 1] - bs[b] == 1
            if budget > 0 and b + 1 < len(bs) - 1:
                assert s + slots[bs[b + 1]] > budget   # greedy: next task overflows


# ---------------------------------------------------------- pack, unpack ---
def _lane_views(buf, sizes, S):
    out, off = [], 0
    for sz in sizes:
        out.append(buf[off:off + S * sz])
        off += (S * sz + 255) // 256 * 256
    assert off == len(buf)
    return out


def test_pack_gathers_views_with_periodic_shift():
    f = ics.perturb(ics.uniform_lattice(n_side=12, jitter=0.45, seed=81), seed=82,
                    v_amp=0.3, u_amp=0.2, alpha_diff=0.3)
    rng = np.random.Generator(np.random.PCG64(83))
    for k in ("rho", "f_gradh", "balsara"):
        f[k][:] = rng.uniform(0.5, 1.5, f[k].shape).astype(np.float32)
    f["time_bin"][:] = rng.integers(0, 5, f["time_bin"].shape).astype(np.int8)
    nc, perm, cs = oracle.grid(f)
    ci, cj, sh = oracle.tasks(nc, cs)
    t0, t1 = 5, 60
    # slot -> particle and shift, listed independently of the oracle
    parts, shifts = [], []
    for t in range(t0, t1):
        for side, c in ((0, ci[t]), (1, cj[t])):
            if c < 0:
                continue
            idx = perm[cs[c]:cs[c + 1]]
            parts.append(idx)
            shifts.append(np.tile(sh[t] if side else np.zeros(3, np.int8), (len(idx), 1)))
    p = np.concatenate(parts)
    s = np.concatenate(shifts).astype(np.float64)
    S = len(p)
    buf = oracle.pack(oracle.FORCE, f, perm, cs, ci, cj, sh, t0, t1)
    lanes = _lane_views(buf, [8, 8, 8, 16, 4, 4, 4, 4, 4, 4, 4, 1], S)
    for d in range(3):
        np.testing.assert_array_equal(lanes[d].view(np.float64), f["x"][p, d] + s[:, d])
    vm = lanes[3].view(np.float32).reshape(S, 4)
    np.testing.assert_array_equal(vm[:, :3], f["v"][p])
    np.testing.assert_array_equal(vm[:, 3], f["mass"][p])
    for lane, k in zip(lanes[4:11], ("h", "u", "rho", "f_gradh", "balsara",
                                     "alpha_visc", "alpha_diff")):
        np.testing.assert_array_equal(lane.view(np.float32), f[k][p])
    np.testing.assert_array_equal(lanes[11].view(np.int8), f["time_bin"][p])
    # density view is the prefix of the force view
    bd = oracle.pack(oracle.DENSITY, f, perm, cs, ci, cj, sh, t0, t1)
    ld = _lane_views(bd, [8, 8, 8, 16, 4], S)
    for a, b in zip(ld, lanes[:5]):
        np.testing.assert_array_equal(a, b)


def test_unpack_is_a_compensated_sum_and_a_max():
    f = ics.uniform_lattice(n_side=12, jitter=0.45, seed=91)
    nc, perm, cs = oracle.grid(f)
    ci, cj, sh = oracle.tasks(nc, cs)
    t0, t1 = 0, len(ci)
    parts = []
    for t in range(t0, t1):
        for c in (ci[t], cj[t]):
            if c >= 0:
                parts.append(perm[cs[c]:cs[c + 1]])
    p = np.concatenate(parts)
    S = len(p)
    n = f["x"].shape[0]
    eps = 2.0 ** -24
    for loop, sizes in ((oracle.DENSITY, [16, 16]), (oracle.GRADIENT, [8]),
                        (oracle.FORCE, [16, 8])):
        nbytes = oracle.buffer_bytes(loop, 1, S)
        buf = ics.random_result_lanes(nbytes, seed=92 + loop)
        g = ics.empty_fields(n)
        g["x"] = f["x"]
        oracle.unpack(loop, g, perm, cs, ci, cj, t0, t1, buf)
        lanes = _lane_views(buf, sizes, S)
        cols = np.concatenate([l.view(np.float32).reshape(S, -1) for l in lanes], 1)
        nslot = np.bincount(p, minlength=n)

        def check_sum(got, col):
            # exact sum (float64 is exact for <= 27 floats in [-1,1)) against
            # Kahan's bound (2u + O(n u^2)) sum|x|, u = 2^-24 (Higham, Acc. and
            # Stab. of Num. Alg., 4.3) ...
            exact = np.bincount(p, weights=cols[:, col].astype(np.float64), minlength=n)
            mag = np.bincount(p, weights=np.abs(cols[:, col]).astype(np.float64), minlength=n)
            err = np.abs(got.astype(np.float64) - exact)
            assert np.all(err <= (2 * eps + 4 * nslot * eps * eps) * mag)
            # ... and clearly better than a plain float32 running sum in the
            # same order (numpy's unbuffered add.at adds in input order)
            plain = np.zeros(n, np.float32)
            np.add.at(plain, p, cols[:, col])
            err_plain = np.abs(plain.astype(np.float64) - exact)
            assert err.mean() < 0.5 * err_plain.mean()

        def smax(col):
            out = np.zeros(n, np.float32)
            np.maximum.at(out, p, cols[:, col])
            return out
        if loop == oracle.DENSITY:
            for col, k in enumerate(("rho", "rho_dh", "wcount", "wcount_dh", "div_v")):
                check_sum(g[k], col)
            for c in range(3):
                check_sum(g["rot_v"][:, c], 5 + c)
        elif loop == oracle.GRADIENT:
            np.testing.assert_array_equal(g["v_sig_grad"], smax(0))
            check_sum(g["laplace_u"], 1)
        else:
            for c in range(3):
                check_sum(g["a"][:, c], c)
            check_sum(g["u_dt"], 3)
            check_sum(g["h_dt"], 4)
            np.testing.assert_array_equal(g["v_sig"], smax(5))


def test_unpack_folds_from_the_stored_value():
    # two bundles give the same sums as one when the second starts from the
    # first's stored result (the fold restarts its compensation per bundle)
    f = ics.uniform_lattice(n_side=12, jitter=0.45, seed=93)
    nc, perm, cs = oracle.grid(f)
    ci, cj, sh = oracle.tasks(nc, cs)
    n = f["x"].shape[0]
    bs = oracle.bundles(ci, cj, cs, 3000)
    assert len(bs) > 2
    g = ics.empty_fields(n)
    g["x"] = f["x"]
    total = np.zeros(n)
    for b in range(len(bs) - 1):
        S = oracle.bundle_slots(ci, cj, cs, bs[b], bs[b + 1])
        buf = ics.random_result_lanes(oracle.buffer_bytes(oracle.GRADIENT, 1, S), seed=b)
        oracle.unpack(oracle.GRADIENT, g, perm, cs, ci, cj, bs[b], bs[b + 1], buf)
        parts = []
        for t in range(bs[b], bs[b + 1]):
            for c in (ci[t], cj[t]):
                if c >= 0:
                    parts.append(perm[cs[c]:cs[c + 1]])
        pp = np.concatenate(parts)
        vals = buf[: 8 * S].view(np.float32).reshape(S, 2)[:, 1]
        total += np.bincount(pp, weights=vals.astype(np.float64), minlength=n)
    assert np.max(np.abs(g["laplace_u"] - total)) < 1e-5


# ----------------------------------------------------------------- layouts ---
_CT = {0: (C.c_double * 3), 1: (C.c_float * 3), 2: (C.c_float * 3), 8: C.c_int8,
       15: (C.c_float * 3), 24: C.c_int64, 25: (C.c_uint8 * 8)}


def _ctype(fid, comp):
    if comp >= 0:
        return C.c_double if fid == 0 else C.c_float
    return _CT.get(fid, C.c_float)


@pytest.mark.parametrize("layout", range(11))
def test_layout_records_match_c_struct_rules(layout):
    groups = oracle.layout_groups(layout, seed=7)
    seen = []
    for rec, mem in groups:
        fields = [("m%d" % k, _ctype(fid, comp)) for k, (fid, comp, off) in enumerate(mem)]
        S = type("S", (C.Structure,), {"_fields_": fields})
        assert C.sizeof(S) == rec
        for k, (fid, comp, off) in enumerate(mem):
            assert getattr(S, "m%d" % k).offset == off
            seen.append((fid, comp))
    # every field (or every component, for SoA) is stored exactly once, except
    # the density view's inputs in the replicated layout, stored twice
    names = oracle.FIELD_NAMES
    want = []
    for fid, name in enumerate(names):
        ncomp = 3 if name in ("x", "v", "a", "rot_v") else 1
        if layout == 8 and ncomp == 3:
            want += [(fid, c) for c in range(3)]
        else:
            want.append((fid, -1))
        if layout == 9 and name in ("x", "v", "mass", "h"):
            want.append((fid, -1))
    assert sorted(seen) == sorted(want)


def test_aos_record_is_the_papers_160_bytes():
    # 2.5 GiB of particle data for 256^3 particles (Sec. 3.4)
    assert 2.5 * 2 ** 30 / 256 ** 3 == 160.0
    assert oracle.layout_groups(0)[0][0] == 160


def test_splitmix64_published_first_output():
    # SplitMix64 seeded with 0 returns 0xE220A8397B1DCDAF first (the value
    # of java.util.SplittableRandom(0).nextLong(), -2152535657050944081)
    assert oracle.splitmix64(0, 1)[0] == 0xE220A8397B1DCDAF


def test_random_order_layout_is_a_seeded_shuffle():
    a = [fid for fid, _, _ in oracle.layout_groups(1, seed=3)[0][1]]
    b = [fid for fid, _, _ in oracle.layout_groups(1, seed=4)[0][1]]
    assert sorted(a) == list(range(26)) and a != b
    assert a == [fid for fid, _, _ in oracle.layout_groups(1, seed=3)[0][1]]


@pytest.mark.parametrize("layout", range(11))
def test_store_encoding_reads_back_through_numpy(layout):
    f = ics.perturb(ics.uniform_lattice(n_side=5, jitter=0.3), seed=1, v_amp=1.0)
    rng = np.random.Generator(np.random.PCG64(2))
    for k, arr in f.items():
        if arr.dtype == np.float32 and k not in ("v", "mass", "h"):
            arr[...] = rng.uniform(-1, 1, arr.shape).astype(np.float32)
    f["time_bin"][:] = rng.integers(-5, 5, f["time_bin"].shape)
    n = f["x"].shape[0]
    perm = rng.permutation(n).astype(np.int64)
    img = oracle.store_encode(layout, f, perm, seed=9)
    base = 0
    for rec, mem in oracle.layout_groups(layout, seed=9):
        block = img[base:base + n * rec].reshape(n, rec)
        for fid, comp, off in mem:
            name = oracle.FIELD_NAMES[fid]
            if name == "ballast":
                assert not block[:, off:off + 8].any()
                continue
            arr = f[name][perm]
            if comp >= 0:
                arr = arr[:, comp]
            nb = arr.dtype.itemsize * (arr.shape[1] if arr.ndim > 1 else 1)
            got = np.ascontiguousarray(block[:, off:off + nb]).view(arr.dtype)
            np.testing.assert_array_equal(got.reshape(arr.shape), arr)
        base += (n * rec + 255) // 256 * 256
    assert base == len(img)


# ------------------------------------------------- h-derivative scales ---
def test_dh_scales_bound_the_h_derivative_sums():
    """The conditioning scales (sums of the terms' magnitudes, the exactly
    cancelling self term of wcount_dh by its two parts) bound the sums; the
    rho_dh terms cancel for most particles of a random set; the wcount_dh
    terms never change sign (d/dH (H^3 W) = -(sigma/H) q w'(q) >= 0), so
    past its self term the scale is the sum itself; and a lone particle's
    scales are its self terms in closed form, 3 m sigma / H^4 and
    (4 pi / 3) 6 sigma / H, while its wcount_dh is 0."""
    f = _random_box(400, seed=71)
    P = oracle.params()
    out = oracle.chain(f, P)
    s_rho, s_w = oracle.dh_scales(f, P)
    H = oracle.KERNEL_GAMMA * f["h"].astype(np.float64)
    sigma = 8.0 / math.pi
    self_w = 4 * math.pi / 3 * 6 * sigma / H
    assert np.all(np.abs(out["rho_dh"]) <= s_rho * (1 + 1e-12))
    assert np.median(s_rho / np.abs(out["rho_dh"])) > 1.1
    np.testing.assert_allclose(s_w - self_w, np.abs(out["wcount_dh"]), rtol=1e-9,
                               atol=1e-12 * self_w.max())
    g = ics.empty_fields(2)
    g["x"][:] = [[0.2, 0.5, 0.5], [0.7, 0.5, 0.5]]     # 0.5 apart: no neighbour
    g["mass"][:] = 0.25
    g["h"][:] = 0.0625
    g["u"][:] = 1.0
    lone = oracle.chain(g, P)
    s2, w2 = oracle.dh_scales(g, P)
    H1 = oracle.KERNEL_GAMMA * 0.0625
    np.testing.assert_allclose(s2, 3 * 0.25 * sigma / H1 ** 4, rtol=1e-14)
    np.testing.assert_allclose(w2, 4 * math.pi / 3 * 6 * sigma / H1, rtol=1e-14)
    assert np.all(np.abs(lone["wcount_dh"]) <= 1e-12 * w2)
