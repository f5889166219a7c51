"""Pins of the adjoint oracle (CPU): its forward chain equals the C oracle's,
and its autograd gradient equals central finite differences of the C
oracle's loss (FP64), away from the kinks of min(0, w), |div v| and
sqrt(|P_i - P_j|)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import adjoint
from paper_2606_23891_b300 import ics


def system(n_side=8, seed=3, alpha_diff=0.3, inactive=False):
    f = ics.perturb(ics.uniform_lattice(n_side=n_side, jitter=0.4, seed=seed), seed=seed + 1,
                    v_amp=0.4, u_amp=0.3, alpha_diff=alpha_diff, h_amp=0.1)
    rng = np.random.Generator(np.random.PCG64(seed + 2))
    f["alpha_visc"][:] = rng.uniform(0.2, 1.2, f["alpha_visc"].shape).astype(np.float32)
    f["mass"][:] *= rng.uniform(0.8, 1.2, f["mass"].shape).astype(np.float32)
    if inactive:
        f["time_bin"][::7] = 3
    return f


@pytest.mark.parametrize("inactive", [False, True])
def test_forward_equals_the_c_oracle(inactive):
    f = system(inactive=inactive)
    ref = oracle.chain(f, oracle.params())
    H = oracle.KERNEL_GAMMA * np.asarray(f["h"], np.float64)
    x = torch.tensor(np.asarray(f["x"], np.float64))
    m = torch.tensor(np.asarray(f["mass"], np.float64))
    u = torch.tensor(np.asarray(f["u"], np.float64))
    got = adjoint.chain(x, m, u, f, adjoint.pair_list(f["x"], H))
    act = np.asarray(f["time_bin"]) <= 0
    for k in ("rho", "rho_dh", "div_v", "rot_v", "f_gradh", "pressure", "soundspeed", "balsara"):
        np.testing.assert_allclose(got[k].numpy(), ref[k], rtol=1e-10, atol=1e-10 * np.abs(ref[k]).max(),
                                   err_msg=k)
    for k in ("a", "u_dt"):
        np.testing.assert_allclose(got[k].numpy()[act], ref[k][act], rtol=1e-10,
                                   atol=1e-10 * np.abs(ref[k]).max(), err_msg=k)
    assert abs(float(got["loss"]) - adjoint.loss_c(f)) <= 1e-10 * adjoint.loss_c(f)


def central(f, name, p, comp, eps):
    """Central difference of the C oracle's loss in f[name][p, comp]; None
    when the one-sided slopes disagree (a kink inside the step)."""
    def at(delta):
        g = {k: v.copy() for k, v in f.items()}
        if g[name].ndim == 2:
            g[name][p, comp] += delta
        else:
            g[name][p] += delta
        return adjoint.loss_c(g)
    l0, lp, lm = at(0.0), at(eps), at(-eps)
    dp, dm = (lp - l0) / eps, (l0 - lm) / eps
    if abs(dp - dm) > 1e-3 * max(abs(dp), abs(dm)) + 1e-300:
        return None
    return 0.5 * (dp + dm)


@pytest.mark.parametrize("alpha_diff", [0.0, 0.3])
def test_gradient_equals_central_differences(alpha_diff):
    f = system(alpha_diff=alpha_diff)
    # the C oracle reads positions as FP64 and masses, energies as FP32:
    # perturb positions directly and differentiate m, u on FP64 copies
    loss, gx, gm, gu = adjoint.gradient(f)
    assert abs(loss - adjoint.loss_c(f)) <= 1e-10 * loss
    rng = np.random.Generator(np.random.PCG64(9))
    H = oracle.KERNEL_GAMMA * float(np.median(f["h"]))
    checked = 0
    for p in rng.choice(f["x"].shape[0], 6, replace=False):
        scale = np.abs(gx[p]).max()
        for c in range(3):
            fd = central(f, "x", p, c, 1e-6 * H)
            if fd is None:
                continue
            assert abs(fd - gx[p, c]) <= 1e-5 * scale, (p, c, fd, gx[p, c])
            checked += 1
    assert checked >= 12
    # masses and energies: the C oracle takes FP32 inputs, so compare the
    # autograd gradient with differences of the torch chain itself, which
    # equals the C chain (previous test), in FP64
    H_all = oracle.KERNEL_GAMMA * np.asarray(f["h"], np.float64)
    pairs = adjoint.pair_list(f["x"], H_all)
    x = torch.tensor(np.asarray(f["x"], np.float64))
    m0 = torch.tensor(np.asarray(f["mass"], np.float64))
    u0 = torch.tensor(np.asarray(f["u"], np.float64))

    def L(m, u):
        return float(adjoint.chain(x, m, u, f, pairs)["loss"])
    for p in rng.choice(f["x"].shape[0], 6, replace=False):
        for name, g, base in (("m", gm, m0), ("u", gu, u0)):
            eps = 1e-6 * float(base[p])
            hi, lo = base.clone(), base.clone()
            hi[p] += eps
            lo[p] -= eps
            fd = (L(hi, u0) - L(lo, u0)) / (2 * eps) if name == "m" else \
                (L(m0, hi) - L(m0, lo)) / (2 * eps)
            assert abs(fd - g[p]) <= 1e-5 * max(abs(g[p]), 1e-30) + 1e-8 * np.abs(g).max(), \
                (name, p, fd, g[p])


def lone_and_wide(seed=6):
    """Two particles: A with no other particle inside its own support, and B
    whose wider support reaches A."""
    f = system(n_side=6, seed=seed)
    g = {k: v[:2].copy() for k, v in f.items()}
    g["x"][0] = [0.5, 0.5, 0.5]
    g["x"][1] = [0.52, 0.5, 0.5]
    g["h"][0] = 0.004           # H_A = 0.0073 < 0.02
    g["h"][1] = 0.02            # H_B = 0.0365 > 0.02
    g["time_bin"][:] = 0
    return g


def test_a_particle_without_neighbours_takes_f_gradh_one():
    """Omega = 1 + H/(3 rho) drho/dH is exactly 0 for a particle whose
    support holds no other particle (rho and drho/dH are its self terms), so
    f_gradh = 1/Omega is undefined; the reading is f_gradh = 1.  Its force
    comes only from the wider support of B, equal and opposite in m a."""
    f = lone_and_wide()
    ref = oracle.chain(f, oracle.params())
    H0 = oracle.KERNEL_GAMMA * float(f["h"][0])
    m0 = float(f["mass"][0])
    assert ref["f_gradh"][0] == 1.0
    assert ref["rho"][0] == pytest.approx(m0 * 8.0 / np.pi / H0 ** 3, rel=1e-12)
    assert ref["div_v"][0] == 0.0
    assert np.isfinite(ref["f_gradh"]).all() and ref["f_gradh"][1] != 1.0
    pa = float(f["mass"][0]) * ref["a"][0]
    pb = float(f["mass"][1]) * ref["a"][1]
    assert np.abs(pa).max() > 0.0
    np.testing.assert_allclose(pa, -pb, rtol=1e-10)
    # the autograd restatement agrees, value and gradient finite
    x = torch.tensor(np.asarray(f["x"], np.float64), requires_grad=True)
    m = torch.tensor(np.asarray(f["mass"], np.float64))
    u = torch.tensor(np.asarray(f["u"], np.float64))
    H = oracle.KERNEL_GAMMA * np.asarray(f["h"], np.float64)
    got = adjoint.chain(x, m, u, f, adjoint.pair_list(f["x"], H))
    for k in ("rho", "f_gradh", "a", "u_dt"):
        np.testing.assert_allclose(got[k].detach().numpy(), ref[k], rtol=1e-10,
                                   atol=1e-12 * np.abs(ref[k]).max(), err_msg=k)
    got["loss"].backward()
    assert torch.isfinite(x.grad).all()
