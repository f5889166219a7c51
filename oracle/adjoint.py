"""Reference gradient of the density -> ghost -> force chain (test infrastructure).

The loss of the differentiation workload is

    L = sum_i |a_i|^2 + sum_i (du_i/dt)^2        (active particles)

and its gradient is wanted with respect to positions, masses and internal
energies; smoothing lengths, velocities and the viscosity / conduction
switches are held fixed.  This module restates the density sums, the ghost
update and the force sums of ``sph_oracle.c`` (Sec. 2.1; the forms are the
oracle's: cubic spline M4, grad-h terms, Monaghan viscosity with a Balsara
switch, Price conduction) as FP64 torch operations over a brute-force
minimum-image pair list, so that autograd gives the exact gradient of the
chain.  The pair list itself is not differentiated: it is recomputed for
every evaluation, as the GPU path recomputes its neighbour lists.

Parity pins (tests): the forward values equal ``oracle.chain``; the gradient
equals central finite differences of the C oracle's loss.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import BALSARA_EPS, BETA_VISC, GAMMA, KERNEL_GAMMA

NORM = 8.0 / math.pi


def pair_list(x: np.ndarray, H: np.ndarray, box=(1.0, 1.0, 1.0)):
    """Ordered pairs (i, j), i != j, with minimum-image r < max(H_i, H_j),
    by brute force in blocks of rows."""
    x = np.asarray(x, np.float64)
    H = np.asarray(H, np.float64)
    b = np.asarray(box, np.float64)
    n = x.shape[0]
    I, J = [], []
    for s in range(0, n, 256):
        d = x[s:s + 256, None, :] - x[None, :, :]
        d -= b * np.rint(d / b)
        r2 = (d * d).sum(axis=2)
        hm = np.maximum(H[s:s + 256, None], H[None, :])
        ii, jj = np.nonzero(r2 < hm * hm)
        keep = ii + s != jj
        I.append(ii[keep] + s)
        J.append(jj[keep])
    return np.concatenate(I), np.concatenate(J)


def _w(q):
    return torch.where(q < 0.5, 1 - 6 * q * q + 6 * q ** 3,
                       torch.where(q < 1.0, 2 * (1 - q) ** 3, torch.zeros_like(q)))


def _dw(q):
    return torch.where(q < 0.5, -12 * q + 18 * q * q,
                       torch.where(q < 1.0, -6 * (1 - q) ** 2, torch.zeros_like(q)))


def chain(x, m, u, f: dict, pairs, box=(1.0, 1.0, 1.0), active_bin: int = 0,
          gamma=GAMMA, kernel_gamma=KERNEL_GAMMA, beta=BETA_VISC, eps=BALSARA_EPS):
    """Forward chain with torch tensors x (n, 3), m (n,), u (n,) (FP64, may
    require grad); the other inputs come from the field dict ``f``.  Returns
    the ghost and force outputs and the loss."""
    I = torch.as_tensor(pairs[0])
    J = torch.as_tensor(pairs[1])
    n = x.shape[0]
    dt = torch.float64
    h = torch.as_tensor(np.asarray(f["h"], np.float64))
    v = torch.as_tensor(np.asarray(f["v"], np.float64))
    av = torch.as_tensor(np.asarray(f["alpha_visc"], np.float64))
    ad = torch.as_tensor(np.asarray(f["alpha_diff"], np.float64))
    active = torch.as_tensor(np.asarray(f["time_bin"], np.int64) <= active_bin)
    H = kernel_gamma * h
    bx = torch.as_tensor(np.asarray(box, np.float64))
    d = x[I] - x[J]
    d = d - bx * torch.round((d / bx).detach())
    r = torch.sqrt((d * d).sum(dim=1))
    rhat = d / r[:, None]
    dv = v[I] - v[J]
    wdot = (dv * rhat).sum(dim=1)
    # density sums over r < H_i (the raw sums of the density loop)
    Hi, Hj = H[I], H[J]
    dens = (r < Hi).to(dt)
    qi = r / Hi
    Wi = NORM / Hi ** 3 * _w(qi)
    Fi = NORM / Hi ** 4 * _dw(qi)
    dWdH = -NORM / Hi ** 4 * (3 * _w(qi) + qi * _dw(qi))
    mj = m[J]
    Srho = torch.zeros(n, dtype=dt).index_add(0, I, dens * mj * Wi)
    Sdh = torch.zeros(n, dtype=dt).index_add(0, I, dens * mj * dWdH)
    Sdiv = torch.zeros(n, dtype=dt).index_add(0, I, -dens * mj * wdot * Fi)
    cross = torch.stack([dv[:, 1] * rhat[:, 2] - dv[:, 2] * rhat[:, 1],
                         dv[:, 2] * rhat[:, 0] - dv[:, 0] * rhat[:, 2],
                         dv[:, 0] * rhat[:, 1] - dv[:, 1] * rhat[:, 0]], dim=1)
    Srot = torch.zeros(n, 3, dtype=dt).index_add(0, I, (dens * mj * Fi)[:, None] * cross)
    # ghost
    rho = Srho + m * NORM / H ** 3
    rho_dh = Sdh - 3 * m * NORM / H ** 4
    div = Sdiv / rho
    rot = Srot / rho[:, None]
    omega = 1 + H / (3 * rho) * rho_dh
    # no neighbour inside the support: Omega is exactly 0 and f_gradh = 1
    lone = torch.zeros(n, dtype=dt).index_add(0, I, dens) == 0
    fgh = torch.where(lone, torch.ones_like(omega), 1 / torch.where(lone, torch.ones_like(omega),
                                                                   omega))
    P = (gamma - 1) * rho * u
    c = torch.sqrt(gamma * (gamma - 1) * u)
    R2 = (rot * rot).sum(dim=1)
    R = torch.where(R2 > 0, torch.sqrt(torch.where(R2 > 0, R2, torch.ones_like(R2))),
                    torch.zeros_like(R2))
    D = torch.abs(div)
    B = D / (D + R + eps * c / h)
    # force over r < max(H_i, H_j), active i
    Fj = NORM / Hj ** 4 * _dw(r / Hj)
    mu = torch.clamp(wdot, max=0.0)
    Fbar = 0.5 * (Fi + Fj)
    rhobar = 0.5 * (rho[I] + rho[J])
    alpha = 0.5 * (av[I] * B[I] + av[J] * B[J])
    vs = c[I] + c[J] - beta * mu
    Pi = -alpha * vs * mu / rhobar
    A = fgh * P / rho ** 2
    s = A[I] * Fi + A[J] * Fj + Pi * Fbar
    act = active[I].to(dt)
    a = torch.zeros(n, 3, dtype=dt).index_add(0, I, -(act * mj * s)[:, None] * rhat)
    dP = P[I] - P[J]
    sq = torch.where(dP != 0, torch.sqrt(torch.abs(torch.where(dP != 0, dP, torch.ones_like(dP)))
                                         / rhobar), torch.zeros_like(dP))
    cond = 0.5 * (ad[I] + ad[J]) * sq * (u[I] - u[J]) * Fbar / rhobar
    udt = torch.zeros(n, dtype=dt).index_add(
        0, I, act * mj * (A[I] * Fi * wdot + 0.5 * Pi * Fbar * wdot + cond))
    loss = ((a * a).sum(dim=1) + udt * udt)[active].sum()
    return {"rho": rho, "rho_dh": rho_dh, "div_v": div, "rot_v": rot, "f_gradh": fgh,
            "pressure": P, "soundspeed": c, "balsara": B, "a": a, "u_dt": udt, "loss": loss}


def gradient(f: dict, box=(1.0, 1.0, 1.0), active_bin: int = 0):
    """(loss, dL/dx (n, 3), dL/dm (n,), dL/du (n,)) in FP64 by autograd."""
    x = torch.tensor(np.asarray(f["x"], np.float64), requires_grad=True)
    m = torch.tensor(np.asarray(f["mass"], np.float64), requires_grad=True)
    u = torch.tensor(np.asarray(f["u"], np.float64), requires_grad=True)
    H = KERNEL_GAMMA * np.asarray(f["h"], np.float64)
    out = chain(x, m, u, f, pair_list(f["x"], H, box), box, active_bin)
    out["loss"].backward()
    return (out["loss"].item(), x.grad.numpy(), m.grad.numpy(), u.grad.numpy())


def loss_c(f: dict, box=(1.0, 1.0, 1.0), active_bin: int = 0) -> float:
    """The same loss from the C oracle's chain (FP64)."""
    from . import chain as c_chain, params
    out = c_chain(f, params(box=box, active_bin=active_bin))
    act = np.asarray(f["time_bin"], np.int64) <= active_bin
    return float(((out["a"] ** 2).sum(axis=1) + out["u_dt"] ** 2)[act].sum())
