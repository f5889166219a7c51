"""Pins of the force loop's magnitudes (Sec. 2.1, Table 1 p-f / u-f).

Momentum and energy conservation do not fix the force loop's scale: a
pressure term scaled consistently in a and du/dt, or a viscosity whose sign
turns heating into cooling, still conserves both.  These tests fix the
magnitudes against facts the force loop does not compute itself:

- grad-h SPH derives the pressure force from the thermal energy
  E = sum_j m_j u_j.  Under adiabatic change du_j = (P_j / rho_j^2) d rho_j,
  and with h_j tied to rho_j (h^3 rho fixed) a change of the density sum at
  fixed h becomes d rho_j = f_j d rho_j|_h.  So
      m_i a_i = -dE/dx_i = -sum_j m_j f_j P_j / rho_j^2  d rho_j / d x_i |_h,
  and likewise du_i/dt = f_i P_i / rho_i^2  D rho_i / Dt |_h and
  dh_i/dt = -(h_i / (3 rho_i)) f_i  D rho_i / Dt |_h along the flow.  The
  right-hand sides use only the density sum (pinned to the lattice sum and
  finite differences in H), f (pinned by the ghost tests) and FP64 central
  differences of the positions;
- on a static lattice with u = u0 (1 + A sin kx), the acceleration tends to
  -grad P / rho = -(gamma - 1) u0 A k cos kx, whatever the density;
- the artificial viscosity only heats (du/dt >= 0), heats wherever the flow
  converges, is exactly zero where every pair recedes, and removes kinetic
  energy at the rate it adds heat;
- for two particles approaching head-on its effect has a closed form,
  derived in the docstring of that test.

Each pin is then shown to fail on a copy of the oracle with a plausible
mistake planted in it (compiled on the CPU by oracle.variant).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2606_23891_b300 import ics

GAMMA = oracle.GAMMA
TOL = 1e-7          # FD pins: the central differences carry about 1e-10


def _copy(f):
    return {k: v.copy() for k, v in f.items()}


def _static_set():
    """Jittered lattice, v = 0 (no viscosity), no conduction, masses and so
    densities around 2.7 (so P / rho and P / rho^2 differ), u and h scattered
    (so f departs from 1 by up to about 40%)."""
    f = ics.perturb(ics.uniform_lattice(n_side=8, jitter=0.3, seed=61), seed=62,
                    u_amp=0.4, h_amp=0.1)
    rng = np.random.Generator(np.random.PCG64(63))
    f["mass"] *= (2.7 * rng.uniform(0.7, 1.3, f["mass"].shape)).astype(np.float32)
    f["alpha_visc"][:] = 0.0
    f["alpha_diff"][:] = 0.0
    return f


def energy_gradient_error():
    """max |a_i - (-dE/dx_i / m_i)| / rms(a) over a few particles and axes."""
    f = _static_set()
    P = oracle.params()
    full = oracle.chain(f, P)
    m = f["mass"].astype(np.float64)
    coef = m * full["f_gradh"] * full["pressure"] / full["rho"] ** 2
    scale = np.sqrt(np.mean(full["a"] ** 2))
    eps = 1e-6
    worst = 0.0
    for i in (0, 77, 300, 511):
        for c in range(3):
            g = _copy(f)
            g["x"][i, c] += eps
            rp = oracle.density(g, P)[0][:, 0]
            g["x"][i, c] -= 2 * eps
            rm = oracle.density(g, P)[0][:, 0]
            ref = -(coef * (rp - rm) / (2 * eps)).sum() / m[i]
            worst = max(worst, abs(full["a"][i, c] - ref) / scale)
    return worst


def adiabatic_rate_errors():
    """(du/dt, dh/dt) errors against the density's rate along the flow, each
    max error over the field's rms."""
    f = ics.perturb(_static_set(), seed=64, v_amp=0.5)
    P = oracle.params()
    full = oracle.chain(f, P)
    v = f["v"].astype(np.float64)
    eps = 1e-6
    g = _copy(f)
    g["x"] = f["x"] + eps * v
    rp = oracle.density(g, P)[0][:, 0]
    g["x"] = f["x"] - eps * v
    rm = oracle.density(g, P)[0][:, 0]
    rate = (rp - rm) / (2 * eps)           # D rho / Dt at fixed h
    du = full["f_gradh"] * full["pressure"] / full["rho"] ** 2 * rate
    dh = -(f["h"].astype(np.float64) / (3 * full["rho"])) * full["f_gradh"] * rate

    def err(a, b):
        return float(np.max(np.abs(a - b)) / np.sqrt(np.mean(b * b)))
    return err(full["u_dt"], du), err(full["h_dt"], dh)


def continuum_pressure_error():
    """Static perfect lattice of density 2.7 with u = u0 (1 + A sin kx):
    (max |a_x - (-(gamma-1) u0 A k cos kx)|, max |a_y|, |a_z|) over the
    amplitude (gamma - 1) u0 A k, on a row of particles along x."""
    ns = 32
    f = ics.uniform_lattice(n_side=ns, jitter=0.0)
    f["mass"][:] = np.float32(2.7 / f["x"].shape[0])
    A, k, u0 = 0.05, 2 * math.pi, 1.3
    f["u"][:] = (u0 * (1 + A * np.sin(k * f["x"][:, 0]))).astype(np.float32)
    f["alpha_visc"][:] = 0.0
    f["alpha_diff"][:] = 0.0
    sel = np.arange(ns)                     # index order: x fastest
    out = oracle.chain(f, oracle.params(), sel)
    amp = (GAMMA - 1) * u0 * A * k
    ref = -amp * np.cos(k * f["x"][sel, 0])
    return (float(np.max(np.abs(out["a"][:, 0] - ref)) / amp),
            float(np.max(np.abs(out["a"][:, 1:])) / amp))


def converging_flow():
    """Perfect 16^3 lattice with v_x = -A sin(kx), u uniform, no conduction:
    the viscous parts (alpha_visc = 1 minus alpha_visc = 0) of du/dt and a on
    a row of particles along x, with the row's phases kx and kH."""
    ns = 16
    f = ics.uniform_lattice(n_side=ns, jitter=0.0)
    A, k = 0.3, 2 * math.pi
    f["v"][:, 0] = (-A * np.sin(k * f["x"][:, 0])).astype(np.float32)
    f["alpha_diff"][:] = 0.0
    sel = np.arange(ns)
    on, off = _copy(f), _copy(f)
    on["alpha_visc"][:] = 1.0
    off["alpha_visc"][:] = 0.0
    P = oracle.params()
    o1, o0 = oracle.chain(on, P, sel), oracle.chain(off, P, sel)
    phase = np.mod(k * f["x"][sel, 0], 2 * math.pi)
    kH = k * oracle.KERNEL_GAMMA * float(f["h"][0])
    m = f["mass"][sel].astype(np.float64)
    v = f["v"][sel].astype(np.float64)
    return (o1["u_dt"] - o0["u_dt"], o1["a"] - o0["a"], phase, kH, m, v)


def two_particle_case():
    """Two equal particles on the x axis, separation d = 0.3 H, approaching
    head-on at speeds +-V; every input is exact in FP32.  Returns the
    viscous parts of (du_1/dt, a_1x) and their closed forms.

    Derivation from the force loop's definition (Sec. 2.1 forms):
    particle 1 sits at x - d/2 moving +V, particle 2 at x + d/2 moving -V.
    With rhat = (x_1 - x_2) / r = -xhat and v_12 = 2V xhat,
    w = v_12 . rhat = -2V, so mu = min(0, w) = -2V.  Each density is
    rho = m W(0, H) + m W(d, H).  F = dW/dr(d, H) < 0 for both; the
    divergence is div v_1 = -(1/rho) m w F = 2 m V F / rho and the curl is
    0, so the Balsara switch is B = |div| / (|div| + eps c / h).  Then
    alpha_12 = alpha B, v_sig = 2c - beta mu = 2c + 6V and
    Pi = -alpha_12 v_sig mu / rhobar = 2 alpha B V (2c + 6V) / rho.
    Viscous heating: du_1/dt = m (1/2) Pi Fbar w = -m Pi F V  (> 0, F < 0).
    Viscous acceleration: a_1 = -m Pi Fbar rhat = m Pi F xhat, so
    a_1x = m Pi F < 0 brakes particle 1.
    """
    h, m, V, u, alpha = 0.0625, 0.0078125, 0.75, 1.25, 0.75
    H = oracle.KERNEL_GAMMA * h
    d = 0.3 * H
    f = ics.empty_fields(2)
    f["x"][:] = [[0.5 - d / 2, 0.5, 0.5], [0.5 + d / 2, 0.5, 0.5]]
    f["v"][:] = [[V, 0.0, 0.0], [-V, 0.0, 0.0]]
    f["mass"][:] = m
    f["h"][:] = h
    f["u"][:] = u
    f["alpha_visc"][:] = alpha
    off = _copy(f)
    off["alpha_visc"][:] = 0.0
    P = oracle.params()
    o1, o0 = oracle.chain(f, P), oracle.chain(off, P)
    r = float(f["x"][1, 0] - f["x"][0, 0])
    rho = m * oracle.W(0.0, H) + m * oracle.W(r, H)
    F = oracle.dWdr(r, H)
    c = math.sqrt(GAMMA * (GAMMA - 1) * u)
    div = 2 * m * V * F / rho
    B = abs(div) / (abs(div) + oracle.BALSARA_EPS * c / h)
    Pi = 2 * alpha * B * V * (2 * c + 6 * V) / rho
    got = (float(o1["u_dt"][0] - o0["u_dt"][0]), float(o1["a"][0, 0] - o0["a"][0, 0]))
    return got, (-m * Pi * F * V, m * Pi * F)


def viscosity_errors():
    """(sign violations, dissipation balance error, closed-form error):
    every quantity that should be 0 for a correct viscosity."""
    du, da, phase, kH, m, v = converging_flow()
    scale = float(np.max(np.abs(du)))
    neg = float(max(0.0, -du.min()) / scale)
    conv = np.cos(phase) > 0.5
    # where every pair within H recedes (v_x increasing over the whole span)
    recede = np.abs(phase - math.pi) + kH < 0.5 * math.pi
    heats = float(min(1.0, du[conv].min() / (1e-3 * scale)))
    zero = float(np.max(np.abs(du[recede])) / scale)
    kin = float((m * (v * da).sum(1)).sum())
    th = float((m * du).sum())
    balance = abs(kin + th) / (abs(kin) + abs(th))
    got, ref = two_particle_case()
    closed = max(abs(g - r) / abs(r) for g, r in zip(got, ref))
    return {"negative_heating": neg, "converging_not_heated": 1.0 - heats,
            "receding_heated": zero, "kinetic_not_dissipated": float(kin >= 0.0),
            "energy_balance": balance, "closed_form": closed}


# ------------------------------------------------------------ the pins ---
def test_pressure_force_is_minus_the_gradient_of_thermal_energy():
    assert energy_gradient_error() < TOL


def test_adiabatic_du_dt_and_dh_dt_follow_the_density_rate():
    eu, eh = adiabatic_rate_errors()
    assert eu < TOL and eh < TOL


def test_pressure_force_tends_to_the_continuum_gradient():
    ex, eyz = continuum_pressure_error()
    # kernel smoothing at kH = 0.44 and f = 1.011 on this lattice: < 1%
    assert ex < 0.02
    assert eyz < 1e-10


def test_viscosity_heats_converging_flow_only():
    du, da, phase, kH, m, v = converging_flow()
    e = viscosity_errors()
    assert e["negative_heating"] < 1e-12
    assert e["converging_not_heated"] == 0.0
    assert e["receding_heated"] == 0.0
    assert np.count_nonzero(np.abs(phase - math.pi) + kH < 0.5 * math.pi) >= 2
    assert e["kinetic_not_dissipated"] == 0.0
    assert e["energy_balance"] < 1e-12


def test_two_particle_viscosity_closed_form():
    (du, ax), (du_ref, ax_ref) = two_particle_case()
    assert du > 0.0 and ax < 0.0
    assert abs(du - du_ref) <= 1e-12 * abs(du_ref)
    assert abs(ax - ax_ref) <= 1e-12 * abs(ax_ref)


# ------------------------------------------- planted mistakes are caught ---
A_I = "double Ai = fgh[i] * pres[i] / (rho[i] * rho[i]);"
A_J = "double Aj = fgh[j] * pres[j] / (rho[j] * rho[j]);"
PLANTED = {
    "P/rho in place of P/rho^2": [(A_I, "double Ai = fgh[i] * pres[i] / rho[i];"),
                                  (A_J, "double Aj = fgh[j] * pres[j] / rho[j];")],
    "f_i dropped": [(A_I, "double Ai = pres[i] / (rho[i] * rho[i]);")],
    "f_j dropped": [(A_J, "double Aj = pres[j] / (rho[j] * rho[j]);")],
    "pressure force doubled in a and du/dt": [
        (A_I, "double Ai = 2.0 * fgh[i] * pres[i] / (rho[i] * rho[i]);"),
        (A_J, "double Aj = 2.0 * fgh[j] * pres[j] / (rho[j] * rho[j]);")],
    "viscosity sign flipped": [("double Pi = -alpha * vs * mu / rhobar;",
                                "double Pi = alpha * vs * mu / rhobar;")],
    "viscous heating without the 1/2": [("0.5 * Pi * Fbar * w", "Pi * Fbar * w")],
    "viscosity without 1/rhobar": [("double Pi = -alpha * vs * mu / rhobar;",
                                    "double Pi = -alpha * vs * mu;")],
    "signal velocity with +beta mu": [("double vs = cs[i] + cs[j] - P->beta_visc * mu;",
                                       "double vs = cs[i] + cs[j] + P->beta_visc * mu;")],
}


def _caught():
    errs = {"energy_gradient": energy_gradient_error()}
    eu, eh = adiabatic_rate_errors()
    errs.update(adiabatic_du=eu, adiabatic_dh=eh)
    ex, eyz = continuum_pressure_error()
    errs.update(continuum=ex / 0.02, continuum_yz=eyz / 1e-10)
    v = viscosity_errors()
    errs.update(v)
    bars = {"energy_gradient": TOL, "adiabatic_du": TOL, "adiabatic_dh": TOL,
            "continuum": 1.0, "continuum_yz": 1.0, "negative_heating": 1e-12,
            "converging_not_heated": 0.0, "receding_heated": 0.0,
            "kinetic_not_dissipated": 0.0, "energy_balance": 1e-12, "closed_form": 1e-12}
    return sorted(k for k, b in bars.items() if errs[k] > b)


def test_pins_pass_on_the_oracle():
    assert _caught() == []


@pytest.mark.parametrize("mistake", sorted(PLANTED))
def test_pins_catch_a_planted_mistake(mistake):
    with oracle.variant(PLANTED[mistake]):
        failed = _caught()
    assert failed, mistake
