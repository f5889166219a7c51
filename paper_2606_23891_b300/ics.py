"""Seeded synthetic initial conditions for the SPH offload pipeline.

This module only draws inputs: particle positions, velocities, masses,
internal energies, smoothing lengths and the per-particle switches.  It holds
none of the method's arithmetic (no kernel, no neighbour search, no cell
assignment), so that the CUDA path and the independent CPU oracle can both be
fed from it without sharing any computation.

Workloads (stand-ins for the paper's traces, Sec. 3.4, which are not
available):

* ``uniform_lattice``: the tiny plain case, a 16^3 cubic lattice in the unit
  periodic box with uniform +-0.1 spacing jitter, rho = 1, u = 1, v = 0.
* ``gresho``: a Gresho-Chan vortex shaped set (the "Gresho256" experiment of
  Sec. 3.4) on a jittered 256^3 lattice.  A jitter of +-0.52 spacing on cells
  of four lattice spacings reproduces the paper's 55/73/64/64 min/max/mean/
  median particles per cell.
* ``lognormal``: a cosmology-clustering shaped set (the "Eagle25" trace of
  Sec. 3.4 stands behind it): particles drawn from a lognormal density field
  with sigma(ln rho) = 2, so that densities span about nine decades and
  smoothing lengths about three.

Smoothing lengths follow the usual SPH relation h = eta (m / rho)^(1/3) with
rho the *prescribed* density of the recipe (not a measured one).
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = 5.0 / 3.0
ETA = 1.2348

# Field names of the logical particle record, in the order the C-ABI's
# sph_fields struct lists them.  Vector fields have three components.
INPUT_FIELDS = ("x", "v", "mass", "h", "u", "alpha_visc", "alpha_diff",
                "time_bin", "id")
FIELD_DTYPES = {
    "x": (np.float64, 3), "v": (np.float32, 3), "a": (np.float32, 3),
    "mass": (np.float32, 1), "h": (np.float32, 1), "u": (np.float32, 1),
    "u_dt": (np.float32, 1), "rho": (np.float32, 1),
    "time_bin": (np.int8, 1), "alpha_visc": (np.float32, 1),
    "alpha_diff": (np.float32, 1), "rho_dh": (np.float32, 1),
    "wcount": (np.float32, 1), "wcount_dh": (np.float32, 1),
    "div_v": (np.float32, 1), "rot_v": (np.float32, 3),
    "f_gradh": (np.float32, 1), "pressure": (np.float32, 1),
    "soundspeed": (np.float32, 1), "balsara": (np.float32, 1),
    "v_sig_grad": (np.float32, 1), "laplace_u": (np.float32, 1),
    "h_dt": (np.float32, 1), "v_sig": (np.float32, 1), "id": (np.int64, 1),
}


def empty_fields(n: int) -> dict:
    """Zero-filled arrays for every logical field of ``n`` particles."""
    out = {}
    for name, (dt, k) in FIELD_DTYPES.items():
        out[name] = np.zeros((n, k) if k > 1 else (n,), dtype=dt)
    return out


def jittered_lattice(n_side: int, jitter: float, seed: int,
                     box: float = 1.0) -> np.ndarray:
    """Cubic lattice at (i + 1/2) spacing plus U(-jitter, +jitter) spacing
    per coordinate, wrapped into [0, box).  Index order: x fastest."""
    rng = np.random.Generator(np.random.PCG64(seed))
    dx = box / n_side
    i = np.arange(n_side, dtype=np.float64)
    gz, gy, gx = np.meshgrid(i, i, i, indexing="ij")
    x = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1)
    x = (x + 0.5) * dx
    if jitter > 0.0:
        x += rng.uniform(-jitter, jitter, size=x.shape) * dx
    x = np.mod(x, box)
    x[x >= box] -= box          # np.mod can round up to exactly box
    return x


def _base_fields(x: np.ndarray, rho0: float, box: float, seed: int) -> dict:
    n = x.shape[0]
    f = empty_fields(n)
    f["x"][:] = x
    m = rho0 * box ** 3 / n
    f["mass"][:] = m
    f["h"][:] = ETA * (m / rho0) ** (1.0 / 3.0)
    f["id"][:] = np.arange(n, dtype=np.int64)
    return f


def uniform_lattice(n_side: int = 16, jitter: float = 0.1, seed: int = 1,
                    u0: float = 1.0, alpha_visc: float = 0.1,
                    alpha_diff: float = 0.0, box: float = 1.0) -> dict:
    """The tiny plain case: jittered lattice, rho = 1, u = u0, v = 0."""
    x = jittered_lattice(n_side, jitter, seed, box)
    f = _base_fields(x, 1.0, box, seed)
    f["u"][:] = u0
    f["alpha_visc"][:] = alpha_visc
    f["alpha_diff"][:] = alpha_diff
    return f


def gresho_pressure(r: np.ndarray, p0: float = 5.0) -> np.ndarray:
    """Piecewise pressure that balances the Gresho-Chan vortex rotation."""
    r = np.asarray(r, dtype=np.float64)
    p = np.full_like(r, p0 - 2.0 + 4.0 * math.log(2.0))
    a = r < 0.2
    b = (r >= 0.2) & (r < 0.4)
    p[a] = p0 + 12.5 * r[a] ** 2
    rb = r[b]
    p[b] = p0 + 12.5 * rb ** 2 + 4.0 - 20.0 * rb + 4.0 * np.log(5.0 * rb)
    return p


def gresho_vphi(r: np.ndarray) -> np.ndarray:
    r = np.asarray(r, dtype=np.float64)
    v = np.zeros_like(r)
    a = r < 0.2
    b = (r >= 0.2) & (r < 0.4)
    v[a] = 5.0 * r[a]
    v[b] = 2.0 - 5.0 * r[b]
    return v


def gresho(n_side: int = 256, jitter: float = 0.52, seed: int = 3,
           alpha_visc: float = 0.1, alpha_diff: float = 0.0,
           box: float = 1.0) -> dict:
    """Gresho-Chan vortex about the z axis through (0.5, 0.5) in a periodic
    unit box: rho = 1, v_phi(r) and p(r) piecewise, u = p / ((gamma-1) rho)."""
    x = jittered_lattice(n_side, jitter, seed, box)
    f = _base_fields(x, 1.0, box, seed)
    dxc = x[:, 0] - 0.5 * box
    dyc = x[:, 1] - 0.5 * box
    r = np.sqrt(dxc * dxc + dyc * dyc)
    vphi = gresho_vphi(r)
    with np.errstate(invalid="ignore", divide="ignore"):
        s = np.where(r > 0.0, vphi / r, 0.0)
    f["v"][:, 0] = (-dyc * s).astype(np.float32)
    f["v"][:, 1] = (dxc * s).astype(np.float32)
    f["u"][:] = (gresho_pressure(r) / ((GAMMA - 1.0) * 1.0)).astype(np.float32)
    f["alpha_visc"][:] = alpha_visc
    f["alpha_diff"][:] = alpha_diff
    return f


def _field_k(g: int):
    """Integer wavenumbers of a g^3 real FFT grid (rfftn layout) and |k|."""
    k1 = np.fft.fftfreq(g, 1.0 / g)
    kz = np.fft.rfftfreq(g, 1.0 / g)
    kx, ky, kz = np.meshgrid(k1, k1, kz, indexing="ij")
    return kx, ky, kz, np.sqrt(kx * kx + ky * ky + kz * kz)


def lognormal(n_side: int = 376, sigma_ln: float = 2.0, grid: int = 0,
              slope: float = -2.0, smooth: float = 2.5, seed: int = 11,
              v_amp: float = 0.3, box: float = 1.0, h_iters: int = 4) -> dict:
    """Clustered set of n_side^3 equal-mass particles in the unit periodic box.

    A Gaussian random field with power spectrum k^slope exp(-(2 pi k s / g)^2 / 2)
    (s = ``smooth`` field cells) on a grid^3 mesh (default: the power of two
    nearest n_side / 3, about 27 particles per mesh cell) is scaled to unit variance;
    the density is rho = exp(sigma_ln delta - sigma_ln^2 / 2) normalised to a
    mean of 1.  Particle counts per mesh cell are multinomial in rho, and
    positions uniform inside each cell.  Velocities follow the field's
    gradient flow (the linear-theory displacement direction, scaled to an rms
    of ``v_amp`` per component); u rises with density as rho^(2/3);
    alpha_visc, alpha_diff are drawn uniformly.  Smoothing lengths use
    h = eta (m / rho_bar)^(1/3) with rho_bar the particles' number density
    counted on the mesh and averaged over a sphere of radius ~ the support
    (damped fixed-point iterations on mesh averages at radii 2^j cells), so
    that particles in thin regions see the density around them rather than
    their own cell's and the neighbour counts stay near the target."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = n_side ** 3
    g = grid or 2 ** max(2, int(round(math.log2(n_side / 3.0))))
    kx, ky, kz, kk = _field_k(g)
    with np.errstate(divide="ignore"):
        amp = np.where(kk > 0, kk ** (0.5 * slope), 0.0)
    amp *= np.exp(-0.25 * (2.0 * np.pi * kk * smooth / g) ** 2)
    dk = np.fft.rfftn(rng.standard_normal((g, g, g))) * amp
    delta = np.fft.irfftn(dk, s=(g, g, g), axes=(0, 1, 2))
    delta /= delta.std()
    rho = np.exp(sigma_ln * delta - 0.5 * sigma_ln ** 2)
    rho /= rho.mean()
    counts = rng.multinomial(n, (rho / rho.sum()).ravel())
    cell = np.repeat(np.arange(g ** 3, dtype=np.int64), counts)
    del counts
    iz, rem = np.divmod(cell, g * g)
    iy, ix = np.divmod(rem, g)
    del rem
    x = np.empty((n, 3), np.float64)
    for d, idx in enumerate((ix, iy, iz)):
        x[:, d] = (idx + rng.random(n)) * (box / g)
    del ix, iy, iz
    m = box ** 3 / n
    f = empty_fields(n)
    f["x"][:] = x
    f["mass"][:] = m
    f["id"][:] = np.arange(n, dtype=np.int64)
    # mesh averages of the particles' number density over spheres of radius
    # 2^j cells (top-hat filter), interpolated in log radius at the support
    nd = np.bincount(cell, minlength=g ** 3).reshape(g, g, g) * (g ** 3 / n)
    rk = np.fft.rfftn(nd)
    levels = [nd.ravel()]
    radii = [0.5]                       # a particle's own cell
    for j in range(0, int(math.log2(g // 4)) + 1):
        r = 2.0 ** j
        xk = 2.0 * np.pi * kk * r / g
        with np.errstate(invalid="ignore", divide="ignore"):
            w = np.where(xk > 1e-8, 3.0 * (np.sin(xk) - xk * np.cos(xk)) / xk ** 3, 1.0)
        levels.append(np.maximum(np.fft.irfftn(rk * w, s=(g, g, g), axes=(0, 1, 2)), 1e-6).ravel())
        radii.append(r)
    lr = np.log2(np.array(radii) * (box / g))
    kernel_gamma = 1.825742
    H = kernel_gamma * ETA * (m / np.maximum(levels[0][cell], 1e-6)) ** (1.0 / 3.0)
    for _ in range(h_iters):
        t = np.clip(np.log2(H), lr[0], lr[-1])
        j = np.minimum(np.searchsorted(lr, t, side="right") - 1, len(lr) - 2)
        wgt = (t - lr[j]) / (lr[j + 1] - lr[j])
        lo = np.empty(n)
        hi = np.empty(n)
        for L in range(len(lr) - 1):
            sel = j == L
            lo[sel] = levels[L][cell[sel]]
            hi[sel] = levels[L + 1][cell[sel]]
        rho_bar = np.exp((1.0 - wgt) * np.log(lo) + wgt * np.log(hi))
        H = np.sqrt(H * kernel_gamma * ETA * (m / rho_bar) ** (1.0 / 3.0))   # damped
    f["h"][:] = (H / kernel_gamma).astype(np.float32)
    # velocities: gradient flow of the field, sampled at the particle's cell
    with np.errstate(invalid="ignore", divide="ignore"):
        phi = np.where(kk > 0, dk / (kk * kk), 0.0)
    for d, kd in enumerate((kx, ky, kz)):
        vd = np.fft.irfftn(1j * kd * phi, s=(g, g, g), axes=(0, 1, 2)).ravel()
        vd *= v_amp / max(vd.std(), 1e-30)
        f["v"][:, d] = vd[cell].astype(np.float32)
    f["u"][:] = (rho.ravel()[cell] ** (2.0 / 3.0)).astype(np.float32)
    f["alpha_visc"][:] = rng.uniform(0.1, 1.0, n).astype(np.float32)
    f["alpha_diff"][:] = rng.uniform(0.0, 0.2, n).astype(np.float32)
    return f


def perturb(fields: dict, seed: int, v_amp: float = 0.0, u_amp: float = 0.0,
            alpha_diff: float | None = None, h_amp: float = 0.0) -> dict:
    """Seeded perturbations used by tests to exercise every term: random
    velocities, internal-energy and smoothing-length scatter, conduction."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = fields["x"].shape[0]
    if v_amp:
        fields["v"] += rng.uniform(-v_amp, v_amp, (n, 3)).astype(np.float32)
    if u_amp:
        fields["u"] *= (1.0 + rng.uniform(-u_amp, u_amp, n)).astype(np.float32)
    if h_amp:
        fields["h"] *= (1.0 + rng.uniform(-h_amp, h_amp, n)).astype(np.float32)
    if alpha_diff is not None:
        fields["alpha_diff"][:] = rng.uniform(0.0, alpha_diff, n).astype(np.float32)
    return fields


def random_result_lanes(nbytes: int, seed: int) -> np.ndarray:
    """Seeded float32 payload for unpack tests: values in [-1, 1) written as
    raw bytes (the unpack reduction is defined on arbitrary floats)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nf = nbytes // 4
    vals = rng.uniform(-1.0, 1.0, nf).astype(np.float32)
    out = np.zeros(nbytes, dtype=np.uint8)
    out[: nf * 4] = vals.view(np.uint8)
    return out
