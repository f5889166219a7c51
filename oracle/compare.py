"""Error metrics of GPU outputs against the oracle's (test infrastructure).

One number per output field, each on the scale the parity bars use:
relative error for the positive sums (rho, wcount, f_gradh, pressure,
soundspeed, the two signal velocities), the conditioning scales of the
cancelling h-derivative sums (the sum of their terms' magnitudes, self term
included: oracle.dh_scales) for rho_dh and wcount_dh, max error
over the field's rms for the signed vector-like sums (div v, curl v,
Laplacian of u, a, du/dt, dh/dt), and the absolute error of the Balsara
switch (a number in [0, 1]).
"""
from __future__ import annotations

import numpy as np

RELATIVE = ("rho", "wcount", "f_gradh", "pressure", "soundspeed", "v_sig_grad", "v_sig")
RMS = ("laplace_u", "div_v", "rot_v", "a", "u_dt", "h_dt")
LOOP_OF = {"rho": "density", "rho_dh": "density", "wcount": "density",
           "wcount_dh": "density", "div_v": "density", "rot_v": "density",
           "f_gradh": "density", "pressure": "density", "soundspeed": "density",
           "balsara": "density", "v_sig_grad": "gradient", "laplace_u": "gradient",
           "a": "force", "u_dt": "force", "h_dt": "force", "v_sig": "force"}


def _rel(a, b):
    d = np.abs(a - b)
    return np.where(d == 0.0, 0.0, d / np.maximum(np.abs(b), 1e-300))


def errors(got: dict, ref: dict, scales) -> dict:
    """Per-field error of ``got`` (arrays indexed like ``ref``) against the
    oracle's ``ref``; ``scales`` = oracle.dh_scales of the same particles."""
    g = {k: np.asarray(got[k], np.float64) for k in LOOP_OF}
    r = {k: np.asarray(ref[k], np.float64) for k in LOOP_OF}
    s_rho, s_w = (np.asarray(s, np.float64) for s in scales)
    out = {}
    for k in RELATIVE:
        out[k] = float(np.max(_rel(g[k], r[k]), initial=0.0))
    for k, sc in (("rho_dh", s_rho), ("wcount_dh", s_w)):
        d = np.abs(g[k] - r[k])     # 0/0 (a lone particle's wcount_dh) reads as 0
        out[k] = float(np.max(np.where(d == 0.0, 0.0, d / np.maximum(sc, 1e-300)),
                              initial=0.0))
    for k in RMS:
        s = np.sqrt(np.mean(r[k] * r[k])) if r[k].size else 0.0
        e = float(np.max(np.abs(g[k] - r[k]), initial=0.0))
        out[k] = e / s if s > 0 else e
    out["balsara"] = float(np.max(np.abs(g["balsara"] - r["balsara"]), initial=0.0))
    return out


def per_loop(err: dict) -> dict:
    """Worst field error of each loop."""
    res = {}
    for k, v in err.items():
        loop = LOOP_OF[k]
        res[loop] = max(res.get(loop, 0.0), v)
    return res


def relative_distribution(got, ref, scale) -> dict:
    """Percentiles of |got - ref| / |ref| and of |got - ref| / scale (for a
    cancelling sum the first is large where the value is near 0)."""
    g, r = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    d = np.abs(g - r)
    rel = np.where(d == 0.0, 0.0, d / np.maximum(np.abs(r), 1e-300))
    cond = np.where(d == 0.0, 0.0, d / np.maximum(np.asarray(scale, np.float64), 1e-300))
    q = (50, 90, 99, 100)
    return {"rel_to_value": {"p%d" % p: float(np.percentile(rel, p)) for p in q},
            "rel_to_scale": {"p%d" % p: float(np.percentile(cond, p)) for p in q},
            "value_over_scale_median": float(np.median(np.abs(r) / np.asarray(scale)))}
