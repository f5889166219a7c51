"""CPU oracle of the SPH cell-pair offload pipeline (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It wraps ``sph_oracle.c`` (plain FP64 C,
brute-force O(N^2) minimum-image neighbour search) with numpy in and out, and
shares no code with the CUDA library.

Parity status of each function (what pins it is in the tests):
  W, dW/dr, dW/dH        pinned (volume integral, finite differences)
  density sums + ghost   pinned (lattice sum, FD in H, library neighbour
                         counts, sinusoidal div/curl fields)
  gradient               pinned (closed form v_sig = 2c, sinusoidal Laplacian)
  force                  pinned (momentum and energy conservation, lattice
                         symmetry, dh/dt = (h/3) f div v identity; magnitudes:
                         pressure force = -grad of the thermal energy by
                         central differences of the density sum, adiabatic
                         du/dt and dh/dt from the density's rate along the
                         flow, the continuum pressure gradient of a
                         sinusoidal u, viscous heating >= 0 and zero in
                         receding flow, a two-particle viscosity closed form)
  dh_scales              tolerance scales, not results (bounded below by the
                         sums they scale, equal to them when no term cancels)
  grid / tasks / bundles pinned (library KD-tree pair coverage)
  pack / unpack          pinned (minimum-image positions, bincount sums)
  store layouts          pinned (ctypes struct offsets, paper's 160 B record)
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import shutil
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

GAMMA = 5.0 / 3.0
KERNEL_GAMMA = 1.825742
BETA_VISC = 3.0
BALSARA_EPS = 1e-4

DENSITY, GRADIENT, FORCE = 0, 1, 2
LAYOUTS = ("aos", "aos_random", "pack_grad", "pack_force", "pack_shared",
           "pack_grad_type", "pack_force_type", "pack_shared_type", "soa",
           "pack_force_repl", "fused")
FIELD_NAMES = ("x", "v", "a", "mass", "h", "u", "u_dt", "rho", "time_bin",
               "alpha_visc", "alpha_diff", "rho_dh", "wcount", "wcount_dh",
               "div_v", "rot_v", "f_gradh", "pressure", "soundspeed", "balsara",
               "v_sig_grad", "laplace_u", "h_dt", "v_sig", "id", "ballast")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP) next to its source."""
    if force or not os.path.exists(_LIB) or \
            os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared",
                               "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("kernel_gamma", C.c_double),
                ("beta_visc", C.c_double), ("balsara_eps", C.c_double),
                ("support_eps", C.c_double), ("box", C.c_double * 3),
                ("active_bin", C.c_int32), ("pad", C.c_int32)]


class Fields(C.Structure):
    _fields_ = [(name, C.c_void_p) for name in FIELD_NAMES if name != "ballast"]


_lib = None


def _bind(L):
    d, i64, p = C.c_double, C.c_int64, C.c_void_p
    for name in ("oracle_w", "oracle_dw"):
        getattr(L, name).restype = d
        getattr(L, name).argtypes = [d]
    for name in ("oracle_W", "oracle_dWdr", "oracle_dWdH"):
        getattr(L, name).restype = d
        getattr(L, name).argtypes = [d, d]
    L.oracle_density.restype = i64
    L.oracle_density.argtypes = [i64, p, p, p, p, p, i64, p, p]
    L.oracle_dh_scales.restype = None
    L.oracle_dh_scales.argtypes = [i64, p, p, p, p, i64, p, p]
    L.oracle_ghost.restype = None
    L.oracle_ghost.argtypes = [i64, p, p, p, p, p, p, p]
    L.oracle_gradient.restype = i64
    L.oracle_gradient.argtypes = [i64, p, p, p, p, p, p, p, i64, p, p]
    L.oracle_force.restype = i64
    L.oracle_force.argtypes = [i64] + [p] * 13 + [p, i64, p, p]
    L.oracle_grid.restype = C.c_int
    L.oracle_grid.argtypes = [i64, p, p, p, d, p, p, p, p]
    L.oracle_tasks.restype = i64
    L.oracle_tasks.argtypes = [p, p, p, p, p]
    L.oracle_bundles.restype = i64
    L.oracle_bundles.argtypes = [i64, p, p, p, i64, p]
    L.oracle_buffer_bytes.restype = i64
    L.oracle_buffer_bytes.argtypes = [C.c_int, C.c_int, i64]
    L.oracle_pack.restype = C.c_int
    L.oracle_pack.argtypes = [C.c_int, p, p, p, p, p, p, i64, i64, p, p]
    L.oracle_unpack.restype = C.c_int
    L.oracle_unpack.argtypes = [C.c_int, p, i64, p, p, p, p, i64, i64, p]
    L.oracle_splitmix64.restype = C.c_uint64
    L.oracle_splitmix64.argtypes = [p]
    L.oracle_layout_group.restype = C.c_int
    L.oracle_layout_group.argtypes = [C.c_int, C.c_uint64, C.c_int, p, p, p, p]
    L.oracle_layout_ngroups.restype = C.c_int
    L.oracle_layout_ngroups.argtypes = [C.c_int, C.c_uint64]
    L.oracle_store_bytes.restype = i64
    L.oracle_store_bytes.argtypes = [C.c_int, C.c_uint64, i64]
    L.oracle_store_encode.restype = C.c_int
    L.oracle_store_encode.argtypes = [C.c_int, C.c_uint64, i64, p, p, p]
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = _bind(C.CDLL(build()))
    return _lib


def build_variant(edits) -> str:
    """Compile a copy of the oracle with text edits applied and return the
    library's path.  Tests use it to plant a mistake in the oracle (on the
    CPU) and show that a pin catches it; each ``(old, new)`` edit must match
    the source exactly once."""
    with open(_SRC) as fh:
        src = fh.read()
    for old, new in edits:
        if src.count(old) != 1:
            raise ValueError("edit does not match exactly once: %r" % old)
        src = src.replace(old, new)
    d = tempfile.mkdtemp(prefix="oracle_variant_")
    path = os.path.join(d, "sph_oracle_variant.c")
    with open(path, "w") as fh:
        fh.write(src)
    so = os.path.join(d, "liboracle_variant.so")
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                           "-o", so, path, "-lm"])
    return so


@contextlib.contextmanager
def variant(edits):
    """Run the oracle's functions on an edited copy for the duration of the
    block (see build_variant); the real oracle is restored afterwards."""
    global _lib
    saved = lib()
    so = build_variant(edits)
    try:
        _lib = _bind(C.CDLL(so))
        yield
    finally:
        _lib = saved
        shutil.rmtree(os.path.dirname(so), ignore_errors=True)


def _p(a):
    return None if a is None else a.ctypes.data


def params(box=(1.0, 1.0, 1.0), active_bin=0, support_eps=0.0,
           gamma=GAMMA, kernel_gamma=KERNEL_GAMMA, beta_visc=BETA_VISC,
           balsara_eps=BALSARA_EPS) -> Params:
    P = Params()
    P.gamma, P.kernel_gamma, P.beta_visc = gamma, kernel_gamma, beta_visc
    P.balsara_eps, P.support_eps = balsara_eps, support_eps
    P.box[0], P.box[1], P.box[2] = box
    P.active_bin = active_bin
    return P


def W(r, H):
    return lib().oracle_W(float(r), float(H))


def dWdr(r, H):
    return lib().oracle_dWdr(float(r), float(H))


def dWdH(r, H):
    return lib().oracle_dWdH(float(r), float(H))


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _sel(sel, n):
    if sel is None:
        return None, n
    s = _c(sel, np.int64)
    return s, s.shape[0]


def density(f: dict, P: Params, sel=None):
    """Raw density-loop sums (no self term) for the selected particles:
    (out[nsel, 8], pair count)."""
    n = f["x"].shape[0]
    s, ns = _sel(sel, n)
    x, v = _c(f["x"], np.float64), _c(f["v"], np.float32)
    m, h = _c(f["mass"], np.float32), _c(f["h"], np.float32)
    out = np.zeros((ns, 8), np.float64)
    pairs = lib().oracle_density(n, _p(x), _p(v), _p(m), _p(h), C.byref(P),
                                 ns, _p(s), _p(out))
    return out, pairs


def dh_scales(f: dict, P: Params, sel=None):
    """Conditioning scales of the cancelling h-derivative sums for the
    selected particles: (rho_dh scale, wcount_dh scale), each the sum of its
    terms' magnitudes with the self term included (tolerance scales only)."""
    n = f["x"].shape[0]
    s, ns = _sel(sel, n)
    x = _c(f["x"], np.float64)
    m, h = _c(f["mass"], np.float32), _c(f["h"], np.float32)
    out = np.zeros((ns, 2), np.float64)
    lib().oracle_dh_scales(n, _p(x), _p(m), _p(h), C.byref(P), ns, _p(s), _p(out))
    return out[:, 0], out[:, 1]


def ghost(f: dict, P: Params, dens, sel=None):
    """Ghost after density: out[nsel, 12] = rho, rho_dh, wcount, wcount_dh,
    div_v, rot_v[3], f_gradh, P, c, balsara."""
    n = f["x"].shape[0]
    s, ns = _sel(sel, n)
    m, h, u = (_c(f[k], np.float32) for k in ("mass", "h", "u"))
    dens = _c(dens, np.float64)
    out = np.zeros((ns, 12), np.float64)
    lib().oracle_ghost(ns, _p(s), _p(m), _p(h), _p(u), _p(dens), C.byref(P),
                       _p(out))
    return out


def gradient(f: dict, P: Params, rho, sel=None):
    n = f["x"].shape[0]
    s, ns = _sel(sel, n)
    x = _c(f["x"], np.float64)
    v, m, h, u = (_c(f[k], np.float32) for k in ("v", "mass", "h", "u"))
    rho = _c(rho, np.float64)
    out = np.zeros((ns, 2), np.float64)
    pairs = lib().oracle_gradient(n, _p(x), _p(v), _p(m), _p(h), _p(u),
                                  _p(rho), C.byref(P), ns, _p(s), _p(out))
    return out, pairs


def force(f: dict, P: Params, g: dict, sel=None):
    """Force loop; ``g`` holds full-length FP64 arrays rho, f_gradh, pressure,
    soundspeed, balsara (only neighbours of the selection are read)."""
    n = f["x"].shape[0]
    s, ns = _sel(sel, n)
    x = _c(f["x"], np.float64)
    v, m, h, u = (_c(f[k], np.float32) for k in ("v", "mass", "h", "u"))
    av, ad = _c(f["alpha_visc"], np.float32), _c(f["alpha_diff"], np.float32)
    tb = _c(f["time_bin"], np.int8)
    gs = [_c(g[k], np.float64) for k in ("rho", "f_gradh", "pressure",
                                         "soundspeed", "balsara")]
    out = np.zeros((ns, 6), np.float64)
    pairs = lib().oracle_force(n, _p(x), _p(v), _p(m), _p(h), _p(u),
                               *[_p(a) for a in gs], _p(av), _p(ad), _p(tb),
                               C.byref(P), ns, _p(s), _p(out))
    return out, pairs


def neighbours(f: dict, P: Params, i: int, symmetric: bool = True,
               margin: float = 1e-4):
    """Indices j != i with r_ij < max(H_i, H_j) (or H_i) times (1 + margin)."""
    x = np.asarray(f["x"], np.float64)
    box = np.array([P.box[0], P.box[1], P.box[2]])
    d = x[i] - x
    d -= box * np.rint(d / box)
    r = np.sqrt((d * d).sum(axis=1))
    H = P.kernel_gamma * np.asarray(f["h"], np.float64)
    lim = np.maximum(H[i], H) if symmetric else np.full_like(H, H[i])
    nb = np.nonzero(r < lim * (1.0 + margin))[0]
    return nb[nb != i]


def chain(f: dict, P: Params, sel=None) -> dict:
    """Full density -> ghost -> gradient -> force pass.  With ``sel`` only the
    selected particles' outputs are produced (their neighbours' densities are
    evaluated too, each by an O(N) brute-force scan).  Returns FP64 arrays
    indexed like ``sel`` (or all particles) plus per-loop pair counts."""
    n = f["x"].shape[0]
    if sel is None:
        J = np.arange(n, dtype=np.int64)
        sel_arr = J
    else:
        sel_arr = _c(sel, np.int64)
        parts = [sel_arr] + [neighbours(f, P, int(i)) for i in sel_arr]
        J = np.unique(np.concatenate(parts)).astype(np.int64)
    raw, pd = density(f, P, J)
    gh = ghost(f, P, raw, J)
    full = {k: np.full(n, np.nan) for k in
            ("rho", "f_gradh", "pressure", "soundspeed", "balsara")}
    for col, k in ((0, "rho"), (8, "f_gradh"), (9, "pressure"),
                   (10, "soundspeed"), (11, "balsara")):
        full[k][J] = gh[:, col]
    gr, pg = gradient(f, P, full["rho"], sel_arr)
    fo, pf = force(f, P, full, sel_arr)
    pos = np.searchsorted(J, sel_arr)
    ghs = gh[pos]
    out = {
        "rho": ghs[:, 0], "rho_dh": ghs[:, 1], "wcount": ghs[:, 2],
        "wcount_dh": ghs[:, 3], "div_v": ghs[:, 4], "rot_v": ghs[:, 5:8],
        "f_gradh": ghs[:, 8], "pressure": ghs[:, 9], "soundspeed": ghs[:, 10],
        "balsara": ghs[:, 11], "v_sig_grad": gr[:, 0], "laplace_u": gr[:, 1],
        "a": fo[:, 0:3], "u_dt": fo[:, 3], "h_dt": fo[:, 4], "v_sig": fo[:, 5],
    }
    if sel is None:
        out["pairs"] = {"density": pd, "gradient": pg, "force": pf}
    else:
        # density pairs of the selection only (the chain also scanned for J)
        _, pd_sel = density(f, P, sel_arr)
        out["pairs"] = {"density": pd_sel, "gradient": pg, "force": pf}
    return out


# --------------------------------------------------------------------------
# cells, tasks, bundles, pack, unpack, layouts
# --------------------------------------------------------------------------
def grid(f: dict, box=(1.0, 1.0, 1.0), kernel_gamma=KERNEL_GAMMA, ncell=None):
    """(ncell[3], perm[n], cell_start[ncell + 1]) or None if invalid."""
    n = f["x"].shape[0]
    x, h = _c(f["x"], np.float64), _c(f["h"], np.float32)
    bx = np.array(box, np.float64)
    nin = np.zeros(3, np.int32) if ncell is None else np.array(ncell, np.int32)
    nout = np.zeros(3, np.int32)
    if lib().oracle_grid(n, _p(x), _p(h), _p(bx), kernel_gamma, _p(nin),
                         _p(nout), None, None) != 0:
        return None
    perm = np.zeros(n, np.int64)
    cs = np.zeros(int(np.prod(nout.astype(np.int64))) + 1, np.int64)
    lib().oracle_grid(n, _p(x), _p(h), _p(bx), kernel_gamma, _p(nin), _p(nout),
                      _p(perm), _p(cs))
    return nout, perm, cs


def tasks(ncell, cell_start):
    nc = np.array(ncell, np.int32)
    cs = _c(cell_start, np.int64)
    nt = lib().oracle_tasks(_p(nc), _p(cs), None, None, None)
    ci = np.zeros(nt, np.int32)
    cj = np.zeros(nt, np.int32)
    sh = np.zeros((nt, 3), np.int8)
    lib().oracle_tasks(_p(nc), _p(cs), _p(ci), _p(cj), _p(sh))
    return ci, cj, sh


def bundles(ci, cj, cell_start, max_slots=0):
    ci, cj = _c(ci, np.int32), _c(cj, np.int32)
    cs = _c(cell_start, np.int64)
    nb = lib().oracle_bundles(ci.shape[0], _p(ci), _p(cj), _p(cs), max_slots, None)
    bs = np.zeros(nb + 1, np.int64)
    lib().oracle_bundles(ci.shape[0], _p(ci), _p(cj), _p(cs), max_slots, _p(bs))
    return bs


def buffer_bytes(loop: int, in_or_out: int, nslots: int) -> int:
    return lib().oracle_buffer_bytes(loop, in_or_out, nslots)


def bundle_slots(ci, cj, cell_start, t0, t1) -> int:
    cnt = np.diff(np.asarray(cell_start, np.int64))
    s = cnt[ci[t0:t1]].sum()
    cjs = np.asarray(cj[t0:t1])
    s += cnt[cjs[cjs >= 0]].sum()
    return int(s)


def _fields_struct(f: dict, keep: list):
    F = Fields()
    for name in FIELD_NAMES:
        if name == "ballast" or name not in f:
            continue
        arr = f[name]
        if not arr.flags["C_CONTIGUOUS"]:
            raise ValueError("field %s must be C-contiguous" % name)
        keep.append(arr)
        setattr(F, name, arr.ctypes.data)
    return F


def pack(loop: int, f: dict, perm, cell_start, ci, cj, shift, t0, t1,
         box=(1.0, 1.0, 1.0)) -> np.ndarray:
    keep = []
    F = _fields_struct(f, keep)
    S = bundle_slots(ci, cj, cell_start, t0, t1)
    buf = np.zeros(buffer_bytes(loop, 0, S), np.uint8)
    bx = np.array(box, np.float64)
    arrs = [_c(perm, np.int64), _c(cell_start, np.int64), _c(ci, np.int32),
            _c(cj, np.int32), _c(shift, np.int8)]
    lib().oracle_pack(loop, C.byref(F), *[_p(a) for a in arrs], t0, t1,
                      _p(bx), _p(buf))
    return buf


def unpack(loop: int, f: dict, perm, cell_start, ci, cj, t0, t1, buf) -> None:
    """Fold result lanes into the output fields of ``f`` in place."""
    keep = []
    F = _fields_struct(f, keep)
    n = f["x"].shape[0]
    arrs = [_c(perm, np.int64), _c(cell_start, np.int64), _c(ci, np.int32),
            _c(cj, np.int32)]
    b = _c(buf, np.uint8)
    lib().oracle_unpack(loop, C.byref(F), n, *[_p(a) for a in arrs], t0, t1, _p(b))


def splitmix64(seed: int, count: int):
    st = C.c_uint64(seed)
    return [lib().oracle_splitmix64(C.byref(st)) for _ in range(count)]


def layout_groups(layout: int, seed: int = 0):
    """[(record_bytes, [(field_id, comp, offset), ...]), ...]"""
    L = lib()
    ng = L.oracle_layout_ngroups(layout, seed)
    out = []
    for g in range(ng):
        nm = C.c_int32()
        fl = np.zeros(32, np.int32)
        co = np.zeros(32, np.int32)
        of = np.zeros(32, np.int32)
        rec = L.oracle_layout_group(layout, seed, g, C.byref(nm), _p(fl), _p(co), _p(of))
        out.append((rec, [(int(fl[k]), int(co[k]), int(of[k])) for k in range(nm.value)]))
    return out


def store_bytes(layout: int, n: int, seed: int = 0) -> int:
    return lib().oracle_store_bytes(layout, seed, n)


def store_encode(layout: int, f: dict, perm=None, seed: int = 0) -> np.ndarray:
    keep = []
    F = _fields_struct(f, keep)
    n = f["x"].shape[0]
    out = np.zeros(store_bytes(layout, n, seed), np.uint8)
    pm = None if perm is None else _c(perm, np.int64)
    lib().oracle_store_encode(layout, seed, n, C.byref(F), _p(pm), _p(out))
    return out
