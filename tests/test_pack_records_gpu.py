"""The compact records of the list pipeline's pack (sph_batch_pack_list),
bit for bit against a numpy restatement of their definition, from the
particles' own fields: for every cell of a bundle, the slot order (the
particles sorted stably by the octant of their position's high part about
the centre of the cell's bounding box, cells of up to 32 particles and
above 2048 in store order), and for every slot the record of its particle:

  density (fixed-point plans): (X, Y, Z, H), (v, m) with X = round(x 2^32 / L)
      mod 2^32 stored as the float's bits and H = gamma_K h in FP32;
  density (two-float plans): (hi, H), (lo, m), (v, 0) and the same two lanes;
  gradient: (X, Y, Z, m / rho), (v, u), (H, 0, 0, 0);
  force: (hi, 1 / H), (lo, m), (v, u), (rho, f P / rho^2, alpha_visc B,
      alpha_diff) with P = (gamma - 1) rho u, the activity byte and h f / rho,

where hi is x rounded to 24 significant bits (ties away from zero) and lo
the remainder x - hi rounded to FP32, so hi + lo = x to 2^-48 relative; the
per-cell largest support; and the store index of each slot."""
import numpy as np
import pytest

from paper_2606_23891_b300 import ics, sph

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2606_23891_b300.pipeline import Offload  # noqa: E402
from test_parity_gpu import ragged  # noqa: E402

F32 = np.float32


def r256(b):
    return (b + 255) // 256 * 256


def lane_offsets(loop, S):
    """Byte offsets of a bundle buffer's lanes: nf float4 record lanes (the
    density loop two more), the store index lane, activity, h f / rho, cellh."""
    nf = (3, 4, 5)[loop]
    nl = nf + 2 if loop == 0 else nf
    rec = lambda f: r256(S * 16) * f
    perm = rec(nl)
    tb = perm + r256(S * 4)
    hf = tb + r256(S)
    return {"rec": rec, "fx": lambda k: rec(nf + k), "perm": perm, "tb": tb, "hf": hf,
            "cellh": hf + r256(S * 4)}


def split_hi_lo(x):
    """hi: x rounded to 24 significant bits, ties away from zero; lo: the
    remainder rounded to FP32 (integer arithmetic on the binary64 fields)."""
    x = np.asarray(x, np.float64)
    b = x.view(np.uint64)
    e = ((b >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64)
    m = (b & np.uint64((1 << 52) - 1)) | np.uint64(1 << 52)
    top = (m >> np.uint64(29)).astype(np.int64)
    top += ((m & np.uint64((1 << 29) - 1)) >= np.uint64(1 << 28)).astype(np.int64)
    hi = np.ldexp(top.astype(np.float64), e - 1023 - 23)
    hi = np.where(e < 1023 - 74, 0.0, hi) * np.sign(x)
    lo = np.where(e < 1023 - 74, 0.0, x - hi)
    return hi.astype(F32), lo.astype(F32)


def fixed_bits(x, box=1.0):
    X = np.rint(np.asarray(x, np.float64) * (4294967296.0 / box)).astype(np.int64)
    return (X & 0xFFFFFFFF).astype(np.uint32).view(F32)


def slot_order(hi):
    """Store positions of a cell's particles in slot order."""
    n = hi.shape[0]
    if n <= 32 or n > 2048:
        return np.arange(n)
    ctr = F32(0.5) * (hi.min(axis=0) + hi.max(axis=0))
    key = ((hi[:, 0] > ctr[0]).astype(np.int64) | (hi[:, 1] > ctr[1]).astype(np.int64) << 1 |
           (hi[:, 2] > ctr[2]).astype(np.int64) << 2)
    return np.argsort(key, kind="stable")


def f4(buf, off, S):
    return buf[off:off + S * 16].view(F32).reshape(S, 4)


def check_bundle(off, loop, b, fields, fixed):
    cells = sph.sph_batch_cells(off.bplan, b)
    S = int(cells[-1, 2] + cells[-1, 1])
    sph.sph_batch_pack_list(off.store, off.bplan, loop, b, off.bbuf_in.data_ptr(), off.params,
                            off.stream)
    torch.cuda.synchronize()
    L = lane_offsets(loop, S)
    buf = off.bbuf_in[: L["cellh"] + r256(4 * len(cells))].cpu().numpy()
    perm = buf[L["perm"]:L["perm"] + 4 * S].view(np.int32)
    orig = off.perm                    # store index -> original particle
    x = fields["x"]
    hi, lo = split_hi_lo(x.reshape(-1))
    hi, lo = hi.reshape(-1, 3), lo.reshape(-1, 3)
    kg = F32(1.825742)
    H = kg * fields["h"]
    # slot order and per-cell largest support
    cellh = buf[L["cellh"]:L["cellh"] + 4 * len(cells)].view(F32)
    want_perm = np.empty(S, np.int64)
    for c, (p0, n, slot) in enumerate(cells):
        ids = orig[p0:p0 + n]
        want_perm[slot:slot + n] = p0 + slot_order(hi[ids])
        if loop == 0:
            assert cellh[c] == H[ids].max(), c
    np.testing.assert_array_equal(perm, want_perm)
    o = orig[want_perm]                # each slot's original particle
    v, m, u = fields["v"][o], fields["mass"][o], fields["u"][o]
    rho, fg, bal = fields["rho"][o], fields["f_gradh"][o], fields["balsara"][o]
    Hs = H[o]
    X = fixed_bits(x[o].reshape(-1)).reshape(-1, 3)
    zero = np.zeros(S, F32)
    if loop == 0:
        want = {L["fx"](0): np.column_stack([X, Hs]), L["fx"](1): np.column_stack([v, m])}
        if not fixed:
            want.update({L["rec"](0): np.column_stack([hi[o], Hs]),
                         L["rec"](1): np.column_stack([lo[o], m]),
                         L["rec"](2): np.column_stack([v, zero])})
    elif loop == 1:
        want = {L["rec"](0): np.column_stack([X, m / rho]), L["rec"](1): np.column_stack([v, u]),
                L["rec"](2): np.column_stack([Hs, zero, zero, zero])}
    else:
        P = (F32(5.0 / 3.0) - F32(1.0)) * rho * u
        want = {L["rec"](0): np.column_stack([hi[o], F32(1.0) / Hs]),
                L["rec"](1): np.column_stack([lo[o], m]), L["rec"](2): np.column_stack([v, u]),
                L["rec"](3): np.column_stack([rho, fg * P / (rho * rho), fields["alpha_visc"][o] * bal,
                                              fields["alpha_diff"][o]])}
        np.testing.assert_array_equal(buf[L["tb"]:L["tb"] + S].view(np.int8),
                                      fields["time_bin"][o])
        np.testing.assert_array_equal(buf[L["hf"]:L["hf"] + 4 * S].view(F32),
                                      fields["h"][o] * (fg / rho))
    for lane_off, arr in want.items():
        got = f4(buf, lane_off, S)
        np.testing.assert_array_equal(got.view(np.uint32), np.asarray(arr, F32).view(np.uint32),
                                      err_msg="loop %d lane at %d" % (loop, lane_off))
    # the two-float split reconstructs every position to 2^-48 relative
    rec_x = hi.astype(np.float64) + lo.astype(np.float64)
    assert np.all(np.abs(rec_x - x) <= 2.0 ** -48 * np.abs(x))


def clumped(seed=78):
    """A background with a dense clump: one cell above 128 particles (packed
    by the block kernel) among cells of a few dozen (one warp each)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n_bg, n_cl = 3000, 400
    n = n_bg + n_cl
    f = ics.empty_fields(n)
    x = rng.uniform(0, 1, (n, 3))
    x[n_bg:] = 0.31 + rng.uniform(0, 0.04, (n_cl, 3))
    f["x"][:] = x
    f["v"][:] = rng.uniform(-0.5, 0.5, (n, 3)).astype(np.float32)
    f["mass"][:] = np.float32(1.0 / n)
    f["h"][:] = np.float32(0.07)
    f["u"][:] = rng.uniform(0.5, 1.5, n).astype(np.float32)
    f["alpha_visc"][:] = rng.uniform(0.1, 1.0, n).astype(np.float32)
    f["alpha_diff"][:] = rng.uniform(0.0, 0.3, n).astype(np.float32)
    f["time_bin"][::7] = 3
    return f


CASES = {
    "ragged24 grid (8 cells: fixed-point build)": (lambda: ragged(24, 8), "grid"),
    "lattice16 grid (4 cells: two-float build)": (lambda: ics.uniform_lattice(), "grid"),
    "clump grid (a cell above 128)": (clumped, "grid"),
    "lognormal24 tree": (lambda: ics.lognormal(n_side=24, seed=31), "tree"),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_list_pack_records_are_bit_exact(case):
    make, plan = CASES[case]
    f = make()
    off = Offload(f, layout="pack_force_type", plan=plan)
    if plan == "grid":
        off.batch()
    if case.startswith("clump"):
        assert off.info["max_cell"] > 128
    if plan == "grid":
        assert sph.sph_batch_list_fixed(off.bplan) == (off.info["ncell_x"] >= 5)
    off.list_step()                      # rho, f_gradh, balsara in the store
    sph.sph_sync(off.stream)
    got = off.export()
    fields = {k: np.asarray(f[k]) for k in ("x", "v", "mass", "h", "u", "alpha_visc",
                                            "alpha_diff", "time_bin")}
    fields.update({k: got[k] for k in ("rho", "f_gradh", "balsara")})
    fixed = sph.sph_batch_list_fixed(off.bplan)
    for loop in range(3):
        for b in range(off.binfo["nbundles"]):
            check_bundle(off, loop, b, fields, fixed)
