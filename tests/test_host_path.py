"""Host side of the host-staged offload cycle (the paper's own setting): the
store in host memory, pack and unpack on the host.  Pack/unpack bytes and
values must be identical to the oracle's definitions; these tests need no
GPU."""
import numpy as np
import pytest

import oracle
from paper_2606_23891_b300 import build, ics, sph
from paper_2606_23891_b300.pipeline import HostOffload

ALL_FIELDS = ("x", "v", "a", "mass", "h", "u", "u_dt", "rho", "time_bin",
              "alpha_visc", "alpha_diff", "rho_dh", "wcount", "wcount_dh",
              "div_v", "rot_v", "f_gradh", "pressure", "soundspeed", "balsara",
              "v_sig_grad", "laplace_u", "h_dt", "v_sig", "id")


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def fields(seed):
    f = ics.perturb(ics.uniform_lattice(n_side=12, jitter=0.45, seed=seed), seed=seed + 1,
                    v_amp=0.3, u_amp=0.3, alpha_diff=0.5, h_amp=0.1)
    rng = np.random.Generator(np.random.PCG64(seed + 2))
    for k in ALL_FIELDS:
        if k in ("x", "v", "mass", "h", "id"):
            continue
        if f[k].dtype == np.float32:
            f[k][...] = rng.uniform(0.2, 2.0, f[k].shape).astype(np.float32)
    f["time_bin"][:] = rng.integers(0, 4, f["time_bin"].shape).astype(np.int8)
    return f


def lane_slices(loop, S):
    sizes = {0: [8, 8, 8, 16, 4], 1: [8, 8, 8, 16, 4, 4, 4],
             2: [8, 8, 8, 16, 4, 4, 4, 4, 4, 4, 4, 1]}[loop]
    out, o = [], 0
    for sz in sizes:
        out.append(slice(o, o + S * sz))
        o += (S * sz + 255) // 256 * 256
    return out


@pytest.mark.parametrize("layout", range(11))
def test_host_store_image_and_round_trip(layout):
    f = fields(3)
    off = HostOffload(f, layout=layout, gpu=False)
    off.import_fields(f, ALL_FIELDS)
    ref = oracle.store_encode(layout, {k: np.ascontiguousarray(f[k]) for k in ALL_FIELDS},
                              off.perm)
    np.testing.assert_array_equal(off.store_bytes(), ref)
    back = off.export(ALL_FIELDS)
    for k in ALL_FIELDS:
        np.testing.assert_array_equal(back[k], f[k])


@pytest.mark.parametrize("layout", [0, 1, 3, 7, 8])
@pytest.mark.parametrize("loop", [0, 1, 2])
def test_host_pack_is_bit_exact(layout, loop):
    f = fields(5)
    off = HostOffload(f, layout=layout, bundle_max_slots=4000, gpu=False)
    off.import_fields(f, ALL_FIELDS)
    ci, cj, sh, cs, bs = off.task_list()
    buf = off.host_in[0][0]
    for b in range(len(bs) - 1):
        sph.sph_pack_host(off.store, off.tasks, loop, b, buf.ctypes.data)
        ref = oracle.pack(loop, f, off.perm, cs, ci, cj, sh, int(bs[b]), int(bs[b + 1]))
        S = oracle.bundle_slots(ci, cj, cs, bs[b], bs[b + 1])
        for sl in lane_slices(loop, S):
            np.testing.assert_array_equal(buf[sl], ref[sl])


@pytest.mark.parametrize("layout", [0, 4, 8])
@pytest.mark.parametrize("loop", [0, 1, 2])
def test_host_unpack_is_bit_exact(layout, loop):
    f = fields(7)
    off = HostOffload(f, layout=layout, bundle_max_slots=3000, gpu=False)
    off.import_fields(f, ALL_FIELDS)
    ci, cj, sh, cs, bs = off.task_list()
    ref = {k: np.ascontiguousarray(f[k]).copy() for k in ALL_FIELDS}
    buf = off.host_out[0][0]
    for b in range(len(bs) - 1):
        S = oracle.bundle_slots(ci, cj, cs, bs[b], bs[b + 1])
        lanes = ics.random_result_lanes(oracle.buffer_bytes(loop, 1, S), seed=200 + b)
        buf[: len(lanes)] = lanes
        sph.sph_unpack_host(off.store, off.tasks, loop, b, buf.ctypes.data)
        oracle.unpack(loop, ref, off.perm, cs, ci, cj, int(bs[b]), int(bs[b + 1]), lanes)
    got = off.export(ALL_FIELDS)
    for k in ALL_FIELDS:
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)


def test_host_init_and_ghost_follow_the_oracle():
    f = fields(9)
    f["time_bin"][::2] = 5
    off = HostOffload(f, layout=6, gpu=False)
    off.import_fields(f, ALL_FIELDS)
    P = sph.params(active_bin=2)
    sph.sph_init_host(off.store, sph.SPH_FORCE, P)
    got = off.export(ALL_FIELDS)
    active = f["time_bin"] <= 2
    assert np.all(got["a"][active] == 0) and np.all(got["a"][~active] == f["a"][~active])
    assert np.all(got["v_sig"][active] == 0) and np.all(got["v_sig"][~active] == f["v_sig"][~active])
    # ghost on raw density sums (the oracle's own sums as input)
    raw, _ = oracle.density(f, oracle.params())
    g = {"rho": raw[:, 0].astype(np.float32), "rho_dh": raw[:, 1].astype(np.float32),
         "wcount": raw[:, 2].astype(np.float32), "wcount_dh": raw[:, 3].astype(np.float32),
         "div_v": raw[:, 4].astype(np.float32),
         "rot_v": np.ascontiguousarray(raw[:, 5:8]).astype(np.float32)}
    off.import_fields(g, list(g))
    sph.sph_ghost_host(off.store, sph.SPH_DENSITY, sph.params())
    got = off.export(ALL_FIELDS)
    ref = oracle.ghost({k: g[k] if k in g else f[k] for k in f},
                       oracle.params(), g_raw := np.concatenate(
                           [g["rho"][:, None], g["rho_dh"][:, None], g["wcount"][:, None],
                            g["wcount_dh"][:, None], g["div_v"][:, None], g["rot_v"]], 1))
    for col, k in ((0, "rho"), (8, "f_gradh"), (9, "pressure"), (10, "soundspeed")):
        np.testing.assert_allclose(got[k], ref[:, col], rtol=2e-6)
    np.testing.assert_allclose(got["balsara"], ref[:, 11], atol=1e-5)


@pytest.mark.parametrize("fission", range(5))
@pytest.mark.parametrize("layout", [0, 6, 8, 9, 10])
def test_loop_fission_variants_write_the_same_bytes(layout, fission):
    """Every loop-fission variant of the host pack gives the default pack's
    buffer, and every variant of the unpack its store (Sec. 3.3)."""
    f = fields(11)
    off = HostOffload(f, layout=layout, bundle_max_slots=5000, gpu=False)
    off.import_fields(f, ALL_FIELDS)
    ci, cj, sh, cs, bs = off.task_list()
    buf = off.host_in[0][0]
    ref = np.empty_like(buf)
    for loop in range(3):
        for b in range(len(bs) - 1):
            buf[:] = 0
            sph.sph_pack_host(off.store, off.tasks, loop, b, buf.ctypes.data)
            ref[:] = buf
            buf[:] = 0
            sph.sph_pack_host_fission(off.store, off.tasks, loop, b, buf.ctypes.data, fission)
            np.testing.assert_array_equal(buf, ref)
    a = HostOffload(f, layout=layout, bundle_max_slots=5000, gpu=False)
    a.import_fields(f, ALL_FIELDS)
    out = off.host_out[0][0]
    for loop in range(3):
        for b in range(len(bs) - 1):
            S = oracle.bundle_slots(ci, cj, cs, bs[b], bs[b + 1])
            lanes = ics.random_result_lanes(oracle.buffer_bytes(loop, 1, S), seed=300 + b)
            out[: len(lanes)] = lanes
            sph.sph_unpack_host(a.store, a.tasks, loop, b, out.ctypes.data)
            sph.sph_unpack_host_fission(off.store, off.tasks, loop, b, out.ctypes.data, fission)
    np.testing.assert_array_equal(off.store_bytes(), a.store_bytes())


def test_loop_fission_rejects_unknown_variants():
    f = fields(12)
    off = HostOffload(f, layout=0, gpu=False)
    buf = off.host_in[0][0]
    with pytest.raises(sph.SphError):
        sph.sph_pack_host_fission(off.store, off.tasks, 0, 0, buf.ctypes.data, 5)
