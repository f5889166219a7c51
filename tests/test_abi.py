"""The C-ABI library loads, exports every entry point of include/sph.h, and
its host-side logic (layout engine, cell grid, task list, bundles, buffer
sizes, argument checks) matches the oracle's independent definitions.  No
call here touches a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
from paper_2606_23891_b300 import build, ics, sph

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sph.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sph_\w+)\s*\(", src)))


def test_library_exports_every_declared_entry_point():
    names = declared_functions()
    assert len(names) >= 25
    lib = C.CDLL(sph.LIB_PATH)
    for name in names:
        assert hasattr(lib, name), name
    # the binding wraps all of them under the same names
    for name in names:
        assert hasattr(sph, name), name


def test_binding_structs_match_the_header():
    src = open(os.path.join(ROOT, "include", "sph.h")).read()
    body = src[src.index("typedef struct {\n    double *x;"):src.index("} sph_fields;")]
    names = re.findall(r"\*(\w+);", body)
    assert tuple(names) == sph.FIELD_NAMES
    assert C.sizeof(sph.Fields) == 8 * len(names)
    assert C.sizeof(sph.Params) == 40 and C.sizeof(sph.GridParams) == 56


@pytest.mark.parametrize("layout", range(11))
@pytest.mark.parametrize("seed", [0, 17])
def test_layout_engine_matches_the_oracle(layout, seed):
    assert sph.sph_layout_group_count(layout, seed) == \
        len(oracle.layout_groups(layout, seed))
    for g, (rec, mem) in enumerate(oracle.layout_groups(layout, seed)):
        assert sph.sph_layout_describe(layout, seed, g) == (rec, mem)
    for n in (0, 1, 1000, 4097):
        assert sph.sph_store_bytes(n, layout, seed) == oracle.store_bytes(layout, n, seed)


def test_aos_is_160_bytes_and_splits_shrink_the_pack_views():
    assert sph.sph_layout_describe(sph.SPH_AOS, 0, 0)[0] == 160
    # the 52-byte gradient view is one 56-byte substruct in pack-gradient
    rec, mem = sph.sph_layout_describe(sph.SPH_SAOS_PACK_GRAD, 0, 0)
    assert rec == 56 and [m[0] for m in mem] == [0, 1, 3, 4, 5, 7]


def test_bad_arguments_are_rejected_with_a_message():
    L = sph.lib()
    assert L.sph_store_bytes(10, 99, 0) == 0
    assert L.sph_store_bytes(-1, 0, 0) == 0
    h = C.c_void_p()
    rc = L.sph_store_create(10, 0, 0, None, 0, C.byref(h))
    assert rc == 1 and b"store needs" in L.sph_last_error()
    gp = sph.grid_params()
    rc = L.sph_tasks_build(10, None, None, C.byref(gp), None, C.byref(h))
    assert rc == 1 and b"bad arguments" in L.sph_last_error()
    with pytest.raises(sph.SphError) as e:
        sph.sph_layout_describe(0, 0, 5)
    assert e.value.status == 1
    assert L.sph_buffer_bytes(None, 0, 0) == 0


def _build(f, **kw):
    n = f["x"].shape[0]
    x = np.ascontiguousarray(f["x"])
    h = np.ascontiguousarray(f["h"])
    perm = np.empty(n, np.int64)
    gp = sph.grid_params(**kw)
    t = sph.sph_tasks_build(n, x.ctypes.data, h.ctypes.data, gp, perm.ctypes.data)
    info = sph.sph_tasks_info(t)
    nt = info["ntasks"]
    ncell = info["ncell_x"] * info["ncell_y"] * info["ncell_z"]
    ci = np.empty(nt, np.int32)
    cj = np.empty(nt, np.int32)
    sh = np.empty((nt, 3), np.int8)
    cs = np.empty(ncell + 1, np.int64)
    bs = np.empty(info["nbundles"] + 1, np.int64)
    sph.sph_tasks_get(t, ci.ctypes.data, cj.ctypes.data, sh.ctypes.data, cs.ctypes.data,
                      bs.ctypes.data)
    return t, info, perm, ci, cj, sh, cs, bs


CASES = {
    "lattice16": lambda: ics.uniform_lattice(),
    "ragged12": lambda: ics.uniform_lattice(n_side=12, jitter=0.45, seed=3),
    "random": lambda: ics.perturb(ics.uniform_lattice(n_side=14, jitter=0.5, seed=9),
                                  seed=10, h_amp=0.2),
    "gresho32": lambda: ics.gresho(n_side=32),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("budget", [0, 700, 5000])
def test_task_builder_matches_the_oracle(case, budget):
    f = CASES[case]()
    t, info, perm, ci, cj, sh, cs, bs = _build(f, bundle_max_slots=budget)
    try:
        nc, operm, ocs = oracle.grid(f)
        assert (info["ncell_x"], info["ncell_y"], info["ncell_z"]) == tuple(nc)
        np.testing.assert_array_equal(perm, operm)
        np.testing.assert_array_equal(cs, ocs)
        oci, ocj, osh = oracle.tasks(nc, ocs)
        np.testing.assert_array_equal(ci, oci)
        np.testing.assert_array_equal(cj, ocj)
        np.testing.assert_array_equal(sh, osh)
        obs = oracle.bundles(oci, ocj, ocs, budget)
        np.testing.assert_array_equal(bs, obs)
        big = max(oracle.bundle_slots(oci, ocj, ocs, obs[b], obs[b + 1])
                  for b in range(len(obs) - 1))
        for loop in range(3):
            for io in range(2):
                assert sph.sph_buffer_bytes(t, loop, io) == oracle.buffer_bytes(loop, io, big)
    finally:
        sph.sph_tasks_destroy(t)


def test_task_builder_rejects_supports_wider_than_a_third_of_the_box():
    f = ics.uniform_lattice(n_side=8)
    with pytest.raises(sph.SphError) as e:
        _build(f)
    assert e.value.status == 6
    f = ics.uniform_lattice(n_side=16)
    with pytest.raises(sph.SphError):
        _build(f, ncell=(9, 9, 9))      # edges below the largest support


def test_empty_particle_set_builds_no_tasks():
    f = ics.empty_fields(0)
    t, info, *_ = _build(f)
    assert info["ntasks"] == 0 and info["nbundles"] == 0
    assert sph.sph_buffer_bytes(t, 0, 0) == 0
    sph.sph_tasks_destroy(t)


def test_host_io_and_measurement_calls_check_their_arguments():
    """Sizes and argument checks of the host I/O handle, the staged-cycle
    statistics and the peak microbenchmark, without a GPU."""
    L = sph.lib()
    assert C.sizeof(sph.StagedStats) == 80
    src = open(os.path.join(ROOT, "include", "sph.h")).read()
    body = src[src.index("typedef struct {\n    double wall_s;"):src.index("} sph_staged_stats;")]
    assert re.findall(r"(?:double|int64_t) (\w+);", body) == [n for n, _ in sph.StagedStats._fields_]
    ins, outs = sph.Fields(), sph.Fields()
    ins.x = ins.v = 1          # selections: only non-NULL matters
    outs.rho = 1
    # two staging sets, each field rounded up to 256 bytes
    assert sph.sph_hostio_bytes(1000, ins, outs) == 2 * (24064 + 12032 + 4096)
    assert sph.sph_hostio_bytes(-1, ins, outs) == 0
    h = C.c_void_p()
    assert L.sph_hostio_create(None, None, C.byref(ins), C.byref(outs), None, 0, None, None,
                               C.byref(h)) == 1
    assert L.sph_hostio_begin(None, C.byref(ins), None) == 1
    assert L.sph_hostio_destroy(None) == 0
    fl = C.c_double()
    assert L.sph_peak_run(7, 10, None, None, C.byref(fl)) == 1
    assert L.sph_peak_run(0, 0, None, None, C.byref(fl)) == 1
    st = sph.StagedStats()
    arr = (C.c_void_p * 2)()
    assert L.sph_offload_loop_host_stats(None, None, 0, arr, arr, arr, arr, None, arr, 0,
                                         C.byref(st)) == 1
