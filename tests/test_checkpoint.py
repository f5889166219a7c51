"""Checkpoint and resume: the file round-trips every field exactly, damaged
files are refused, and a run resumed from a checkpoint continues with the
results of the uninterrupted run."""
import os

import numpy as np
import pytest

from paper_2606_23891_b300 import build, checkpoint, ics, sph
from paper_2606_23891_b300.pipeline import HostOffload


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def fields(seed=5, n_side=10):
    f = ics.perturb(ics.uniform_lattice(n_side=n_side, jitter=0.45, seed=seed), seed=seed + 1,
                    v_amp=0.3, u_amp=0.3, alpha_diff=0.5, h_amp=0.1)
    rng = np.random.Generator(np.random.PCG64(seed + 2))
    f["time_bin"] = rng.integers(0, 3, len(f["x"])).astype(np.int8)
    return f


def test_file_round_trip_is_exact(tmp_path):
    rng = np.random.Generator(np.random.PCG64(1))
    arrays = {"x": rng.random((37, 3)), "t": rng.integers(-5, 5, 37).astype(np.int8),
              "id": rng.integers(0, 1 << 40, 37), "u": rng.random(37).astype(np.float32),
              "empty": np.zeros((0, 3), np.float32)}
    meta = {"n": 37, "note": "round trip", "box": [1.0, 2.0, 0.5]}
    p = str(tmp_path / "c.sph")
    checkpoint.write(p, meta, arrays)
    m2, a2 = checkpoint.read(p)
    assert m2 == meta
    assert list(a2) == list(arrays)
    for k in arrays:
        assert a2[k].dtype == arrays[k].dtype and np.array_equal(a2[k], arrays[k]), k


def test_damaged_files_are_refused(tmp_path):
    p = str(tmp_path / "c.sph")
    checkpoint.write(p, {"n": 64}, {"x": np.arange(192, dtype=np.float64).reshape(64, 3),
                                    "u": np.ones(64, np.float32)})
    raw = open(p, "rb").read()
    cases = {"magic": b"NOTACKPT\n" + raw[9:], "header": raw[:20], "data": raw[:-10]}
    flip = bytearray(raw)
    flip[len(raw) - 100] ^= 0x40
    cases["bit flip"] = bytes(flip)
    for name, body in cases.items():
        q = str(tmp_path / ("bad_" + name.replace(" ", "_")))
        open(q, "wb").write(body)
        with pytest.raises(ValueError):
            checkpoint.read(q)


@pytest.mark.parametrize("layout, other", [("aos", "soa"), ("aos_random", "pack_force_type"),
                                           ("pack_force_repl", "fused")])
def test_host_store_resumes_with_every_field(tmp_path, layout, other):
    """Every field of a host store (not only the inputs) comes back, in the
    saved layout and in another one."""
    f = fields()
    off = HostOffload(f, layout=layout, seed=9, box=(1.0, 1.0, 1.0), gpu=False)
    rng = np.random.Generator(np.random.PCG64(3))
    extra = {}
    for k in sph.FIELD_NAMES:
        if k in f:
            continue
        a = off.export([k])[k]
        extra[k] = (rng.standard_normal(a.shape) * 3).astype(a.dtype)
    off.import_fields(extra, names=tuple(extra))
    want = off.export(sph.FIELD_NAMES)
    p = str(tmp_path / "h.sph")
    checkpoint.save(off, p)
    for lay in (None, other):
        back = checkpoint.resume(p, layout=lay, host=True, gpu=False)
        assert back.layout == (off.layout if lay is None else sph.LAYOUTS[lay])
        assert back.seed == 9
        got = back.export(sph.FIELD_NAMES)
        for k in sph.FIELD_NAMES:
            assert np.array_equal(got[k], want[k]), (lay, k)
        if lay is None:
            assert np.array_equal(back.store_bytes(), off.store_bytes())


def test_resume_checks_the_particle_count(tmp_path):
    p = str(tmp_path / "c.sph")
    checkpoint.write(p, {"n": 5, "layout": 0, "seed": 0, "box": [1, 1, 1], "plan": "grid",
                         "leaf_max": 64, "params": {}}, {"x": np.zeros((4, 3))})
    with pytest.raises(ValueError):
        checkpoint.resume(p, host=True, gpu=False)


@pytest.mark.gpu
@pytest.mark.parametrize("plan", ["grid", "tree"])
def test_resumed_run_continues_bit_for_bit(tmp_path, plan):
    """Step, checkpoint, step again; a run resumed from the checkpoint gives
    the second step's results exactly."""
    from paper_2606_23891_b300.pipeline import Offload
    f = ics.lognormal(n_side=24, seed=31) if plan == "tree" else ics.gresho(n_side=24)
    off = Offload(f, layout="pack_force_type", seed=4, plan=plan)
    off.batch()
    off.list_step()
    p = str(tmp_path / "run.sph")
    checkpoint.save(off, p)
    off.list_step()
    want = off.export(sph.FIELD_NAMES)
    back = checkpoint.resume(p)
    back.batch()
    back.list_step()
    got = back.export(sph.FIELD_NAMES)
    for k in sph.FIELD_NAMES:
        assert np.array_equal(got[k], want[k]), k
    os.remove(p)
