"""Host-side fault injection: a simulated failure of a device allocation or of
a metadata copy surfaces as an error from the call that met it, leaves no
device memory behind, and the next call succeeds with the same results.  No
device fault is caused: the injected site returns before the CUDA call."""
import numpy as np
import pytest

from paper_2606_23891_b300 import ics, sph

torch = pytest.importorskip("torch")

# uploads made by each plan: tasks, unpack cells, unpack entries; cells,
# targets, neighbour entries, items, counters
TASK_UPLOADS = 3
BATCH_UPLOADS = 5
EXPECT = {sph.SPH_FAULT_DEVICE_ALLOC: 2, sph.SPH_FAULT_COPY: 3}   # ENOMEM, ECUDA


@pytest.fixture(autouse=True)
def disarm():
    yield
    sph.sph_fault_inject(sph.SPH_FAULT_NONE, 0)


@pytest.mark.parametrize("site, countdown", [(3, 1), (-1, 1), (1, -1)])
def test_bad_arguments_are_rejected(site, countdown):
    with pytest.raises(sph.SphError) as e:
        sph.sph_fault_inject(site, countdown)
    assert e.value.status == 1


def test_arming_and_disarming_need_no_device():
    sph.sph_fault_inject(sph.SPH_FAULT_COPY, 4)
    sph.sph_fault_inject(sph.SPH_FAULT_COPY, 0)
    sph.sph_fault_inject(sph.SPH_FAULT_NONE, 7)


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.gpu
@pytest.mark.parametrize("site", [sph.SPH_FAULT_DEVICE_ALLOC, sph.SPH_FAULT_COPY])
def test_task_upload_failure_surfaces_then_recovers(site):
    from paper_2606_23891_b300.pipeline import Offload
    f = ics.gresho(n_side=24)
    ref = Offload(f, layout="pack_force_type")
    ref.step()
    want = ref.export()
    for k in range(1, TASK_UPLOADS + 1):
        sph.sph_fault_inject(site, k)
        with pytest.raises(sph.SphError) as e:
            Offload(f, layout="pack_force_type")
        assert e.value.status == EXPECT[site], k
    off = Offload(f, layout="pack_force_type")
    off.step()
    got = off.export()
    for name in want:
        assert np.array_equal(got[name], want[name]), name


@pytest.mark.gpu
@pytest.mark.parametrize("site", [sph.SPH_FAULT_DEVICE_ALLOC, sph.SPH_FAULT_COPY])
def test_batch_upload_failure_surfaces_then_recovers(site):
    from paper_2606_23891_b300.pipeline import Offload
    f = ics.gresho(n_side=24)
    ref = Offload(f, layout="pack_force_type")
    ref.batch()
    ref.list_step()
    want = ref.export()
    off = Offload(f, layout="pack_force_type")
    for k in range(1, BATCH_UPLOADS + 1):
        sph.sph_fault_inject(site, k)
        with pytest.raises(sph.SphError) as e:
            off.batch()
        assert e.value.status == EXPECT[site], k
        assert getattr(off, "bplan", None) is None
    off.batch()
    off.list_step()
    got = off.export()
    for name in want:
        assert np.array_equal(got[name], want[name]), name


@pytest.mark.gpu
def test_tree_plan_failure_surfaces_then_recovers():
    from paper_2606_23891_b300.pipeline import Offload
    f = ics.lognormal(n_side=24, seed=31)
    sph.sph_fault_inject(sph.SPH_FAULT_COPY, 3)
    with pytest.raises(sph.SphError) as e:
        Offload(f, layout="pack_force_type", plan="tree")
    assert e.value.status == 3
    off = Offload(f, layout="pack_force_type", plan="tree")
    off.list_step()
    assert np.isfinite(off.export()["a"]).all()


@pytest.mark.gpu
def test_failed_uploads_leave_no_device_memory():
    """Failures after the first allocations of a plan a few MB large, many
    times over: the device's free memory comes back to where it was."""
    from paper_2606_23891_b300.pipeline import Offload
    f = ics.gresho(n_side=64)
    off = Offload(f, layout="pack_force_type")
    off.batch()
    off.close_batch()
    x = np.ascontiguousarray(f["x"], np.float64)
    h = np.ascontiguousarray(f["h"], np.float32)
    gp = sph.grid_params((1.0, 1.0, 1.0), off.params.kernel_gamma, (0, 0, 0), 0)
    perm = np.empty(len(x), np.int64)
    before = _free_bytes()
    for rep in range(6):
        for k in range(2, BATCH_UPLOADS + 1):
            sph.sph_fault_inject(sph.SPH_FAULT_COPY, k)
            with pytest.raises(sph.SphError):
                off.batch()
            sph.sph_fault_inject(sph.SPH_FAULT_DEVICE_ALLOC, k)
            with pytest.raises(sph.SphError):
                off.batch()
        for k in range(2, TASK_UPLOADS + 1):
            t = sph.sph_tasks_build(len(x), x.ctypes.data, h.ctypes.data, gp, perm.ctypes.data)
            try:
                sph.sph_fault_inject(sph.SPH_FAULT_COPY, k)
                with pytest.raises(sph.SphError):
                    sph.sph_tasks_upload(t)
            finally:
                sph.sph_tasks_destroy(t)
    after = _free_bytes()
    assert before - after < (4 << 20), (before, after)


def _run_with_env(value: str, code: str):
    import os
    import subprocess
    import sys
    env = dict(os.environ, SPH_FAULT_INJECT=value)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env["PYTHONPATH"] = root + os.pathsep + env.get("PYTHONPATH", "")
    return subprocess.run([sys.executable, "-c", code], env=env, cwd=root,
                          capture_output=True, text=True, timeout=300)


def test_environment_variable_that_is_not_understood_is_reported():
    r = _run_with_env("sometimes", "from paper_2606_23891_b300 import sph; sph.lib()")
    assert r.returncode == 0, r.stderr
    assert "SPH_FAULT_INJECT=sometimes not understood" in r.stderr


@pytest.mark.gpu
def test_environment_variable_arms_the_site_at_load():
    code = """
from paper_2606_23891_b300 import ics, sph
from paper_2606_23891_b300.pipeline import Offload
f = ics.gresho(n_side=16)
try:
    Offload(f, layout="aos")
except sph.SphError as e:
    assert e.status == 3, e
    Offload(f, layout="aos").step()
    print("injected")
"""
    r = _run_with_env("copy:2", code)
    assert r.returncode == 0, r.stderr
    assert "injected" in r.stdout
