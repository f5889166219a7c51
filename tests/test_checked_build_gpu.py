"""Bounds of every gathered and scattered index, on the GPU.

compute-sanitizer is not available, so the library has an index-checked
build (libsph_check.so, -DSPH_CHECK): each checked index outside its buffer
latches SPH_EBOUNDS.  The cycles run under it on grid and tree plans, with one
and several bundles, and with the adjoint.  sph_sync must report no violation,
and the results must equal the default build's bit for bit."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RUN = r'''
import sys
import numpy as np, torch
sys.path.insert(0, "tests")
from paper_2606_23891_b300 import ics, sph
from paper_2606_23891_b300.pipeline import Offload
from test_parity_gpu import ragged
out = {}
def keep(tag, off):
    sph.sph_sync(off.stream)
    for k, v in off.export(("rho", "f_gradh", "v_sig_grad", "laplace_u", "a", "u_dt", "h_dt",
                            "v_sig")).items():
        out[tag + "/" + k] = v
cases = [("grid", ragged(12, 71), {}, 0), ("grid3", ragged(12, 72), {}, 37),
         ("grid8", ragged(24, 73), {}, 0),
         ("tree", ics.lognormal(n_side=24, seed=31), {"plan": "tree"}, 101)]
for tag, f, kw, mtc in cases:
    off = Offload(f, layout="pack_force_type", **kw)
    off.batch(max_target_cells=mtc)
    off.list_step(); keep(tag + "/list", off)
    off.batch_step(); keep(tag + "/batched", off)
    if tag == "grid":
        off.step(); keep(tag + "/per-task", off)
        off.batch()
        off.list_step()
        g = torch.Generator(device="cuda").manual_seed(3)
        abar = torch.randn((off.n, 3), device="cuda", generator=g)
        ebar = torch.randn(off.n, device="cuda", generator=g)
        gx, gm, gu = off.adjoint(abar, ebar)
        sph.sph_sync(off.stream)
        out["adjoint/gx"], out["adjoint/gm"], out["adjoint/gu"] = (
            gx.cpu().numpy(), gm.cpu().numpy(), gu.cpu().numpy())
np.savez(sys.argv[1], **out)
print("checked" if sph.LIB_PATH.endswith("_check.so") else "default", sph.LIB_PATH)
'''


def run(path, checked):
    env = dict(os.environ, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    env["SPH_CHECKED_BUILD"] = "1" if checked else "0"
    r = subprocess.run([sys.executable, "-c", RUN, path], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return r.stdout


def test_every_index_stays_in_bounds_and_results_are_unchanged(tmp_path):
    from paper_2606_23891_b300 import build
    build.build()
    build.build(check=True)
    a, b = str(tmp_path / "checked.npz"), str(tmp_path / "default.npz")
    assert run(a, True).startswith("checked")
    assert run(b, False).startswith("default")
    got, want = np.load(a), np.load(b)
    assert sorted(got.files) == sorted(want.files)
    for k in want.files:
        assert np.array_equal(got[k], want[k]), k
