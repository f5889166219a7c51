"""The host-staged cycle end to end: store in pinned host memory, host pack,
H2D, kernel, D2H, host unpack, double-buffered on two streams."""
import numpy as np
import pytest

import oracle
from paper_2606_23891_b300 import ics

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2606_23891_b300.pipeline import HostOffload, Offload  # noqa: E402
from test_parity_gpu import check_physics, ragged, rms_err  # noqa: E402


@pytest.mark.parametrize("layout", [0, 6, 8])
def test_host_staged_pass_matches_oracle_and_device_path(layout):
    assert torch.cuda.is_available()
    f = ragged(24, 8)
    host = HostOffload(f, layout=layout, bundle_max_slots=40000)
    assert host.info["nbundles"] > 4          # exercises the double buffering
    host.step()
    got = host.export()
    check_physics(f, got)
    dev = Offload(f, layout=layout, bundle_max_slots=40000)
    dev.step()
    want = dev.export()
    # identical pack bytes, kernels and unpack fold; only the ghost's FP32
    # arithmetic runs on the host compiler instead of the GPU (about one ulp in
    # f_gradh, P, c, B), amplified by the cancellation in the force sums
    for k in want:
        assert rms_err(got[k], want[k]) <= 1e-5, k


def test_host_staged_gresho_slice():
    f = ics.perturb(ics.gresho(n_side=32), seed=4, alpha_diff=0.3)
    host = HostOffload(f, layout="pack_shared_type", bundle_max_slots=20000)
    host.step()
    check_physics(f, host.export())


# ------------------------------------------------ host-staged batched cycle --
@pytest.mark.parametrize("mtc", [0, 50])
def test_host_staged_batched_on_the_tree_plan(mtc):
    """A clustered set kept in pinned host memory, staged through the tree
    plan's bundles (the clustered host-staged configuration)."""
    from paper_2606_23891_b300 import sph
    f = ics.lognormal(n_side=24, seed=33)
    host = HostOffload(f, layout="pack_force_type", plan="tree", max_target_cells=mtc)
    if mtc:
        assert sph.sph_batch_info(host.bplan)["nbundles"] > 4
    host.batch_step()
    got = host.export()
    check_physics(f, got)
    dev = Offload(f, layout="pack_force_type", plan="tree")
    dev.batch_step()
    want = dev.export()
    for k in want:
        assert rms_err(got[k], want[k]) <= 1e-5, k


def test_host_staged_batched_on_the_grid_with_inactive_particles():
    from paper_2606_23891_b300 import sph
    f = ragged(24, 9)
    f["time_bin"][::3] = 5
    P = sph.params(active_bin=2)
    host = HostOffload(f, layout=8, params=P)
    host.batch(max_target_cells=40)
    pre = {"a": np.full((f["x"].shape[0], 3), 7.0, np.float32)}
    host.import_fields(pre, ("a",))
    host.batch_step()
    got = host.export()
    inactive = f["time_bin"] > 2
    assert np.all(got["a"][inactive] == 7.0)
    check_physics(f, got, sel=np.nonzero(~inactive)[0], active_bin=2)
