"""The batched pipeline on the octree-leaf plan (clustered sets) against the
oracle, against itself under other bundlings and leaf sizes, and against the
grid plan where both apply.  Same bars as the per-task cycle."""
import numpy as np
import pytest

import oracle
from oracle import compare
from paper_2606_23891_b300 import ics, sph

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2606_23891_b300.pipeline import Offload  # noqa: E402
from test_fp64_gpu import fp64_bars  # noqa: E402
from test_parity_gpu import check_physics, ragged, rms_err  # noqa: E402

CLUSTERED = {
    "lognormal24": lambda: ics.lognormal(n_side=24, seed=31),
    "lognormal32": lambda: ics.lognormal(n_side=32, seed=32),
}


def test_the_grid_plan_cannot_take_a_clustered_set():
    f = CLUSTERED["lognormal32"]()
    with pytest.raises(sph.SphError):
        Offload(f, layout="pack_force_type")


@pytest.mark.parametrize("leaf_max", [16, 64, 512])
@pytest.mark.parametrize("case", sorted(CLUSTERED))
def test_tree_plan_matches_the_oracle(case, leaf_max):
    f = CLUSTERED[case]()
    off = Offload(f, layout="pack_force_type", plan="tree", leaf_max=leaf_max)
    assert off.binfo["kind"] == 1 and off.binfo["max_cell"] <= leaf_max
    off.batch_step()
    ref, lo, hi = check_physics(f, off.export(), bands=True)
    for loop, key in ((0, "density"), (1, "gradient"), (2, "force")):
        c = off.count_pairs(loop)
        assert lo["pairs"][key] <= c <= hi["pairs"][key], key


@pytest.mark.parametrize("threads", [64, 256])
def test_tree_plan_bundling_and_threads_agree(threads):
    f = CLUSTERED["lognormal24"]()
    one = Offload(f, layout=0, plan="tree")
    one.batch_step()
    a = one.export()
    many = Offload(f, layout=8, plan="tree")
    many.batch(max_target_cells=37, threads=threads)
    assert many.binfo["nbundles"] > 5
    many.batch_step()
    b = many.export()
    for k in a:
        assert rms_err(b[k], a[k]) <= 1e-5, k


def test_tree_and_grid_plans_agree_on_a_lattice():
    f = ragged(24, 8)
    grid = Offload(f, layout=6)
    grid.batch()
    grid.batch_step()
    a = grid.export()
    tree = Offload(f, layout=6, plan="tree", leaf_max=48)
    tree.batch_step()
    b = tree.export()
    for k in a:
        assert rms_err(b[k], a[k]) <= 1e-5, k
    for loop in range(3):
        assert abs(tree.count_pairs(loop) - grid.count_pairs(loop)) <= 4


def test_tree_plan_fp64_path_and_inactive_particles():
    f = CLUSTERED["lognormal24"]()
    f["time_bin"][::3] = 5
    P = sph.params(active_bin=2)
    off = Offload(f, layout=5, plan="tree", params=P)
    pre = {"a": np.full((f["x"].shape[0], 3), 7.0, np.float32)}
    off.import_fields(pre, ("a",))
    off.fp64_step()
    got = off.export()
    inactive = f["time_bin"] > 2
    assert np.all(got["a"][inactive] == 7.0)
    sel = np.nonzero(~inactive)[0]
    ref = oracle.chain(f, oracle.params(active_bin=2), sel)
    sc = oracle.dh_scales(f, oracle.params(active_bin=2), sel)
    fp64_bars(compare.errors({k: v[sel] for k, v in got.items()}, ref, sc))


def test_tree_plan_graph_replay_is_bit_identical():
    from paper_2606_23891_b300.autotune import GraphStep
    f = CLUSTERED["lognormal24"]()
    off = Offload(f, layout=6, plan="tree")
    off.batch_step()
    a = off.export()
    gs = GraphStep(off)
    gs.replay()
    torch.cuda.synchronize()
    b = off.export()
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
