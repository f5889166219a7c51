"""Neighbour-list variant of the batched cycle: the same results as the tile
kernels (to the rounding order of r^2) and as the oracle, on the grid and
the tree plans; pool sizing and its overflow report."""
import numpy as np
import pytest

from paper_2606_23891_b300 import ics, sph

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2606_23891_b300.pipeline import Offload  # noqa: E402
from test_parity_gpu import PARITY_CASES, check_physics, ragged, rms_err  # noqa: E402


@pytest.mark.parametrize("threads", [64, 128, 256])
@pytest.mark.parametrize("case", sorted(PARITY_CASES))
def test_list_pass_matches_the_oracle(case, threads):
    f = PARITY_CASES[case]()
    off = Offload(f, layout="pack_force_type")
    off.batch(threads=threads)
    off.list_step()
    check_physics(f, off.export())


@pytest.mark.parametrize("mtc", [0, 37])
def test_list_agrees_with_the_tile_kernels(mtc):
    f = ragged(24, 8)
    off = Offload(f, layout=6)
    off.batch(max_target_cells=mtc)
    off.batch_step()
    a = off.export()
    off.list_step()
    b = off.export()
    for k in a:
        assert rms_err(b[k], a[k]) <= 1e-6, k


def test_list_on_the_tree_plan_and_inactive_particles():
    f = ics.lognormal(n_side=24, seed=31)
    f["time_bin"][::4] = 5
    off = Offload(f, layout=5, plan="tree", params=sph.params(active_bin=2))
    off.batch(max_target_cells=101)
    pre = {"a": np.full((f["x"].shape[0], 3), 7.0, np.float32)}
    off.import_fields(pre, ("a",))
    off.list_step()
    got = off.export()
    inactive = f["time_bin"] > 2
    assert np.all(got["a"][inactive] == 7.0)
    sel = np.nonzero(~inactive)[0]
    check_physics(f, got, sel=sel, active_bin=2)


def test_list_steps_are_reproducible_and_graph_replay_matches():
    from paper_2606_23891_b300.autotune import GraphStep
    f = ragged(12, 41)
    off = Offload(f, layout=8)
    off.batch(threads=64)
    off.list_step()
    a = off.export()
    off.list_step()
    b = off.export()
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    gs = GraphStep(off, step=off.list_step)
    gs.replay()
    torch.cuda.synchronize()
    c = off.export()
    for k in a:
        np.testing.assert_array_equal(a[k], c[k], err_msg=k)


def test_list_pool_overflow_is_reported_and_recovered():
    f = ragged(12, 5)
    off = Offload(f, layout=0)
    off.batch()
    small = sph.sph_batch_list_bytes(off.bplan, 2)
    buf = torch.zeros(small, dtype=torch.uint8, device=off.device)
    sph.sph_batch_list_build(off.store, off.bplan, off.bbuf_in.data_ptr(), buf.data_ptr(),
                             small, off.params, off.stream)
    need, overflow = sph.sph_batch_list_status(buf.data_ptr())
    assert overflow and need > 2
    with pytest.raises(sph.SphError):
        sph.sph_sync(off.stream)
    sph.sph_sync(off.stream)                      # the error was cleared
    big = sph.sph_batch_list_bytes(off.bplan, need)
    buf = torch.zeros(big, dtype=torch.uint8, device=off.device)
    sph.sph_batch_list_build(off.store, off.bplan, off.bbuf_in.data_ptr(), buf.data_ptr(),
                             big, off.params, off.stream)
    need2, overflow2 = sph.sph_batch_list_status(buf.data_ptr())
    assert not overflow2 and need2 == need
    with pytest.raises(sph.SphError):             # buffer below the fixed tables
        sph.sph_batch_list_build(off.store, off.bplan, off.bbuf_in.data_ptr(), buf.data_ptr(),
                                 256, off.params, off.stream)


def test_streaming_steps_give_each_steps_results():
    """Overlapped end-to-end steps: step k's results in pinned memory equal a
    plain list step on step k's inputs, with the copies of neighbouring
    steps in flight."""
    from paper_2606_23891_b300.pipeline import INPUTS, StreamingSteps, field_spec
    base = ragged(12, 60)
    fs = []
    for k in range(3):        # same positions (the plan holds), other v and u
        f = {key: v.copy() for key, v in base.items()}
        rng = np.random.Generator(np.random.PCG64(70 + k))
        f["v"] += rng.uniform(-0.2, 0.2, f["v"].shape).astype(np.float32)
        f["u"] *= rng.uniform(0.8, 1.2, f["u"].shape).astype(np.float32)
        fs.append(f)
    off = Offload(fs[0], layout=6)
    off.batch()
    ref = []
    for f in fs:
        off.import_fields(f)
        off.list_step()
        ref.append(off.export())
    ss = StreamingSteps(off, off.list_step)
    pins_in, pins_out = [], []
    for f in fs:
        d = {}
        for name in INPUTS:
            dt, _ = field_spec(name)
            d[name] = torch.from_numpy(np.ascontiguousarray(f[name], dt)).pin_memory()
        pins_in.append(d)
        pins_out.append({k: torch.empty(v.shape, dtype=v.dtype).pin_memory()
                         for k, v in ss.dev_out[0].items()})
    for k in range(3):
        ss.step(pins_in[k], pins_out[k])
    ss.drain()
    torch.cuda.synchronize()
    for k in range(3):
        for name, v in ref[k].items():
            np.testing.assert_array_equal(pins_out[k][name].numpy(), v, err_msg=name)


def test_list_and_batch_api_reject_misuse():
    f = ragged(12, 52)
    off = Offload(f, layout=0)
    off.batch()
    off.list_step()
    b, st = off.bplan, off.stream
    lb = off.blist_bytes
    with pytest.raises(sph.SphError):          # misaligned list buffer
        sph.sph_batch_list_build(off.store, b, off.bbuf_in.data_ptr(),
                                 off.blist.data_ptr() + 8, lb, off.params, st)
    with pytest.raises(sph.SphError):          # list buffer below its fixed tables
        sph.sph_batch_offload_loop_list(off.store, b, 1, off.bbuf_in.data_ptr(),
                                        off.bbuf_out.data_ptr(), off.blist.data_ptr(), 512,
                                        off.params, st)
    with pytest.raises(sph.SphError):          # bundle out of range
        sph.sph_batch_list_interact(b, 1, 5, off.bbuf_in.data_ptr(), off.bbuf_out.data_ptr(),
                                    off.blist.data_ptr(), lb, off.params, st)
    with pytest.raises(sph.SphError):          # unknown loop
        sph.sph_batch_pack_list(off.store, b, 3, 0, off.bbuf_in.data_ptr(), off.params, st)
    with pytest.raises(sph.SphError):          # a device store on the host-staged call
        sph.sph_batch_offload_loop_host(off.store, b, 0, [1, 1], [1, 1], [1, 1], [1, 1],
                                        off.params, [0, 0])
    with pytest.raises(sph.SphError):          # stores of different particle counts
        g = ragged(8, 53)
        other = Offload(g, layout=0)
        sph.sph_store_convert(other.store, off.store, st)
    with pytest.raises(sph.SphError):          # tree plan with a support above half the box
        bad = {k: v.copy() for k, v in f.items()}
        bad["h"][0] = 0.3
        Offload(bad, plan="tree")
    sph.sph_sync(st)
    # the failed calls left nothing behind: the step still matches
    a = off.export()
    off.list_step()
    for k, v in off.export().items():
        np.testing.assert_array_equal(v, a[k])
