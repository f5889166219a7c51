"""Neighbour-list variant of the batched cycle: the same results as the tile
kernels (to the rounding of the separations) and as the oracle, on the grid
and the tree plans; pool sizing and its overflow report."""
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
    """The list loops of density and gradient take separations from 32-bit
    fixed-point positions (one unit = box / 2^32, then one float rounding),
    the tile kernels from two-float ones: the results agree to a few 1e-7 of
    each field's rms, up to about 1e-6 in the cancelling sum of div v."""
    f = ragged(24, 8)
    off = Offload(f, layout=6)
    off.batch(max_target_cells=mtc)
    off.batch_step()
    a = off.export()
    off.list_step()
    b = off.export()
    for k in a:
        assert rms_err(b[k], a[k]) <= 5e-6, k


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
    from paper_2606_23891_b300.pipeline import (INPUTS, StreamingSteps, field_spec,
                                                fields_struct, host_fields_struct)
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
        d = ss.pinned_in()
        for name in INPUTS:
            dt, _ = field_spec(name)
            d[name].numpy()[...] = np.asarray(f[name], dt)
        pins_in.append(d)
        pins_out.append(ss.pinned_out())
    h2d, d2h = ss.bytes_per_step()
    assert h2d == sum(t.numel() * t.element_size() for t in pins_in[0].values())
    assert d2h == sum(t.numel() * t.element_size() for t in pins_out[0].values())
    for k in range(3):
        ss.step(pins_in[k], pins_out[k])
    ss.drain()
    torch.cuda.synchronize()
    for k in range(3):
        for name, v in ref[k].items():
            np.testing.assert_array_equal(pins_out[k][name].numpy(), v, err_msg=name)
    # pageable host memory and an unselected field are refused before any copy
    bad = {k: v.numpy().copy() for k, v in pins_in[0].items()}
    with pytest.raises(sph.SphError, match="page-locked"):
        sph.sph_hostio_begin(ss.io, host_fields_struct(bad), off.stream)
    extra = dict(pins_in[0])
    extra["rho"] = pins_out[0]["rho"]
    with pytest.raises(sph.SphError, match="not selected"):
        sph.sph_hostio_begin(ss.io, fields_struct(extra), off.stream)
    with pytest.raises(sph.SphError, match="no step was begun"):
        sph.sph_hostio_end(ss.io, fields_struct(pins_out[0]), off.stream)
    ss.close()


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


def _poisoned_outputs(f, seed):
    """Random values in every output field, so that a field the step should
    leave alone (inactive particles) shows if it was written."""
    from paper_2606_23891_b300.pipeline import OUTPUTS, field_spec
    rng = np.random.Generator(np.random.PCG64(seed))
    out = {}
    for k in OUTPUTS:
        dt, c = field_spec(k)
        shape = (len(f["x"]), c) if c > 1 else (len(f["x"]),)
        lo = 0.0 if k.startswith("v_sig") else -3.0     # signal velocities are >= 0
        out[k] = rng.uniform(lo, 3.0, shape).astype(dt)
    return out


@pytest.mark.parametrize("plan, mtc", [("grid", 0), ("grid", 37), ("tree", 101)])
def test_written_unpack_equals_init_then_fold(plan, mtc):
    """The unpack that writes each particle's result leaves the store byte for
    byte as sph_init followed by the adding unpack does (the cycles' former
    form), inactive particles of the force loop included; and the one-call
    list step equals the build followed by the three loop calls."""
    f = ics.lognormal(n_side=20, seed=44) if plan == "tree" else ragged(14, 46)
    f["time_bin"] = (np.arange(len(f["x"])) % 3).astype(np.int8)
    prm = sph.params(active_bin=1)
    poison = _poisoned_outputs(f, 9)
    offs = []
    for _ in range(3):
        o = Offload(f, layout=6, plan=plan, params=prm)
        o.batch(max_target_cells=mtc)
        o.import_fields(poison, tuple(poison))
        offs.append(o)
    fold, loops, step = offs
    # init + adding unpack, bundle by bundle
    fold.list_build()
    for loop in range(3):
        sph.sph_init(fold.store, loop, prm, fold.stream)
        for b in range(fold.binfo["nbundles"]):
            sph.sph_batch_pack_list(fold.store, fold.bplan, loop, b, fold.bbuf_in.data_ptr(),
                                    prm, fold.stream)
            sph.sph_batch_list_interact(fold.bplan, loop, b, fold.bbuf_in.data_ptr(),
                                        fold.bbuf_out.data_ptr(), fold.blist.data_ptr(),
                                        fold.blist_bytes, prm, fold.stream)
            sph.sph_batch_unpack(fold.store, fold.bplan, loop, b, fold.bbuf_out.data_ptr(),
                                 fold.bbuf_in.data_ptr(), fold.stream)
        sph.sph_ghost(fold.store, loop, prm, fold.stream)
    # the build, then the three loop calls (written unpack)
    loops.list_build()
    for loop in range(3):
        loops.list_loop(loop)
    # the one-call step
    step.list_step()
    want = fold.store_bytes()
    assert np.array_equal(loops.store_bytes(), want)
    assert np.array_equal(step.store_bytes(), want)
    got = step.export(("a", "u_dt", "v_sig"))
    inactive = f["time_bin"] > 1
    for k in got:
        assert np.array_equal(got[k][inactive], poison[k][inactive]), k


def test_written_unpack_in_the_tile_cycle_equals_init_then_fold():
    f = ragged(14, 47)
    f["time_bin"] = (np.arange(len(f["x"])) % 2).astype(np.int8)
    prm = sph.params(active_bin=0)
    poison = _poisoned_outputs(f, 10)
    a = Offload(f, layout=2, params=prm)
    b = Offload(f, layout=2, params=prm)
    for o in (a, b):
        o.batch(max_target_cells=29)
        o.import_fields(poison, tuple(poison))
    for loop in range(3):
        sph.sph_init(a.store, loop, prm, a.stream)
        for k in range(a.binfo["nbundles"]):
            sph.sph_batch_pack(a.store, a.bplan, loop, k, a.bbuf_in.data_ptr(), prm, a.stream)
            sph.sph_batch_interact(a.bplan, loop, k, a.bbuf_in.data_ptr(),
                                   a.bbuf_out.data_ptr(), prm, a.stream)
            sph.sph_batch_unpack(a.store, a.bplan, loop, k, a.bbuf_out.data_ptr(),
                                 a.bbuf_in.data_ptr(), a.stream)
        sph.sph_ghost(a.store, loop, prm, a.stream)
    b.batch_step()
    assert np.array_equal(b.store_bytes(), a.store_bytes())


def test_one_call_step_rejects_misuse_before_any_work():
    f = ragged(12, 54)
    off = Offload(f, layout=0)
    off.batch()
    off.list_step()
    before = off.store_bytes()
    b, st, lb = off.bplan, off.stream, off.blist_bytes
    with pytest.raises(sph.SphError):          # misaligned result buffer
        sph.sph_batch_offload_step_list(off.store, b, off.bbuf_in.data_ptr(),
                                        off.bbuf_out.data_ptr() + 4, off.blist.data_ptr(), lb,
                                        off.params, st)
    with pytest.raises(sph.SphError):          # list buffer below its fixed tables
        sph.sph_batch_offload_step_list(off.store, b, off.bbuf_in.data_ptr(),
                                        off.bbuf_out.data_ptr(), off.blist.data_ptr(), 512,
                                        off.params, st)
    with pytest.raises(sph.SphError):          # bundle out of range
        sph.sph_batch_list_build_bundle(off.store, b, 1, off.bbuf_in.data_ptr(),
                                        off.blist.data_ptr(), lb, off.params, st)
    with pytest.raises(sph.SphError):          # unknown loop
        sph.sph_batch_unpack_write(off.store, b, 3, 0, off.bbuf_out.data_ptr(),
                                   off.bbuf_in.data_ptr(), off.params, stream=st)
    sph.sph_sync(st)
    assert np.array_equal(off.store_bytes(), before)


def test_list_pool_regrows_after_the_supports_grow():
    """Supports grown by 20% need about 1.7x the list entries: the enqueued
    step reports SPH_ENOMEM at sph_sync, resize() regrows the pool, and the
    next step equals a fresh offload of the same inputs."""
    f = ragged(12, 80)
    off = Offload(f, layout=6)
    off.batch()
    off.list_step()
    sph.sph_sync(off.stream)
    g = {k: v.copy() for k, v in f.items()}
    g["h"] = (f["h"] * 1.2).astype(np.float32)
    off.import_fields(g, ("h",))
    off.list_step()
    with pytest.raises(sph.SphError) as e:
        sph.sph_sync(off.stream)
    assert e.value.status == 2
    off.resize()
    off.list_step()
    got = off.export()
    ref = Offload(g, layout=6)
    ref.batch()
    ref.list_step()
    want = ref.export()
    for k in want:
        np.testing.assert_array_equal(got[k], want[k], err_msg=k)


def test_list_build_path_follows_the_plan_geometry():
    """Four cells per dimension leave too little room for unambiguous images
    relative to an item's first particle, so the build keeps two-float
    separations; eight cells allow the fixed-point path.  Both match the
    oracle."""
    cases = [(ragged(12, 90), False), (ragged(24, 91), True)]
    for f, fixed in cases:
        off = Offload(f, layout=6)
        off.batch()
        assert sph.sph_batch_list_fixed(off.bplan) == fixed
        off.list_step()
        check_physics(f, off.export())


def test_supports_beyond_the_plan_are_reported():
    """A plan holds for the supports it was built from: the density pack
    reports one beyond the cell's limit (grid: the cell edge; tree: the
    leaf's largest support at build time) at the next sph_sync, and a step
    within the limits is unaffected."""
    f = ragged(12, 5)
    grid = Offload(f, layout=6)
    grid.batch()
    grid.list_step()
    sph.sph_sync(grid.stream)
    # 1% larger supports stay below the grid's cell edge: no report (the
    # list pool is sized again for the extra neighbours)
    grid.import_fields({"h": (f["h"] * np.float32(1.01)).astype(np.float32)}, ("h",))
    grid.resize()
    grid.list_step()
    sph.sph_sync(grid.stream)
    big = f["h"].copy()
    big[17] *= np.float32(3.0)                 # beyond the cell edge
    grid.import_fields({"h": big}, ("h",))
    grid.list_step()
    with pytest.raises(sph.SphError, match="rebuild the plan"):
        sph.sph_sync(grid.stream)
    grid.import_fields({"h": f["h"]}, ("h",))
    grid.list_step()
    sph.sph_sync(grid.stream)
    # a tree plan's limit is each leaf's largest support at build time
    tree = Offload(f, layout=6, plan="tree")
    tree.list_step()
    sph.sph_sync(tree.stream)
    tree.import_fields({"h": (f["h"] * np.float32(1.01)).astype(np.float32)}, ("h",))
    tree.list_step()
    with pytest.raises(sph.SphError, match="rebuild the plan"):
        sph.sph_sync(tree.stream)


@pytest.mark.parametrize("case", ["gresho32", "ragged24", "lognormal24"])
def test_fp64_separation_step_matches_the_oracle(case):
    """The precision study's arm with FP64 pair separations (FP32 fields):
    within the oracle bars, and within rounding of the list step."""
    if case == "lognormal24":
        f = ics.lognormal(n_side=24, seed=31)
        off = Offload(f, layout="pack_force_type", plan="tree")
    else:
        f = PARITY_CASES[case]() if case in PARITY_CASES else ragged(24, 8)
        off = Offload(f, layout="pack_force_type")
        off.batch()
    off.list_step_x64()
    got = off.export()
    check_physics(f, got)
    off.list_step()
    ref = off.export()
    for k in ref:
        assert rms_err(got[k], ref[k]) <= 1e-5, k
    with pytest.raises(sph.SphError, match="needs"):
        sph.sph_batch_offload_step_list_x64(off.store, off.bplan, off.bbuf_in.data_ptr(),
                                            off.bbuf_out.data_ptr(), off.blist.data_ptr(),
                                            off.blist_bytes, off.x64.data_ptr(), 256,
                                            off.params, off.stream)


def read_lists(off):
    """The lists of a list buffer: {(item, lane): sorted bundle slots}."""
    b = off.bplan
    NI = off.binfo["items"]
    fixed = sph.sph_batch_list_bytes(b, 0)
    lo, hi = 0, 1
    while sph.sph_batch_list_bytes(b, hi) <= off.blist_bytes:
        hi *= 2
    while hi - lo > 1:                      # the pool: the most chunks that fit
        mid = (lo + hi) // 2
        if sph.sph_batch_list_bytes(b, mid) <= off.blist_bytes:
            lo = mid
        else:
            hi = mid
    pool = lo
    r256 = lambda x: (x + 255) // 256 * 256
    torch.cuda.synchronize()
    buf = off.blist.cpu().numpy()
    u32 = lambda off_b, n: buf[off_b:off_b + 4 * n].view(np.uint32)
    first = u32(256, NI)
    lcount = u32(256 + r256(4 * NI), 32 * NI).reshape(NI, 32)
    nxt = u32(fixed, pool)
    ents = u32(fixed + r256(4 * pool), pool * 2048)
    out = {}
    for it in range(NI):
        chain, c = [], int(first[it])
        for _ in range((int(lcount[it].max()) + 63) // 64):
            chain.append(c)
            c = int(nxt[c])
        for lane in range(32):
            n = int(lcount[it, lane])
            if n:
                out[(it, lane)] = sorted(int(ents[chain[k // 64] * 2048 + (k % 64) * 32 + lane])
                                         for k in range(n))
    return out


@pytest.mark.parametrize("case", ["ragged24", "gresho32"])
def test_symmetric_list_build_holds_the_same_pairs(case):
    """Testing each cell pair once (a first pass over the forward cells with
    stored hit masks, a second pass transposing them) gives every particle
    the same pairs as testing all neighbour cells per item."""
    f = ragged(24, 8) if case == "ragged24" else PARITY_CASES[case]()
    off = Offload(f, layout="pack_force_type")
    off.batch()
    assert sph.sph_batch_list_symmetric(off.bplan)
    off.list_step()
    sym = read_lists(off)
    got_sym = off.export()
    check_physics(f, got_sym)
    assert not sph.sph_batch_list_symmetric(off.bplan, 0)
    off.list_step()
    one = read_lists(off)
    got_one = off.export()
    assert sym.keys() == one.keys() and len(sym) > 0
    for key in one:
        assert sym[key] == one[key], key
    for k in got_one:       # the same pairs summed in another order (the bar of
        # the other order-changing comparisons: 1e-5 of rms, for the cancelling sums)
        assert rms_err(got_sym[k], got_one[k]) <= 1e-5, k
    # the counting variant counts the same entries either way
    cnt = {}
    for on in (1, 0):
        sph.sph_batch_list_symmetric(off.bplan, on)
        c = torch.zeros(5, dtype=torch.int64, device="cuda")
        sph.sph_batch_pack_list(off.store, off.bplan, 0, 0, off.bbuf_in.data_ptr(), off.params,
                                off.stream)
        sph.sph_batch_list_count(off.store, off.bplan, 0, off.bbuf_in.data_ptr(),
                                 off.blist.data_ptr(), off.blist_bytes, off.params, c.data_ptr(),
                                 off.stream)
        sph.sph_sync(off.stream)
        cnt[on] = c.cpu().tolist()
    assert cnt[1][4] == cnt[0][4] == sum(len(v) for v in one.values())
    assert cnt[1][1] < 0.7 * cnt[0][1]      # roughly half the prefiltered pairs
