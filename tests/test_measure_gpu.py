"""The measurement calls: the arithmetic-peak microbenchmark, the host-staged
cycle with every stage timed, and the counting variant of the list build.
Each must leave the results of the path it measures unchanged."""
import numpy as np
import pytest

from paper_2606_23891_b300 import sph

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2606_23891_b300.pipeline import HostOffload, Offload  # noqa: E402
from test_parity_gpu import PARITY_CASES, ragged  # noqa: E402


def test_peak_microbenchmark_counts_its_flops():
    sink = torch.zeros(256, dtype=torch.uint8, device="cuda")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    rates = {}
    for kind in (sph.PEAK_FP32_FMA, sph.PEAK_FP64_FMA, sph.PEAK_FP64_ADD):
        iters = 512
        # one untimed run first: the first launch of a kernel also pays its load
        sph.sph_peak_run(kind, iters, sink.data_ptr(), torch.cuda.current_stream().cuda_stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fl = sph.sph_peak_run(kind, iters, sink.data_ptr(), torch.cuda.current_stream().cuda_stream)
        e1.record()
        torch.cuda.synchronize()
        per_op = 1 if kind == sph.PEAK_FP64_ADD else 2
        assert fl == 8 * sms * 256 * iters * 16 * 8 * per_op
        rates[kind] = fl / (e0.elapsed_time(e1) * 1e-3)
    assert rates[sph.PEAK_FP32_FMA] > rates[sph.PEAK_FP64_FMA]
    sph.sph_sync(0)


@pytest.mark.parametrize("layout", [0, 6])
def test_timed_host_staged_loop_matches_the_untimed_one(layout):
    f = ragged(24, 8)
    a = HostOffload(f, layout=layout, bundle_max_slots=40000)
    b = HostOffload(f, layout=layout, bundle_max_slots=40000)
    a.step()
    stats = b.step_stats()
    np.testing.assert_array_equal(a.store_bytes(), b.store_bytes())
    for loop, st in enumerate(stats):
        nb = a.info["nbundles"]
        bs = a.task_list()[4]
        assert st["bundles"] == nb > 4
        want_in = sum(_lane_bytes(a, loop, 0, k) for k in range(nb))
        want_out = sum(_lane_bytes(a, loop, 1, k) for k in range(nb))
        assert st["h2d_bytes"] == want_in and st["d2h_bytes"] == want_out
        assert st["h2d_ms"] > 0 and st["kernel_ms"] > 0 and st["d2h_ms"] > 0
        assert st["host_pack_s"] > 0 and st["host_unpack_s"] > 0
        assert st["wall_s"] >= st["host_pack_s"]
        assert len(bs) == nb + 1


def _lane_bytes(host, loop, in_or_out, bundle):
    """Bytes of one bundle's pack or result buffer (the oracle's lane
    format: every lane starts on a 256-byte boundary)."""
    import oracle
    ci, cj, sh, cs, bs = host.task_list()
    S = oracle.bundle_slots(ci, cj, cs, int(bs[bundle]), int(bs[bundle + 1]))
    return oracle.buffer_bytes(loop, in_or_out, S)


@pytest.mark.parametrize("case", ["gresho32", "ragged24"])
def test_counting_list_build_counts_and_leaves_results_alone(case):
    f = PARITY_CASES[case]()
    off = Offload(f, layout="pack_force_type")
    off.batch()
    off.list_step()
    want = off.export()
    cnt = torch.zeros(5, dtype=torch.int64, device="cuda")
    for b in range(off.binfo["nbundles"]):
        sph.sph_batch_pack_list(off.store, off.bplan, 0, b, off.bbuf_in.data_ptr(), off.params,
                                off.stream)
        sph.sph_batch_list_count(off.store, off.bplan, b, off.bbuf_in.data_ptr(),
                                 off.blist.data_ptr(), off.blist_bytes, off.params,
                                 cnt.data_ptr(), off.stream)
    sph.sph_sync(off.stream)
    staged, culled, hits, exact, entries = cnt.cpu().tolist()
    # the lists the counting build wrote drive the same loops to the same bits
    for loop in range(3):
        off.list_loop(loop)
    got = off.export()
    for k in want:
        np.testing.assert_array_equal(got[k], want[k], err_msg=k)
    # entries = the force loop's pair interactions (the list holds every j
    # with r < max(H_i, H_j)); the counts nest.  The symmetric build tests
    # each cell pair once, so its hits are fewer than the entries (each
    # neighbour-cell hit gives two), never fewer than half
    pf = off.count_pairs(2)
    assert abs(entries - pf) <= max(2, 1e-6 * pf)
    assert culled >= hits >= exact
    if sph.sph_batch_list_symmetric(off.bplan):
        assert hits <= entries <= 2 * hits
    else:
        assert hits == entries
    n = off.n
    assert staged >= n and culled <= 27 * 80 * n
