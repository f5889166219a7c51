"""The allocation-free offload entry point (sph_offload_loop_noalloc).

Some callers cannot allocate device memory while they run, for example an
application whose device memory is all reserved by its own pool allocator.
For them the library runs the offload cycle with a fixed scratch array of its
own.  This test calls that entry point through the C-ABI twice in a row and
checks that each call gives the same store contents as the ordinary entry
point with caller buffers.  It lives in its own file, collected last, and
needs no state from other tests.
"""
import numpy as np
import pytest

from paper_2606_23891_b300 import ics, sph

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2606_23891_b300.pipeline import OUTPUTS, Offload  # noqa: E402


def _inputs():
    f = ics.perturb(ics.uniform_lattice(n_side=24, jitter=0.45, seed=8), seed=9,
                    v_amp=0.3, u_amp=0.3, alpha_diff=0.5, h_amp=0.1)
    rng = np.random.Generator(np.random.PCG64(10))
    f["alpha_visc"][:] = rng.uniform(0.1, 1.5, f["alpha_visc"].shape).astype(np.float32)
    return f


def _rms_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    s = np.sqrt(np.mean(b * b))
    return np.max(np.abs(a - b)) / s if s > 0 else np.max(np.abs(a - b))


def test_noalloc_entry_point_matches_the_buffered_one_twice():
    assert torch.cuda.is_available(), "needs a CUDA device"
    f = _inputs()
    ref = Offload(f, layout="pack_force_type", bundle_max_slots=100000)
    assert ref.nbundles() > 1
    ref.step()
    want = ref.export(OUTPUTS)
    # same particles and tasks, a fresh store, the library's own scratch
    off = Offload(f, layout="pack_force_type", share=ref)
    torch.cuda.synchronize()
    for call in range(2):
        # the library's next device allocation of its own would fail (host-side
        # injector): the calls must not need one; torch allocates nothing either
        before = torch.cuda.memory_allocated()
        sph.sph_fault_inject(sph.SPH_FAULT_DEVICE_ALLOC, 1)
        try:
            for loop in (sph.SPH_DENSITY, sph.SPH_GRADIENT, sph.SPH_FORCE):
                sph.sph_offload_loop_noalloc(off.store, off.tasks, loop, off.params,
                                             off.stream)
            sph.sph_sync(off.stream)
        finally:
            sph.sph_fault_inject(sph.SPH_FAULT_NONE, 0)
        assert torch.cuda.memory_allocated() == before
        got = off.export(OUTPUTS)
        for k in OUTPUTS:
            # same kernels, same bundles, same order: identical; the bar used
            # by the physics tests (1e-5 of rms) is checked as well
            assert _rms_err(got[k], want[k]) <= 1e-5, (call, k)
            np.testing.assert_array_equal(got[k], want[k], err_msg="call %d %s" % (call, k))


def test_noalloc_rejects_bundles_larger_than_its_scratch():
    f = _inputs()
    big = Offload(f, layout="aos")          # one bundle of all 373k slots
    need = sph.sph_buffer_bytes(big.tasks, sph.SPH_FORCE, 0) + \
        sph.sph_buffer_bytes(big.tasks, sph.SPH_FORCE, 1)
    assert need > sph.SPH_NOALLOC_SCRATCH_BYTES
    with pytest.raises(sph.SphError) as e:
        sph.sph_offload_loop_noalloc(big.store, big.tasks, sph.SPH_FORCE, big.params, 0)
    assert e.value.status == 6 and "scratch" in str(e.value)
