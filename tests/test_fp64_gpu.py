"""The all-FP64 variant of the batched cycle (precision study) against the
oracle.  Every arithmetic step runs in FP64 and each result is rounded to the
FP32 store once, so what remains against the FP64 oracle is the storage of
values in FP32 between the loops:

  rho, wcount, pressure, soundspeed, v_sig_grad, v_sig : rel <= 2.5e-7
      (at most two FP32 roundings, 2 * 2^-24, with a margin for the FP64
      summation order)
  f_gradh, balsara, rho_dh, wcount_dh : <= 1e-6 on the scales of the
      mixed-precision bars (one rounding of a cancelling sum)
  div_v, rot_v, laplace_u, a, u_dt, h_dt : err / rms <= 1e-5 (their inputs
      rho, f_gradh, balsara are FP32 store values, each term perturbed by
      ~2^-24 relative and the sums cancel)

The same outputs must also agree with the mixed-precision path within the
mixed-precision bars, and be at least as close to the oracle as it is on the
positive sums."""
import numpy as np
import pytest

import oracle
from oracle import compare
from paper_2606_23891_b300 import ics, sph

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2606_23891_b300.pipeline import Offload  # noqa: E402
from test_parity_gpu import PARITY_CASES, check_physics  # noqa: E402

TIGHT = ("rho", "wcount", "pressure", "soundspeed", "v_sig_grad", "v_sig")
MID = ("f_gradh", "balsara", "rho_dh", "wcount_dh")
LOOSE = ("div_v", "rot_v", "laplace_u", "a", "u_dt", "h_dt")


def fp64_bars(err):
    for k in TIGHT:
        assert err[k] <= 2.5e-7, (k, err[k])
    for k in MID:
        assert err[k] <= 1e-6, (k, err[k])
    for k in LOOSE:
        assert err[k] <= 1e-5, (k, err[k])


@pytest.mark.parametrize("mtc", [0, 29])
@pytest.mark.parametrize("case", sorted(PARITY_CASES))
def test_fp64_pass_matches_the_oracle(case, mtc):
    f = PARITY_CASES[case]()
    off = Offload(f, layout="pack_force_type")
    off.batch(max_target_cells=mtc)
    off.fp64_step()
    got64 = off.export()
    ref = oracle.chain(f, oracle.params())
    sc = oracle.dh_scales(f, oracle.params())
    e64 = compare.errors(got64, ref, sc)
    fp64_bars(e64)
    check_physics(f, got64)
    # the mixed path on the same plan: never closer on the positive sums
    off.batch_step()
    e32 = compare.errors(off.export(), ref, sc)
    for k in ("rho", "wcount", "pressure"):
        assert e64[k] <= max(e32[k], 2.5e-7), (k, e64[k], e32[k])


def test_fp64_inactive_particles_and_large_cells():
    rng = np.random.Generator(np.random.PCG64(78))
    n_bg, n_cl = 1500, 2600
    n = n_bg + n_cl
    f = ics.empty_fields(n)
    x = rng.uniform(0, 1, (n, 3))
    x[n_bg:] = 0.3 + rng.uniform(0, 0.05, (n_cl, 3))
    f["x"][:] = x
    f["v"][:] = rng.uniform(-0.5, 0.5, (n, 3)).astype(np.float32)
    f["mass"][:] = np.float32(1.0 / n)
    f["h"][:] = np.float32(0.1)
    f["h"][n_bg:] = np.float32(0.012)
    f["u"][:] = rng.uniform(0.5, 1.5, n).astype(np.float32)
    f["alpha_visc"][:] = 0.5
    f["alpha_diff"][:] = 0.2
    f["time_bin"][::5] = 4
    off = Offload(f, layout=5, params=sph.params(active_bin=2))
    off.batch(threads=128)
    pre = {"a": np.full((n, 3), 7.0, np.float32), "u_dt": np.full(n, 7.0, np.float32),
           "h_dt": np.full(n, 7.0, np.float32), "v_sig": np.full(n, 7.0, np.float32)}
    off.import_fields(pre, tuple(pre))
    off.fp64_step()
    got = off.export()
    inactive = f["time_bin"] > 2
    assert np.all(got["a"][inactive] == 7.0)
    assert np.all(got["v_sig"][inactive] == 7.0)
    sel = np.nonzero(~inactive)[0]
    ref = oracle.chain(f, oracle.params(active_bin=2), sel)
    sc = oracle.dh_scales(f, oracle.params(active_bin=2), sel)
    fp64_bars(compare.errors({k: v[sel] for k, v in got.items()}, ref, sc))


def test_fp64_steps_are_reproducible():
    f = PARITY_CASES["ragged12"]()
    off = Offload(f, layout=0)
    off.batch(max_target_cells=50)
    off.fp64_step()
    a = off.export()
    off.fp64_step()
    b = off.export()
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


def test_fp64_api_rejects_misuse():
    f = PARITY_CASES["ragged12"]()
    off = Offload(f, layout=0)
    off.batch()
    n_in = sph.sph_batch_buffer_bytes_fp64(off.bplan, 0)
    n_out = sph.sph_batch_buffer_bytes_fp64(off.bplan, 1)
    assert n_in > 0 and n_out > 0 and n_in % 256 == 0 and n_out % 256 == 0
    assert sph.sph_batch_buffer_bytes_fp64(off.bplan, 2) == 0
    buf = torch.empty(n_in + n_out + 512, dtype=torch.uint8, device=off.device)
    with pytest.raises(sph.SphError):   # misaligned input buffer
        sph.sph_batch_offload_loop_fp64(off.store, off.bplan, 0, buf.data_ptr() + 16,
                                        buf.data_ptr(), off.params, off.stream)
    with pytest.raises(sph.SphError):   # unknown loop
        sph.sph_batch_offload_loop_fp64(off.store, off.bplan, 3, buf.data_ptr(),
                                        buf.data_ptr() + n_in, off.params, off.stream)
