"""Degenerate inputs through the list, batched and per-task cycles, against
the oracle: one particle, a pair that meets only across the periodic
boundary, a particle with no neighbour in its own support inside a wider
one, isolated particles beside a dense clump, and an empty set."""
import numpy as np
import pytest

from paper_2606_23891_b300 import ics

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2606_23891_b300.pipeline import OUTPUTS, Offload  # noqa: E402
from test_parity_gpu import check_physics  # noqa: E402


def fields(x, h, seed=3):
    x = np.asarray(x, np.float64).reshape(-1, 3)
    n = len(x)
    rng = np.random.Generator(np.random.PCG64(seed))
    f = ics.empty_fields(n)
    f["x"][:] = x
    f["h"][:] = h
    f["mass"][:] = 1.0 / max(n, 1)
    f["v"][:] = rng.uniform(-0.2, 0.2, (n, 3)).astype(np.float32)
    f["u"][:] = rng.uniform(0.5, 1.5, n).astype(np.float32)
    f["alpha_visc"][:] = 0.5
    f["alpha_diff"][:] = 0.3
    f["id"][:] = np.arange(n, dtype=np.int64)
    return f


def each_cycle(f):
    """(name, outputs) of the list, batched and per-task cycles on f."""
    off = Offload(f, layout="pack_force_type")
    off.batch()
    off.list_step()
    yield "list", off.export()
    off.batch_step()
    yield "batched", off.export()
    off.step()
    yield "per-task", off.export()


def test_one_particle_has_only_its_self_terms():
    f = fields([0.5, 0.5, 0.5], 0.05)
    for name, got in each_cycle(f):
        ref, _, _ = check_physics(f, got)
        assert np.all(got["a"] == 0.0) and np.all(got["u_dt"] == 0.0), name
        assert got["rho"][0] > 0.0, name


def test_a_pair_meets_across_the_periodic_boundary():
    f = fields([[0.001, 0.5, 0.5], [0.999, 0.5, 0.5]], [0.01, 0.012])
    for name, got in each_cycle(f):
        ref, _, _ = check_physics(f, got)
        # the two accelerations point along x, equal and opposite in m a
        assert abs(got["a"][0, 0]) > 0.0, name
        assert np.isclose(got["a"][0, 0], -got["a"][1, 0], rtol=1e-4), name


def test_a_lone_particle_inside_a_wider_support():
    """A has no other particle inside its support (f_gradh = 1), B's wider
    support reaches A: the force criterion r < max(H_A, H_B) still pairs
    them, with equal and opposite m a."""
    f = fields([[0.5, 0.5, 0.5], [0.52, 0.5, 0.5]], np.array([0.004, 0.02], np.float32))
    for name, got in each_cycle(f):
        check_physics(f, got)
        assert got["f_gradh"][0] == 1.0, name
        pa = float(f["mass"][0]) * got["a"][0].astype(np.float64)
        pb = float(f["mass"][1]) * got["a"][1].astype(np.float64)
        assert abs(pa[0]) > 0.0, name
        np.testing.assert_allclose(pa, -pb, rtol=1e-4, atol=1e-6 * abs(pa[0]), err_msg=name)


def test_isolated_particles_beside_a_dense_clump():
    rng = np.random.Generator(np.random.PCG64(21))
    d = rng.normal(size=(300, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    clump = 0.5 + 0.05 * d * rng.uniform(0, 1, (300, 1)) ** (1 / 3)
    lone = rng.uniform(0.1, 0.9, (12, 3))
    lone[:, 0] = np.where(lone[:, 0] > 0.5, lone[:, 0] * 0.3 + 0.65, lone[:, 0] * 0.3 + 0.02)
    x = np.concatenate([clump, lone])
    h = np.concatenate([np.full(300, 0.012), np.full(12, 0.004)])
    f = fields(x, h.astype(np.float32), seed=5)
    for name, got in each_cycle(f):
        check_physics(f, got)
        assert np.all(np.isfinite(got["a"])), name


def test_an_empty_set_steps_to_empty_outputs():
    f = fields(np.zeros((0, 3)), np.zeros(0, np.float32))
    for name, got in each_cycle(f):
        for k in OUTPUTS:
            assert got[k].shape[0] == 0, (name, k)
