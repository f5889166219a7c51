"""Pins against values the paper prints: Table 1 (Sec. 2.1) lists the data
type of particle variables and which of them the pack and unpack of each
interaction loop use.  The oracle is checked by behaviour, not by reading its
tables: a variable counts as packed by a loop when changing it changes that
loop's pack buffer, and as unpacked when the loop's unpack changes it."""
import os

import numpy as np
import pytest

import oracle
from paper_2606_23891_b300 import ics
from paper_2606_23891_b300.pipeline import field_spec

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_particle_data.txt")
TYPES = {"double": np.float64, "float": np.float32, "int8": np.int8}


def table1():
    rows = []
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].split()
        if line:
            name, typ, count, *marks = line
            rows.append((name, TYPES[typ], int(count), [m == "1" for m in marks]))
    return rows


def system(seed=2):
    f = ics.perturb(ics.uniform_lattice(n_side=12, jitter=0.3, seed=seed), seed=seed + 1,
                    v_amp=0.3, u_amp=0.3, alpha_diff=0.4, h_amp=0.05)
    rng = np.random.Generator(np.random.PCG64(seed + 2))
    for k, v in f.items():
        if k in ("x", "h", "id"):
            continue
        if v.dtype == np.float32:
            f[k] = (v + rng.uniform(0.5, 1.5, v.shape)).astype(np.float32)
    f["time_bin"][:] = rng.integers(0, 3, f["time_bin"].shape).astype(np.int8)
    nc, perm, cs = oracle.grid(f)
    ci, cj, sh = oracle.tasks(nc, cs)
    return f, perm, cs, ci, cj, sh


def perturbed(f, name):
    g = {k: v.copy() for k, v in f.items()}
    if name == "x":
        g["x"] = g["x"] + 1e-7          # within every cell, the task list still holds
    elif g[name].dtype == np.int8:
        g[name] = (g[name] + 1).astype(np.int8)
    else:
        g[name] = (g[name] * 1.5 + 0.25).astype(g[name].dtype)
    return g


def test_the_table_is_read_completely():
    rows = table1()
    assert [r[0] for r in rows] == ["x", "v", "a", "mass", "h", "u", "u_dt", "rho", "time_bin"]
    assert all(len(r[3]) == 6 for r in rows)


@pytest.mark.parametrize("row", table1(), ids=lambda r: r[0])
def test_data_types_and_counts(row):
    name, dt, count, _ = row
    assert ics.FIELD_DTYPES[name] == (dt, count)
    assert field_spec(name) == (np.dtype(dt), count)


@pytest.mark.parametrize("loop", [0, 1, 2], ids=["density", "gradient", "force"])
def test_pack_uses_the_marked_variables(loop):
    f, perm, cs, ci, cj, sh = system()
    t1 = len(ci)
    base = oracle.pack(loop, f, perm, cs, ci, cj, sh, 0, t1)
    for name, _, _, marks in table1():
        got = oracle.pack(loop, perturbed(f, name), perm, cs, ci, cj, sh, 0, t1)
        assert (not np.array_equal(got, base)) == marks[2 * loop], (name, loop)


@pytest.mark.parametrize("loop", [0, 1, 2], ids=["density", "gradient", "force"])
def test_unpack_writes_the_marked_variables(loop):
    f, perm, cs, ci, cj, sh = system(seed=5)
    t1 = len(ci)
    S = oracle.bundle_slots(ci, cj, cs, 0, t1)
    rng = np.random.Generator(np.random.PCG64(9 + loop))
    lanes = rng.uniform(0.5, 2.0, oracle.buffer_bytes(loop, 1, S) // 4).astype(np.float32)
    g = {k: v.copy() for k, v in f.items()}
    oracle.unpack(loop, g, perm, cs, ci, cj, 0, t1, lanes.view(np.uint8))
    for name, _, _, marks in table1():
        assert (not np.array_equal(g[name], f[name])) == marks[2 * loop + 1], (name, loop)


# ------------------------------------------------------------ layouts --
# The paper's layout rules (Sec. 3, "Particle Memory Layouts"), checked on
# the oracle's layout descriptors with Table 1's marks: pack-gradient puts
# every variable the gradient pack uses into one struct, pack-force every
# variable the force pack uses; the *-type variants split each struct so that
# every substruct holds one data type; AoS is one struct, SoA one array per
# component.
def groups_of(layout):
    names = oracle.FIELD_NAMES
    return [{names[fid] for fid, _, _ in members} for _, members in oracle.layout_groups(layout)]


def marked(col):
    return {name for name, _, _, m in table1() if m[col]}


@pytest.mark.parametrize("layout, col", [("pack_grad", 2), ("pack_force", 4)])
def test_kernel_driven_layouts_keep_their_pack_together(layout, col):
    gs = groups_of(oracle.LAYOUTS.index(layout))
    want = marked(col)
    home = [g for g in gs if want & g]
    assert len(home) == 1 and want <= home[0], (layout, want, gs)
    others = {name for name, _, _, _ in table1()} - want
    assert not (others & home[0]), (layout, others & home[0])


@pytest.mark.parametrize("layout", ["pack_grad_type", "pack_force_type", "pack_shared_type"])
def test_type_split_layouts_hold_one_type_per_struct(layout):
    for g in groups_of(oracle.LAYOUTS.index(layout)):
        types = {np.dtype(ics.FIELD_DTYPES[name][0]) for name in g if name in ics.FIELD_DTYPES}
        assert len(types) <= 1, (layout, g)


@pytest.mark.parametrize("base, split", [("pack_grad", "pack_grad_type"),
                                         ("pack_force", "pack_force_type"),
                                         ("pack_shared", "pack_shared_type")])
def test_type_split_refines_its_baseline(base, split):
    """Each type-split struct lies inside one struct of its baseline."""
    gb = groups_of(oracle.LAYOUTS.index(base))
    for g in groups_of(oracle.LAYOUTS.index(split)):
        assert any(g <= b for b in gb), (split, g)


def test_aos_is_one_struct_and_soa_one_array_per_component():
    aos = oracle.layout_groups(oracle.LAYOUTS.index("aos"))
    assert len(aos) == 1
    soa = oracle.layout_groups(oracle.LAYOUTS.index("soa"))
    assert all(len(members) == 1 for _, members in soa)
