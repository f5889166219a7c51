"""Host logic of the octree-leaf plan (no GPU): leaf ranges, Morton order,
and completeness of the neighbour entries against a brute-force pair search
(scipy's periodic KD-tree, an independent library routine)."""
import numpy as np
import pytest

from paper_2606_23891_b300 import ics, sph

KG = 1.825742


def morton(x, box=1.0, bits=21):
    """Interleaved 21-bit keys (x in the lowest bit of each triple)."""
    q = np.clip(np.floor(np.asarray(x) / box * (1 << bits)), 0, (1 << bits) - 1).astype(np.uint64)
    key = np.zeros(q.shape[0], np.uint64)
    for b in range(bits):
        for d in range(3):
            key |= ((q[:, d] >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b + d)
    return key


def plan(f, leaf_max, rule=0):
    return sph.sph_tree_plan(f["x"], f["h"], leaf_max=leaf_max, rule=rule)


def entries(nb):
    return nb >> 6, nb & 63


CASES = {
    "lognormal24": lambda: ics.lognormal(n_side=24, seed=5),
    "lognormal32": lambda: ics.lognormal(n_side=32, seed=6),
    "lattice12": lambda: ics.perturb(ics.uniform_lattice(n_side=12, jitter=0.45, seed=2),
                                     seed=3, h_amp=0.3),
}


@pytest.mark.parametrize("leaf_max", [8, 64, 300])
@pytest.mark.parametrize("case", sorted(CASES))
def test_leaves_partition_the_particles_in_morton_order(case, leaf_max):
    f = CASES[case]()
    n = f["x"].shape[0]
    perm, ls, nbs, nb = plan(f, leaf_max)
    assert np.array_equal(np.sort(perm), np.arange(n))
    k = morton(f["x"][perm])
    assert np.all(np.diff(k.astype(np.float64)) >= 0)
    ties = np.nonzero(k[1:] == k[:-1])[0]
    assert np.all(perm[ties] < perm[ties + 1])          # index tie-break
    assert ls[0] == 0 and ls[-1] == n and np.all(np.diff(ls) > 0)
    assert np.all(np.diff(ls) <= leaf_max)
    assert nbs[0] == 0 and nbs[-1] == nb.size and np.all(np.diff(nbs) >= 1)


@pytest.mark.parametrize("leaf_max,rule", [(8, 0), (64, 0), (8, 1)])
@pytest.mark.parametrize("case", sorted(CASES))
def test_neighbour_entries_cover_every_interacting_pair(case, leaf_max, rule):
    """Every pair with r < max(H_i, H_j) (minimum image) must find j's leaf,
    with the shift that brings j's image next to i, among i's leaf entries;
    no entry repeats."""
    from scipy.spatial import cKDTree
    f = CASES[case]()
    x = np.asarray(f["x"], np.float64)
    H = (np.float32(KG) * f["h"]).astype(np.float64)
    perm, ls, nbs, nb = plan(f, leaf_max, rule)
    n = x.shape[0]
    leaf_of = np.empty(n, np.int64)                       # by original index
    leaf_of[perm] = np.repeat(np.arange(ls.size - 1), np.diff(ls))
    cell, code = entries(nb)
    owner = np.repeat(np.arange(ls.size - 1), np.diff(nbs))
    L = ls.size - 1
    have = (owner * L + cell) * 64 + code
    assert np.unique(have).size == have.size              # no entry repeats
    assert np.isin((np.arange(L) * L + np.arange(L)) * 64 + 21, have).all()  # self, unshifted
    # ordered pairs with r < H_i, then the reversed ones (r < H_j)
    tree = cKDTree(x, boxsize=1.0)
    lists = tree.query_ball_point(x, H)
    i = np.repeat(np.arange(n), [len(v) for v in lists])
    j = np.concatenate([np.asarray(v, np.int64) for v in lists])
    i, j = np.concatenate([i, j]), np.concatenate([j, i])
    keep = i != j
    i, j = i[keep], j[keep]
    d = x[i] - x[j]
    s = -np.rint(d)                                       # image shift of j
    r = np.sqrt(((d - s) ** 2).sum(axis=1))
    keep = r < np.maximum(H[i], H[j])
    i, j, s = i[keep], j[keep], s[keep].astype(np.int64)
    assert i.size > 0
    codes = (s[:, 0] + 1) | ((s[:, 1] + 1) << 2) | ((s[:, 2] + 1) << 4)
    need = (leaf_of[i] * L + leaf_of[j]) * 64 + codes
    ok = np.isin(need, have)
    assert ok.all(), (i[~ok][:5], j[~ok][:5])


@pytest.mark.parametrize("case", ["lognormal24", "lattice12"])
def test_octree_rule_leaves(case):
    """Rule 1 (the cell tree's rule): a leaf is split no further once half its
    edge is below the largest support inside it; leaves hold up to thousands."""
    f = CASES[case]()
    H = np.float32(KG) * f["h"]
    perm, ls, nbs, nb = plan(f, 8, rule=1)
    perm0, ls0, _, _ = plan(f, 8, rule=0)
    assert np.array_equal(perm, perm0)                   # same Morton order
    k = morton(f["x"][perm])
    cnt = np.diff(ls)
    assert cnt.max() > 8 or case == "lattice12"
    for l in range(cnt.size):
        if cnt[l] <= 8:
            continue
        kk = k[ls[l]:ls[l + 1]]
        # the leaf's level: the longest common Morton prefix of its keys
        x = int(kk[0]) ^ int(kk[-1])
        level = 21 - (x.bit_length() + 2) // 3
        hmax = float(H[perm[ls[l]:ls[l + 1]]].max())
        assert 1.0 / (2 << level) < hmax or level == 21, (l, level, hmax)


def test_tree_plan_rejects_bad_input():
    f = ics.lognormal(n_side=12, seed=1)
    with pytest.raises(sph.SphError):
        sph.sph_tree_plan(f["x"], f["h"], leaf_max=4)
    with pytest.raises(sph.SphError):
        sph.sph_tree_plan(f["x"], f["h"], leaf_max=4096)
    big = f["h"].copy()
    big[3] = 0.3                                          # support above half the box
    with pytest.raises(sph.SphError):
        sph.sph_tree_plan(f["x"], big)
    bad = f["h"].copy()
    bad[0] = 0.0
    with pytest.raises(sph.SphError):
        sph.sph_tree_plan(f["x"], bad)


def test_tree_plan_of_no_particles():
    perm, ls, nbs, nb = sph.sph_tree_plan(np.zeros((0, 3)), np.zeros(0, np.float32))
    assert perm.size == 0 and ls.tolist() == [0] and nb.size == 0
