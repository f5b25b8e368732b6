"""Pins of the oracle's octree and interaction lists.

The FMM needs (Section 2.4, Eq. nearfar and the recursive far field) that
every (target, source) pair be accounted for exactly once: directly through
a U-list pair of their leaves, or through exactly one V, W or X pair between
an ancestor-or-self of the target's leaf and an ancestor-or-self of the
source's leaf.  These tests check that property by brute force over all point
pairs, plus the leaf-capacity rule and the uniform-tree counts (27 near and
189 well-separated boxes around an interior box).
"""
import numpy as np
import pytest

import oracle
import sph_inputs as si


def _leaf_of(tree, n_src, n_trg):
    """leaf box index of each Morton-sorted source / target point."""
    sl = np.full(n_src, -1)
    tl = np.full(n_trg, -1)
    for b in np.flatnonzero(tree["leaf"]):
        sl[tree["src_begin"][b]:tree["src_end"][b]] = b
        tl[tree["trg_begin"][b]:tree["trg_end"][b]] = b
    return sl, tl


def _ancestors(tree, b):
    out = []
    while b >= 0:
        out.append(b)
        b = tree["parent"][b]
    return out


def _coverage(tree, nJ, nT):
    sl, tl = _leaf_of(tree, nJ, nT)
    nb = len(tree["level"])
    cnt = np.zeros((nT, nJ), np.int32)
    # box membership matrices (points x boxes)
    S_in = np.zeros((nJ, nb), bool)
    T_in = np.zeros((nT, nb), bool)
    for b in range(nb):
        S_in[tree["src_begin"][b]:tree["src_end"][b], b] = True
        T_in[tree["trg_begin"][b]:tree["trg_end"][b], b] = True
    for name in ("U", "V", "W", "X"):
        for (bt, bs) in tree[name]:
            ti = np.flatnonzero(T_in[:, bt])
            sj = np.flatnonzero(S_in[:, bs])
            if name == "U" or name == "W":
                ti = ti[tl[ti] == bt]          # bt must be the target's own leaf
            if name == "U" or name == "X":
                sj = sj[sl[sj] == bs]          # bs must be the source's own leaf
            cnt[np.ix_(ti, sj)] += 1
    return cnt


CASES = [
    # (nx, ny, nz, source fraction, target fraction, leaf size, seed)
    (8, 8, 8, 1.0, 1.0, 8, 1),
    (16, 16, 16, 0.05, 0.3, 8, 2),
    (12, 9, 7, 0.2, 0.1, 4, 3),
    (16, 16, 16, 0.02, 1.0, 16, 4),
    (20, 10, 13, 0.5, 0.02, 6, 5),
]


@pytest.mark.parametrize("case", CASES)
def test_every_pair_covered_exactly_once(case):
    nx, ny, nz, fs, ft, S, seed = case
    n = nx * ny * nz
    J = np.flatnonzero(si.uniform01(seed, n) < fs).astype(np.int32)
    T = np.flatnonzero(si.uniform01(seed + 100, n) < ft).astype(np.int32)
    tree = oracle.octree(nx, ny, nz, J, T, S)
    cnt = _coverage(tree, J.size, T.size)
    assert cnt.min() == 1 and cnt.max() == 1


def test_clustered_sources_make_w_and_x_lists():
    """A dense source clump next to sparse targets gives W and X pairs; still exactly once."""
    nx = ny = nz = 16
    X, Y, Z = si._grid(nx, ny, nz, 1.0)
    r2 = (X - 4) ** 2 + (Y - 4) ** 2 + (Z - 4) ** 2
    J = np.flatnonzero(r2.ravel() < 9).astype(np.int32)
    T = np.flatnonzero((si.uniform01(9, nx * ny * nz) < 0.08) | (r2.ravel() > 60)).astype(np.int32)
    T = T[::3]
    tree = oracle.octree(nx, ny, nz, J, T, 4)
    assert len(tree["W"]) > 0 and len(tree["X"]) > 0
    cnt = _coverage(tree, J.size, T.size)
    assert cnt.min() == 1 and cnt.max() == 1


@pytest.mark.parametrize("case", CASES)
def test_leaf_capacity_and_ranges(case):
    nx, ny, nz, fs, ft, S, seed = case
    n = nx * ny * nz
    J = np.flatnonzero(si.uniform01(seed, n) < fs).astype(np.int32)
    T = np.flatnonzero(si.uniform01(seed + 100, n) < ft).astype(np.int32)
    tr = oracle.octree(nx, ny, nz, J, T, S)
    D = tr["depth"]
    ns = tr["src_end"] - tr["src_begin"]
    nt = tr["trg_end"] - tr["trg_begin"]
    leaf = tr["leaf"]
    assert np.all((ns[leaf] <= S) & (nt[leaf] <= S) | (tr["level"][leaf] == D))
    assert np.all((ns[~leaf] > S) | (nt[~leaf] > S))
    assert np.all(ns + nt > 0)
    # children partition the parent's ranges
    for b in np.flatnonzero(~leaf):
        kids = np.flatnonzero(tr["parent"] == b)
        assert ns[kids].sum() == ns[b] and nt[kids].sum() == nt[b]
        assert tr["src_begin"][kids].min() == tr["src_begin"][b]
    # ordering: (level, key) ascending
    lk = tr["level"] * (1 << 40) + tr["key"]
    assert np.all(np.diff(lk) > 0)
    # leaves' point ranges tile [0, nJ) and [0, nT)
    assert ns[leaf].sum() == J.size and nt[leaf].sum() == T.size


def test_uniform_tree_counts():
    """Full 16^3 grid, leaf size 8: leaves are the 8^3 boxes of 2^3 cells; an interior
    leaf has 27 near boxes, and an interior box at level >= 3 has 189 V boxes (6^3 - 3^3)."""
    n = 16
    J = np.arange(n ** 3, dtype=np.int32)
    tr = oracle.octree(n, n, n, J, J, 8)
    lev = tr["level"]
    assert np.sum(tr["leaf"]) == 512 and np.all(lev[tr["leaf"]] == 3)
    U = tr["U"]
    V = tr["V"]
    nu = np.bincount(U[:, 0], minlength=len(lev))
    nv = np.bincount(V[:, 0], minlength=len(lev))

    def coords(b):
        k = int(tr["key"][b])
        i = j = z = 0
        for bit in range(tr["depth"]):
            i |= ((k >> (3 * bit)) & 1) << bit
            j |= ((k >> (3 * bit + 1)) & 1) << bit
            z |= ((k >> (3 * bit + 2)) & 1) << bit
        return i, j, z

    for b in np.flatnonzero(lev == 3):
        c = coords(b)
        if all(1 <= x <= 6 for x in c):
            assert nu[b] == 27
        if all(2 <= x <= 5 for x in c):
            assert nv[b] == 189
    assert len(tr["W"]) == 0 and len(tr["X"]) == 0
