"""Pins for the oracle's tree, node selection and ring graph (Section 4).

The node set must be the unique minimal refinement of the error-balance tree
in which face-adjacent leaves differ by at most one level (Sections 4.1-4.2).
These tests rebuild that set with an independent fix-point iteration (refine
any leaf that is two levels coarser than a face neighbour until nothing
changes), and check face adjacency by brute force over all leaf pairs.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1603_04039_gb300 import inputs

KD = 21


def _split(key, level):
    x = y = z = 0
    for b in range(level):
        z |= ((key >> (3 * b)) & 1) << b
        y |= ((key >> (3 * b + 1)) & 1) << b
        x |= ((key >> (3 * b + 2)) & 1) << b
    return x, y, z


def _join(x, y, z, level):
    k = 0
    for b in range(level - 1, -1, -1):
        k = (k << 3) | (((x >> b) & 1) << 2) | (((y >> b) & 1) << 1) | ((z >> b) & 1)
    return k


def _sorted_keys(x, y, z):
    u = lambda p: np.clip(np.floor((p + 1.0) * 2.0 ** 20), 0, 2 ** 21 - 1).astype(np.int64)
    ix, iy, iz = u(x), u(y), u(z)
    k = np.zeros(len(x), dtype=np.uint64)
    for b in range(KD - 1, -1, -1):
        k = (k << np.uint64(3)) | (((ix >> b) & 1).astype(np.uint64) << np.uint64(2)) | \
            (((iy >> b) & 1).astype(np.uint64) << np.uint64(1)) | ((iz >> b) & 1).astype(np.uint64)
    return np.sort(k)


def _count(skeys, key, level):
    sh = 3 * (KD - level)
    a = np.uint64(key << sh)
    if level == 0:
        return len(skeys)
    b = np.uint64((key + 1) << sh)
    return int(np.searchsorted(skeys, b) - np.searchsorted(skeys, a))


def _fixpoint_leaves(x, y, z, max_depth, c):
    """Independent construction: criterion tree, then refine until 2:1 face balanced."""
    skeys = _sorted_keys(x, y, z)
    leaves = set()
    stack = [(0, 0)]
    while stack:
        lv, k = stack.pop()
        if oracle.criterion_opens(_count(skeys, k, lv), lv, max_depth, -1.0, 1.0, c):
            stack.extend((lv + 1, (k << 3) | o) for o in range(8))
        else:
            leaves.add((lv, k))

    def containing_leaf(lv, cx, cy, cz):
        for l in range(lv, -1, -1):
            sh = lv - l
            kk = _join(cx >> sh, cy >> sh, cz >> sh, l)
            if (l, kk) in leaves:
                return (l, kk)
        return None

    changed = True
    while changed:
        changed = False
        for (lv, k) in list(leaves):
            if (lv, k) not in leaves:
                continue
            cx, cy, cz = _split(k, lv)
            for d in range(3):
                for s in (-1, 1):
                    p = [cx, cy, cz]
                    p[d] += s
                    if p[d] < 0 or p[d] >= (1 << lv):
                        continue
                    nb = containing_leaf(lv, *p)
                    if nb is not None and nb[0] < lv - 1:
                        leaves.discard(nb)
                        leaves.update((nb[0] + 1, (nb[1] << 3) | o) for o in range(8))
                        changed = True
    return leaves


def _leaf_boxes(o):
    key, first, count = o.leaves()
    lv = o.nodes()["level"][: o.n_int].astype(np.int64)
    lo = np.zeros((o.n_int, 3), dtype=np.int64)
    for j in range(o.n_int):
        cx, cy, cz = _split(int(key[j]), int(lv[j]))
        lo[j] = np.array([cx, cy, cz]) << (KD - lv[j])
    size = (np.int64(1) << (KD - lv))
    return lo, lo + size[:, None], lv, key


@pytest.mark.parametrize("n,depth,c,seed", [(20000, 5, 0.5, 1), (60000, 6, 1.0, 2), (3000, 7, 0.2, 3)])
def test_nodes_are_minimal_balanced_refinement(n, depth, c, seed):
    x, y, z, q = inputs.beam_with_halo(n, seed)
    o = oracle.Oracle(max_depth=depth, c_refine=c)
    o.build(x, y, z)
    key, _, _ = o.leaves()
    lv = o.nodes()["level"][: o.n_int]
    got = {(int(a), int(b)) for a, b in zip(lv, key)}
    want = _fixpoint_leaves(x, y, z, depth, c)
    assert got == want


def test_leaves_partition_domain_in_morton_order():
    x, y, z, q = inputs.beam_with_halo(50000, 4)
    o = oracle.Oracle(max_depth=6, c_refine=0.6)
    o.build(x, y, z)
    lo, hi, lv, key = _leaf_boxes(o)
    anchor = key.astype(np.uint64) << (np.uint64(3) * (np.uint64(KD) - lv.astype(np.uint64)))
    span = np.uint64(1) << (np.uint64(3) * (np.uint64(KD) - lv.astype(np.uint64)))
    assert anchor[0] == 0
    assert np.all(anchor[1:] == anchor[:-1] + span[:-1])           # contiguous, no overlap
    assert int(anchor[-1] + span[-1]) == 1 << 63                  # covers the whole cube
    vol = ((hi - lo).astype(float) / 2.0 ** KD).prod(1).sum()
    assert vol == 1.0


def test_every_leaf_meets_criterion_and_opened_cells_are_needed():
    x, y, z, q = inputs.beam_with_halo(40000, 5)
    depth, c = 6, 0.5
    o = oracle.Oracle(max_depth=depth, c_refine=c)
    o.build(x, y, z)
    key, lv, opened, cnt = o.cells()
    for k, l, op, nn in zip(key, lv, opened, cnt):
        if not op:
            assert not oracle.criterion_opens(int(nn), int(l), depth, -1.0, 1.0, c)


def test_face_adjacency_bruteforce():
    x, y, z, q = inputs.beam_with_halo(30000, 6)
    o = oracle.Oracle(max_depth=6, c_refine=0.8)
    o.build(x, y, z)
    n = o.n_int
    assert n < 6000
    lo, hi, lv, _ = _leaf_boxes(o)
    touch = np.zeros((n, n), dtype=bool)
    for d in range(3):
        e = [a for a in range(3) if a != d]
        meet = (hi[:, None, d] == lo[None, :, d]) | (lo[:, None, d] == hi[None, :, d])
        ov = np.ones((n, n), dtype=bool)
        for a in e:
            ov &= (np.minimum(hi[:, None, a], hi[None, :, a]) - np.maximum(lo[:, None, a], lo[None, :, a])) > 0
        touch |= meet & ov
    off, adj = o.adjacency()
    for j in range(n):
        nb = adj[off[j]:off[j + 1]]
        leaves = set(int(v) for v in nb if v < n)
        assert leaves == set(np.nonzero(touch[j])[0].tolist()), j
        # 2:1 face balance
        assert np.all(np.abs(lv[list(leaves)] - lv[j]) <= 1)
        # one boundary node per boundary face
        nbnd = sum(1 for v in nb if v >= n)
        on_bnd = int((lo[j] == 0).sum() + (hi[j] == 1 << KD).sum())
        assert nbnd == on_bnd


def test_boundary_nodes_on_faces():
    x, y, z, q = inputs.beam_with_halo(20000, 8)
    o = oracle.Oracle(max_depth=5, c_refine=0.8)
    o.build(x, y, z)
    nd = o.nodes()
    owner, face = o.boundary()
    ic = nd["icoord"]
    for b in range(o.n_bnd):
        f = int(face[b])
        g = o.n_int + b
        assert ic[g, f // 2] == (1 << 22 if f & 1 else 0)
        others = [d for d in range(3) if d != f // 2]
        assert np.array_equal(ic[g, others], ic[owner[b], others])
    # order: by face, then owner
    order = np.lexsort((owner, face))
    assert np.array_equal(order, np.arange(o.n_bnd))
    assert np.all(nd["kind"][o.n_int:] == 1) and np.all(nd["kind"][: o.n_int] == 0)


def _golden(name):
    vals = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", name)):
        line = line.split("#")[0].strip()
        if line:
            k, v = (t.strip() for t in line.split("="))
            vals[k] = float(v)
    return vals


def test_criterion_worked_example():
    """Sec. 4.3 (fixture tests/golden/criterion_worked_example.txt): with
    c = 0.01 a depth-21 cell of [-1, 1] (edge 2 x 2^-21 = 2^-20) would open
    only with 0.01^2 2^40 = 1.10e8 particles (depth cap lifted to 22 to
    exercise the arithmetic)."""
    g = _golden("criterion_worked_example.txt")
    assert g["depth"] == 21 and (g["hi"] - g["lo"]) * 2.0 ** -g["depth"] == 2.0 ** g["leaf_edge_log2"]
    thr = g["c"] ** 2 * 2.0 ** (-2 * g["leaf_edge_log2"])
    half_ulp = 0.5 * 10 ** (np.floor(np.log10(g["particles_to_open"])) - g["printed_digits"] + 1)
    assert abs(thr - g["particles_to_open"]) < half_ulp
    assert oracle.criterion_opens(109951163, 21, 22, -1.0, 1.0, 0.01)
    assert not oracle.criterion_opens(109951162, 21, 22, -1.0, 1.0, 0.01)
    # one level up the edge doubles and a quarter of the particles suffice
    assert oracle.criterion_opens(27487791, 20, 22, -1.0, 1.0, 0.01)
    assert not oracle.criterion_opens(27487790, 20, 22, -1.0, 1.0, 0.01)
    # empty cells and cells at the depth cap never open
    assert not oracle.criterion_opens(0, 0, 21, -1.0, 1.0, 1e-9)
    assert not oracle.criterion_opens(10 ** 9, 6, 6, -1.0, 1.0, 1e-9)


def test_uniform_grid_stencil_shape():
    """On a uniform grid the 2-ring holds the 24 nodes within L1 distance 2.  The
    octant picks and the nearest fill reach m_target = 20 inside the shell of 6
    nodes at distance 2h, and the tie rule takes the whole shell, so the stencil
    is the full, point-symmetric 2-ring (the balanced stencil of Sec. 3.3)."""
    x, y, z, q = inputs.grid_points(4)
    o = oracle.Oracle(max_depth=4, c_refine=1e-9)
    o.build(x, y, z)
    assert o.n_int == 4096
    st = o.stencils()
    nd = o.nodes()
    ic = nd["icoord"].astype(np.int64)
    h = 1 << 18
    interior = np.all((ic[: o.n_int] > 2 * h) & (ic[: o.n_int] < (1 << 22) - 2 * h), axis=1)
    for j in np.nonzero(interior)[0][:50]:
        m = st["m"][j]
        nb = st["nbr"][j, :m]
        off = (ic[nb] - ic[j]) // h
        d2 = (off ** 2).sum(1)
        assert m == 24 and st["ring"][j] == 2
        assert np.sum(d2 <= 2) == 18 and np.sum(d2 == 4) == 6
        assert np.all(np.diff(d2) >= 0)
        assert {tuple(r) for r in off} == {tuple(-r) for r in off}
        assert np.all(st["nbr"][j, m:] == -1)
