"""Pins of the oracle's stencil selection (Section 3.1, "two nearest nodes
from each quadrant", read in 3-D as two per octant; Section 4.3 ring search).

  * hand-derived selections (fixture tests/golden/octant_selection.txt) for a
    skewed cloud -- a dense cluster on one side of the node, single far nodes
    in the other octants, as next to a level jump -- and for two full shells
    where the 32-node cap decides;
  * the fixture separates the rule from its plausible misreadings: each
    mutated rule below (one per octant, no octant step, zero counted as -,
    no tie rule, no cap, three per octant) selects differently on it;
  * the selection does not depend on the order the candidates come in;
  * on a graded tree every stencil holds the two nearest ring candidates of
    each octant (or all, when an octant has fewer), and the octant step
    changes the stencil of many nodes, so a parity test on that tree
    exercises it.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1603_04039_gb300 import inputs

MMAX = 32


def _cases():
    cases, cur = [], None
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "octant_selection.txt")):
        line = line.split("#")[0].split()
        if not line:
            continue
        if line[0] == "case":
            cur = {"name": line[1], "m": int(line[2].split("=")[1]), "idx": [], "off": []}
            cases.append(cur)
        elif line[0] == "cand":
            cur["idx"].append(int(line[1]))
            cur["off"].append([int(v) for v in line[2:5]])
        elif line[0] == "expect":
            cur["expect"] = [int(v) for v in line[1:]]
    return cases


CASES = _cases()


def test_fixture_is_complete():
    assert [c["name"] for c in CASES] == ["skewed", "shells"]
    for c in CASES:
        assert len(set(c["idx"])) == len(c["idx"])
        assert len(c["expect"]) == len(set(c["expect"])) <= MMAX
        assert set(c["expect"]) <= set(c["idx"])


@pytest.mark.parametrize("case", CASES, ids=lambda c: c["name"])
def test_selection_matches_hand_derivation(case):
    got = oracle.select_neighbours(np.array(case["off"]), np.array(case["idx"]), case["m"])
    assert got.tolist() == case["expect"]


@pytest.mark.parametrize("case", CASES, ids=lambda c: c["name"])
def test_selection_ignores_candidate_order(case):
    rng = np.random.default_rng(11)
    off, idx = np.array(case["off"]), np.array(case["idx"])
    for _ in range(5):
        p = rng.permutation(len(idx))
        assert oracle.select_neighbours(off[p], idx[p], case["m"]).tolist() == case["expect"]


# ---- misreadings of the rule, each a plausible mistake in an implementation
def _mutant(off, idx, mt, per_octant=2, zero_plus=True, ties=True, cap=MMAX):
    off = np.asarray(off)
    d2 = (off ** 2).sum(1)
    pos = (off >= 0) if zero_plus else (off > 0)
    octant = 4 * pos[:, 0] + 2 * pos[:, 1] + pos[:, 2]
    order = sorted(range(len(idx)), key=lambda t: (d2[t], idx[t]))
    taken, chosen = {}, set()
    for t in order:
        if taken.get(octant[t], 0) < per_octant and len(chosen) < cap:
            taken[octant[t]] = taken.get(octant[t], 0) + 1
            chosen.add(t)
    cut = None
    for t in order:
        if len(chosen) >= min(mt, cap):
            break
        if t not in chosen:
            chosen.add(t)
            cut = d2[t]
    if ties:
        for t in order:
            if len(chosen) >= cap:
                break
            if t not in chosen and d2[t] == cut:
                chosen.add(t)
    return [idx[t] for t in order if t in chosen]


MUTANTS = {
    "one_per_octant": dict(per_octant=1),
    "no_octant_step": dict(per_octant=0),
    "three_per_octant": dict(per_octant=3),
    "zero_counted_as_minus": dict(zero_plus=False),
    "no_tie_rule": dict(ties=False),
    "no_cap": dict(cap=10 ** 6),
}


def test_mutant_model_reproduces_the_rule():
    """The unmutated model gives the fixture's answers, so the mutants below
    differ from the rule only in the mutated step."""
    for c in CASES:
        assert _mutant(c["off"], c["idx"], c["m"]) == c["expect"]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_fixture_rejects_misreading(name):
    kw = MUTANTS[name]
    assert any(_mutant(c["off"], c["idx"], c["m"], **kw) != c["expect"] for c in CASES), name


# ---- on a tree with level jumps
@pytest.fixture(scope="module")
def graded():
    x, y, z, q = inputs.beam_with_halo(100000, 1)
    o = oracle.Oracle(max_depth=6, c_refine=1.0)
    o.build(x, y, z)
    st = o.stencils()
    nd = o.nodes()
    off, adj = o.adjacency()
    return o, st, nd, off, adj


def _ring(off, adj, j, k):
    seen = {j}
    front = [j]
    for _ in range(k):
        nxt = []
        for u in front:
            for v in adj[off[u]:off[u + 1]]:
                if v not in seen:
                    seen.add(v)
                    nxt.append(v)
        front = nxt
    seen.discard(j)
    return np.array(sorted(seen))


def test_every_octant_contributes_its_two_nearest(graded):
    o, st, nd, off, adj = graded
    ic = nd["icoord"].astype(np.int64)
    changed = 0
    for j in range(o.n_int):
        m = st["m"][j]
        sel = set(st["nbr"][j, :m].tolist())
        cand = _ring(off, adj, j, st["ring"][j])
        dd = ic[cand] - ic[j]
        d2 = (dd ** 2).sum(1)
        octant = 4 * (dd[:, 0] >= 0) + 2 * (dd[:, 1] >= 0) + (dd[:, 2] >= 0)
        rank = np.lexsort((cand, d2))
        for oc in range(8):
            mine = [cand[t] for t in rank if octant[t] == oc][:2]
            assert set(mine) <= sel, (j, oc)
        # nearest-first prefix (with ties) of the same size: differs when the
        # octant step pulled in a farther node
        far = max(d2[np.isin(cand, list(sel))])
        if np.any((d2 < far) & ~np.isin(cand, list(sel))):
            changed += 1
    # the octant step shapes a good share of the stencils on this tree
    assert changed > o.n_int // 20, changed
