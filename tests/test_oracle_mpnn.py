"""Pins of the learned-preconditioner oracle (CPU only).

  * the backward pass matches central finite differences of the loss for
    every parameter block (an independent check of every chain-rule step);
  * the untrained network (zero head) is exactly Jacobi: s = 1 and u0 = b, so
    Lp and Lg equal their definitions evaluated directly on the matrix;
  * the approximate-inverse objective is minimised over free diagonals by
    s_j = 1 / c_j (c_j the squared column norm of Ahat), the closed form of
    the least-squares problem column by column;
  * aggregation rows are convex combinations (P 1 = 1 on interior rows).
"""
import numpy as np
import pytest

import oracle
from oracle import mpnn
from paper_1603_04039_gb300 import inputs


@pytest.fixture(scope="module")
def system():
    x, y, z, q = inputs.beam_with_halo(4000, 31)
    o = oracle.Oracle(max_depth=4, c_refine=0.4)
    o.build(x, y, z)
    o.stencils()
    rhs, _, _ = o.density_rhs(q)
    rho, *_ = o.solve_density(rhs, rtol=1e-12)
    b = o.poisson_rhs(rho)
    Ah = mpnn.scaled_matrix(*o.matrix("A"))
    nd = o.nodes()
    F, P = mpnn.features(Ah, nd["xyz"], nd["level"], nd["kind"].astype(np.float64), b, 2.0)
    return Ah, F, P, b, nd


def test_aggregation_rows(system):
    Ah, F, P, b, nd = system
    rs = np.asarray(P.sum(axis=1)).ravel()
    interior = nd["kind"] == 0
    assert np.allclose(rs[interior], 1.0, atol=1e-14)
    assert np.all((rs[~interior] == 0.0) | np.isclose(rs[~interior], 1.0, atol=1e-14))
    assert np.allclose(Ah.diagonal(), 1.0, atol=1e-15)


def test_untrained_network_is_jacobi(system):
    Ah, F, P, b, nd = system
    theta = mpnn.init_params(3)
    fw = mpnn.forward(theta, F, P)
    assert np.all(fw["s"] == 1.0) and np.all(fw["gamma"] == 1.0)
    interior = nd["kind"] == 0
    assert np.array_equal(fw["interior"], interior)
    L, Lp, Lg, c, r = mpnn.loss(Ah, b, fw["s"], fw["gamma"], interior)
    n = Ah.shape[0]
    I = np.eye(n)
    dense = Ah.toarray()
    assert np.isclose(Lp, np.linalg.norm((I - dense)[:, interior]) ** 2 / interior.sum(), rtol=1e-12)
    assert np.isclose(Lg, np.linalg.norm(b - dense @ b) ** 2 / np.linalg.norm(b) ** 2, rtol=1e-12)


def test_closed_form_minimiser_of_lp(system):
    Ah, F, P, b, nd = system
    n = Ah.shape[0]
    interior = nd["kind"] == 0
    dense = Ah.toarray()
    c = (dense ** 2).sum(axis=0)
    s_opt = np.where(interior, 1.0 / c, 1.0)
    base = mpnn.loss(Ah, b, s_opt, np.ones(n), interior)[1]
    resid = (np.eye(n) - dense * s_opt[None, :])[:, interior]
    assert np.isclose(base, np.linalg.norm(resid) ** 2 / interior.sum(), rtol=1e-12)
    rng = np.random.default_rng(0)
    for _ in range(5):
        s = s_opt * np.where(interior, np.exp(0.05 * rng.normal(size=n)), 1.0)
        assert mpnn.loss(Ah, b, s, np.ones(n), interior)[1] > base


def test_backward_matches_finite_differences(system):
    Ah, F, P, b, nd = system
    rng = np.random.default_rng(1)
    theta = mpnn.init_params(5)
    # a non-zero head so that every block receives gradient
    p = mpnn.unflatten(theta)
    p["Wo"] = rng.normal(scale=0.3, size=p["Wo"].shape)
    p["bo"] = np.array([0.1, -0.2])
    theta = mpnn.flatten(p)
    (L, Lp, Lg), g, _ = mpnn.loss_and_grad(theta, Ah, F, P, b)
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in mpnn.SHAPES])
    eps = 1e-6
    for k, (name, shape) in enumerate(mpnn.SHAPES):
        idx = rng.choice(np.arange(offs[k], offs[k + 1]), size=min(6, offs[k + 1] - offs[k]), replace=False)
        for i in idx:
            tp = theta.copy(); tp[i] += eps
            tm = theta.copy(); tm[i] -= eps
            fd = (mpnn.loss_and_grad(tp, Ah, F, P, b)[0][0] - mpnn.loss_and_grad(tm, Ah, F, P, b)[0][0]) / (2 * eps)
            assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (name, i, fd, g[i])


def _frac_table():
    import os
    from fractions import Fraction
    rows = {"a": [], "node": [], "p": [], "f": []}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "mpnn_features_4node.txt")):
        t = line.split("#")[0].split()
        if t:
            rows[t[0]].append([float(Fraction(v)) for v in t[1:]])
    return {k: np.array(v) for k, v in rows.items()}


def test_features_of_hand_made_system():
    """Every feature column (fixture tests/golden/mpnn_features_4node.txt):
    a 4-node system whose aggregation weights, offsets, level jumps and
    right-hand side were worked out by hand.  Row and column sums, the
    symmetrised graph, the row-normalised aggregation, offsets scaled by the
    receiving node's own cell edge, and the level offset's direction all
    differ between right and wrong readings here."""
    import scipy.sparse as sp
    g = _frac_table()
    n = 4
    r, c, v = g["a"][:, 0].astype(int), g["a"][:, 1].astype(int), g["a"][:, 2]
    Ah = (sp.csr_matrix((v, (r, c)), shape=(n, n)) + sp.identity(n)).tocsr()
    nd = g["node"]
    F, P = mpnn.features(Ah, nd[:, 1:4], nd[:, 4].astype(np.int8), nd[:, 5], nd[:, 6], 2.0)
    want_P = np.zeros((n, n))
    want_P[g["p"][:, 0].astype(int), g["p"][:, 1].astype(int)] = g["p"][:, 2]
    assert np.allclose(P.toarray(), want_P, rtol=0, atol=1e-15)
    want = g["f"][:, 1:].copy()
    want[:, 2:7] = np.sign(want[:, 2:7]) * np.log1p(np.abs(want[:, 2:7]))
    assert F.shape == (n, mpnn.NF)
    assert np.allclose(F, want, rtol=1e-14, atol=1e-15), np.abs(F - want).max(axis=0)
