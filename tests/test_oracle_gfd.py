"""Pins for the oracle's GFD operators (Section 3.1) and linear systems (Section 3.2).

Each check is fixed by mathematics or by the paper, not by the oracle itself:
second-order GFD reproduces derivatives of quadratics exactly (Section 3.1),
a square stencil reduces to plain interpolation whatever the weights, the
weighted pseudo-inverse is unique (so an SVD-based one must agree), and the
density and Poisson systems are solved exactly by quadratic data.
"""
import numpy as np
import pytest

import oracle
from paper_1603_04039_gb300 import inputs

UNIT = 2.0 ** -21          # (hi - lo) 2^-22 on [-1, 1]


def _quad(rng):
    """Random quadratic f(x) = c + g.x + x^T H x / 2 with its derivative vector."""
    c = rng.normal()
    g = rng.normal(size=3)
    H = rng.normal(size=(3, 3))
    H = H + H.T
    ders = np.array([g[0], g[1], g[2], H[0, 0], H[0, 1], H[0, 2], H[1, 1], H[1, 2], H[2, 2]])

    def f(p):
        return c + p @ g + 0.5 * np.einsum("...i,ij,...j->...", p, H, p)
    return f, ders, H


def _random_stencil(rng, m, spread=1 << 14):
    while True:
        d = rng.integers(-spread, spread + 1, size=(m, 3)) * 2
        if np.all(np.any(d != 0, axis=1)) and len({tuple(r) for r in d}) == m:
            return d.astype(np.int64)


@pytest.mark.parametrize("m", [9, 12, 17, 20, 32])
def test_quadratic_reproduction(m):
    """Sec. 3.1: the Taylor remainder is O(h^3), so quadratics are reproduced to rounding."""
    rng = np.random.default_rng(m)
    for trial in range(20):
        d = _random_stencil(rng, m)
        res = oracle.wls(d, UNIT)
        if res is None:
            continue
        P, lap, lapd, _ = res
        f, ders, H = _quad(rng)
        y0 = rng.normal(size=3) * 0.1
        dy = d * UNIT
        # increment of the quadratic without cancellation
        df = dy @ (ders[:3] + H @ y0) + 0.5 * np.einsum("ji,ik,jk->j", dy, H, dy)
        got = P @ df
        # derivatives at y0 of the quadratic
        g0 = ders[:3] + H @ y0
        want = np.concatenate([g0, ders[3:]])
        scale = np.abs(want).max()
        assert np.allclose(got, want, rtol=0, atol=1e-9 * scale), (got, want)
        assert np.isclose(lap @ df, np.trace(H), rtol=1e-9)
        assert np.isclose(lapd, -lap.sum(), rtol=1e-15)


def test_square_stencil_is_interpolation():
    """With m = 9 the least-squares problem is square: weights cancel and P = V^{-1}."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        d = _random_stencil(rng, 9)
        res = oracle.wls(d, UNIT)
        if res is None:
            continue
        P = res[0]
        dy = d * UNIT
        V = np.column_stack([dy[:, 0], dy[:, 1], dy[:, 2], 0.5 * dy[:, 0] ** 2, dy[:, 0] * dy[:, 1],
                             dy[:, 0] * dy[:, 2], 0.5 * dy[:, 1] ** 2, dy[:, 1] * dy[:, 2],
                             0.5 * dy[:, 2] ** 2])
        if np.linalg.cond(V / np.abs(V).max(axis=0)) > 1e8:
            continue
        Vi = np.linalg.inv(V)
        assert np.allclose(P, Vi, rtol=1e-8, atol=1e-8 * np.abs(Vi).max())


def test_weighted_pseudoinverse_matches_svd():
    """P = (W V)^+ W is unique for full rank; an SVD pseudo-inverse must agree.

    W is the normalized Gaussian of Sec. 3.1 with c = 4 and r_max the largest
    neighbour distance, so W(r_max) = (e^-1 - e^-4)/(1 - e^-4) = 0.35609...
    """
    assert np.isclose((np.exp(-1) - np.exp(-4)) / (1 - np.exp(-4)), 0.35609, atol=5e-6)
    rng = np.random.default_rng(5)
    for m in (12, 20, 28):
        d = _random_stencil(rng, m)
        P, _, _, _ = oracle.wls(d, UNIT)
        dy = d * UNIT
        r2 = (d.astype(float) ** 2).sum(1)
        w = (np.exp(-r2 / r2.max()) - np.exp(-4.0)) / (1 - np.exp(-4.0))
        V = np.column_stack([dy[:, 0], dy[:, 1], dy[:, 2], 0.5 * dy[:, 0] ** 2, dy[:, 0] * dy[:, 1],
                             dy[:, 0] * dy[:, 2], 0.5 * dy[:, 1] ** 2, dy[:, 1] * dy[:, 2],
                             0.5 * dy[:, 2] ** 2])
        want = np.linalg.pinv(w[:, None] * V) * w[None, :]
        assert np.allclose(P, want, rtol=1e-7, atol=1e-9 * np.abs(want).max())
        # sqrt(W) row scaling would give a different operator: the reading matters
        alt = np.linalg.pinv(np.sqrt(w)[:, None] * V) * np.sqrt(w)[None, :]
        assert not np.allclose(P, alt, rtol=1e-4, atol=1e-6 * np.abs(alt).max())


def test_rank_deficient_stencil_rejected():
    """All neighbours on one plane: the z-derivatives are undetermined."""
    d = np.array([[2 * i, 2 * j, 0] for i in range(-2, 3) for j in range(-2, 3) if (i, j) != (0, 0)],
                 dtype=np.int64)
    assert oracle.wls(d, UNIT) is None


@pytest.fixture(scope="module")
def small_problem():
    x, y, z, q = inputs.beam_with_halo(20000, 7)
    o = oracle.Oracle(max_depth=5, c_refine=1.0)
    o.build(x, y, z)
    o.stencils()
    return o


def test_tree_stencils_reproduce_quadratics(small_problem):
    o = small_problem
    nd = o.nodes()
    xyz = nd["xyz"]
    rng = np.random.default_rng(11)
    f, ders, H = _quad(rng)
    fv = f(xyz)
    dphi = o.derivatives(fv)
    g_exact = ders[:3][None, :] + xyz[: o.n_int] @ H
    scale = np.abs(g_exact).max()
    assert np.allclose(dphi[:, :3], g_exact, atol=1e-8 * scale)
    assert np.allclose(dphi[:, 3:], ders[3:][None, :], atol=1e-7 * np.abs(ders).max())


def test_density_system_exact_for_quadratic(small_problem):
    """Reading R6 (Taylor 1/l!): for quadratic rho the exact cell average is
    rho(y) + h^2/24 Lap rho, and B maps nodal rho to exactly that."""
    o = small_problem
    nd = o.nodes()
    xyz = nd["xyz"]
    rng = np.random.default_rng(13)
    f, ders, H = _quad(rng)
    h = 2.0 / 2.0 ** nd["level"].astype(float)
    rhs = f(xyz) + h * h / 24.0 * np.trace(H)
    rhs[o.n_int:] = f(xyz[o.n_int:])          # boundary rows carry rho itself
    rho, it, rr, s = o.solve_density(rhs, rtol=1e-14)
    assert s == 0
    assert np.allclose(rho, f(xyz), rtol=0, atol=1e-10 * np.abs(f(xyz)).max())


def test_poisson_exact_for_quadratic(small_problem):
    """A quadratic phi with Lap phi = const is an exact solution of the GFD system,
    and the Taylor gather reproduces phi and grad phi at any particle."""
    o = small_problem
    nd = o.nodes()
    xyz = nd["xyz"]
    rng = np.random.default_rng(17)
    f, ders, H = _quad(rng)
    rho = np.full(o.n_nodes, np.trace(H))      # poisson_c = 1
    g = f(xyz[o.n_int:])
    phi, it, rr, s = o.solve_poisson(rho, g, rtol=1e-14)
    assert s == 0
    exact = f(xyz)
    assert np.allclose(phi, exact, atol=1e-9 * np.abs(exact).max())
    php, ex, ey, ez = o.gather(phi)
    pts = np.stack([o.x, o.y, o.z], 1)
    assert np.allclose(php, f(pts), atol=1e-9 * np.abs(exact).max())
    grad = ders[:3][None, :] + pts @ H
    assert np.allclose(np.stack([ex, ey, ez], 1), grad, atol=1e-8 * np.abs(grad).max())


def test_every_stencil_has_negative_diagonal():
    """Reading R9: no stored stencil has a Laplacian diagonal >= 0 (a wrong-sign
    row would make the discrete Laplacian indefinite)."""
    x, y, z, q = inputs.beam_with_halo(200000, 3)
    o = oracle.Oracle(max_depth=7, c_refine=0.2)
    o.build(x, y, z)
    st = o.stencils()
    assert np.all(st["lapd"] < 0)
    assert np.all(st["m"] >= 20) and np.all(st["m"] <= 32)


def test_charge_conservation():
    """Leaves partition the domain, so the deposit conserves charge (Sec. 2, N q = 1)."""
    x, y, z, q = inputs.beam_with_halo(30000, 3)
    o = oracle.Oracle(max_depth=6, c_refine=0.7)
    o.build(x, y, z)
    _, first, count = o.leaves()
    assert count.sum() == len(x)
    assert np.array_equal(first[1:], (first + count)[:-1])
    rhs, Qc, total = o.density_rhs(None, 1.0 / len(x))
    assert abs(total - 1.0) < 1e-12
    rng = np.random.default_rng(1)
    qv = rng.uniform(0.5, 1.5, len(x))
    rhs, Qc, total = o.density_rhs(qv)
    assert abs(total - qv.sum()) < 1e-12 * qv.sum()
    # rho_M times the cell volume gives the charge back
    h = 2.0 / 2.0 ** o.nodes()["level"][: o.n_int].astype(float)
    assert np.allclose(rhs[: o.n_int] * h ** 3, Qc, rtol=1e-14)


def test_gmres_matches_dense_solve():
    """The oracle's GMRES against a dense LAPACK solve of the oracle's own matrix."""
    x, y, z, q = inputs.beam_with_halo(100000, 1)
    o = oracle.Oracle(max_depth=6, c_refine=1.0)
    o.build(x, y, z)
    o.stencils()
    for which in ("B", "A"):
        rp, col, val = o.matrix(which)
        n = o.n_nodes
        Ad = np.zeros((n, n))
        rows = np.repeat(np.arange(n), np.diff(rp))
        Ad[rows, col] = val
        b = np.random.default_rng(2).normal(size=n)
        xd = np.linalg.solve(Ad, b)
        xg, it, rr, s = oracle.gmres(rp, col, val, b, rtol=1e-13, max_iter=20000)
        assert s == 0 and rr <= 1e-13
        assert np.linalg.norm(xg - xd) <= 1e-10 * np.linalg.norm(xd)
