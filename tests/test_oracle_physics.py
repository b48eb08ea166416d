"""Physics pins for the oracle: closed-form potentials and brute-force sums.

Potentials solve Lap phi = rho (Eq. Poisson with c = 1, Section 5) so a point
charge Q has phi = -Q / (4 pi r) and E = grad phi (Section 2).
"""
import os

import numpy as np
import pytest
from scipy.special import erf, ndtr

import oracle
from paper_1603_04039_gb300 import inputs


def gauss_phi(p, sig, Q=1.0):
    r = np.linalg.norm(p, axis=-1)
    return -Q * erf(r / (np.sqrt(2) * sig)) / (4 * np.pi * r)


def gauss_grad(p, sig, Q=1.0):
    r = np.linalg.norm(p, axis=-1)
    a = np.sqrt(2) * sig
    dr = Q / (4 * np.pi) * (erf(r / a) / r ** 2 - 2 / np.sqrt(np.pi) * np.exp(-(r / a) ** 2) / (a * r))
    return dr[:, None] * p / r[:, None]


def _gaussian_errors(depth, sig):
    """Section 5 convergence test without Monte Carlo noise: rho_M is the exact
    cell average of the density, g the exact potential on the boundary."""
    x, y, z, q = inputs.grid_points(depth)
    o = oracle.Oracle(max_depth=depth, c_refine=1e-9)
    o.build(x, y, z)
    o.stencils()
    nd = o.nodes()
    xyz = nd["xyz"]
    ni = o.n_int
    h = 2.0 / 2.0 ** nd["level"][:ni].astype(float)
    a = xyz[:ni] - h[:, None] / 2
    b = xyz[:ni] + h[:, None] / 2
    avg = np.prod(ndtr(b / sig) - ndtr(a / sig), axis=1) / h ** 3
    owner, _ = o.boundary()
    rhs = np.concatenate([avg, avg[owner]])
    rho, _, _, _ = o.solve_density(rhs, rtol=1e-13)
    phi, _, _, _ = o.solve_poisson(rho, gauss_phi(xyz[ni:], sig), rtol=1e-13)
    d = o.derivatives(phi)
    ex = gauss_phi(xyz[:ni], sig)
    gx = gauss_grad(xyz[:ni], sig)
    e_phi = np.linalg.norm(phi[:ni] - ex) / np.linalg.norm(ex)
    e_e = np.linalg.norm(d[:, :3] - gx) / np.linalg.norm(gx)
    return e_phi, e_e


def _paper_orders():
    """Orders of Table convergence_order (fixture tests/golden/convergence_order_table.txt)."""
    rows = []
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "convergence_order_table.txt")):
        line = line.split("#")[0].split()
        if line and line[3] != "-":
            rows.append((float(line[3]), float(line[4])))
    return np.array(rows)


@pytest.mark.slow
def test_second_order_convergence_without_mc_noise():
    """Sections 3.3 and 5: with exact cell integrals the second-order method
    converges at order ~2 in both phi and grad phi; every observed order must
    reach the smallest one the paper prints (1.82 for phi, 1.96 for phi_x)
    less 0.05."""
    paper = _paper_orders()
    assert paper.shape == (3, 2)
    errs = [_gaussian_errors(d, 0.15) for d in (4, 5, 6)]
    for (p0, e0), (p1, e1) in zip(errs[:-1], errs[1:]):
        assert np.log2(p0 / p1) > paper[:, 0].min() - 0.05, errs
        assert np.log2(e0 / e1) > paper[:, 1].min() - 0.05, errs
    assert errs[-1][0] < 2e-3 and errs[-1][1] < 6e-3


def _ball(n, R, seed, centre=(0.0, 0.0, 0.0)):
    u = inputs.uniforms(seed, 7, 3 * n).reshape(-1, 3)
    r = R * np.cbrt(u[:, 0])
    cz = 2 * u[:, 1] - 1
    ph = 2 * np.pi * u[:, 2]
    st = np.sqrt(1 - cz ** 2)
    return np.stack([r * st * np.cos(ph), r * st * np.sin(ph), r * cz], 1) + np.asarray(centre)


def test_uniform_sphere_closed_form():
    """A uniformly charged ball of radius R and charge 1: phi = r^2/(8 pi R^3) -
    3/(8 pi R) inside, -1/(4 pi r) outside.  Monte Carlo noise and the kink at R
    limit accuracy, and the error must shrink as the tree is refined."""
    R, N = 0.4, 100000
    P = _ball(N, R, 9)

    def phi_ex(p):
        rr = np.linalg.norm(p, axis=-1)
        return np.where(rr < R, rr ** 2 / (8 * np.pi * R ** 3) - 3 / (8 * np.pi * R),
                        -1 / (4 * np.pi * np.maximum(rr, 1e-300)))

    def e_ex(p):
        rr = np.linalg.norm(p, axis=-1)[:, None]
        return np.where(rr < R, p / (4 * np.pi * R ** 3), p / (4 * np.pi * rr ** 3))

    errs = []
    for depth, c in ((5, 1.0), (6, 0.5)):
        o = oracle.Oracle(max_depth=depth, c_refine=c)
        o.build(P[:, 0], P[:, 1], P[:, 2])
        o.stencils()
        nd = o.nodes()
        rhs, _, tot = o.density_rhs(None, 1.0 / N)
        assert abs(tot - 1.0) < 1e-12
        rho, _, _, _ = o.solve_density(rhs, rtol=1e-12)
        phi, _, _, _ = o.solve_poisson(rho, phi_ex(nd["xyz"][o.n_int:]), rtol=1e-12)
        pp, ex, ey, ez = o.gather(phi)
        e1 = np.linalg.norm(pp - phi_ex(P)) / np.linalg.norm(phi_ex(P))
        E = np.stack([ex, ey, ez], 1)
        e2 = np.linalg.norm(E - e_ex(P)) / np.linalg.norm(e_ex(P))
        errs.append((e1, e2))
    assert errs[0][0] < 3e-2 and errs[0][1] < 6e-2, errs
    assert errs[1][0] < 1e-2 and errs[1][1] < 5e-2, errs
    assert errs[1][0] < 0.5 * errs[0][0] and errs[1][1] < errs[0][1], errs


def test_tiny_n_matches_coulomb_sum():
    """A few hundred charges in a small blob and zero-charge probe particles far
    from it: the probes' phi and E must match the direct Coulomb sum
    -sum q / (4 pi |x - p|) up to the discretisation error, and the error must
    fall as the tree deepens."""
    nq, npr = 400, 60
    charges = _ball(nq, 0.08, 21, centre=(0.1, -0.05, 0.02))
    u = inputs.uniforms(22, 8, 3 * npr).reshape(-1, 3)
    rr = 0.45 + 0.25 * u[:, 0]
    cz = 2 * u[:, 1] - 1
    ph = 2 * np.pi * u[:, 2]
    st = np.sqrt(1 - cz ** 2)
    probes = np.stack([rr * st * np.cos(ph), rr * st * np.sin(ph), rr * cz], 1)
    P = np.concatenate([charges, probes])
    q = np.concatenate([np.full(nq, 1.0 / nq), np.zeros(npr)])

    def direct(x):
        d = x[:, None, :] - charges[None, :, :]
        r = np.linalg.norm(d, axis=-1)
        phi = -(q[None, :nq] / (4 * np.pi * r)).sum(1)
        E = ((q[None, :nq] / (4 * np.pi * r ** 3))[:, :, None] * d).sum(1)
        return phi, E

    errs = []
    for depth, c in ((5, 0.05), (7, 0.01)):
        o = oracle.Oracle(max_depth=depth, c_refine=c)
        o.build(P[:, 0], P[:, 1], P[:, 2])
        o.stencils()
        nd = o.nodes()
        g, _ = direct(nd["xyz"][o.n_int:])
        rhs, _, tot = o.density_rhs(q)
        assert abs(tot - 1.0) < 1e-12
        rho, _, _, _ = o.solve_density(rhs, rtol=1e-12)
        phi, _, _, _ = o.solve_poisson(rho, g, rtol=1e-12)
        pp, ex, ey, ez = o.gather(phi)
        pe, Ee = direct(probes)
        e1 = np.linalg.norm(pp[nq:] - pe) / np.linalg.norm(pe)
        e2 = np.linalg.norm(np.stack([ex, ey, ez], 1)[nq:] - Ee) / np.linalg.norm(Ee)
        errs.append((e1, e2))
    assert errs[-1][0] < 2e-2 and errs[-1][1] < 5e-2, errs
    assert errs[1][0] < errs[0][0] and errs[1][1] < errs[0][1], errs


def test_paper_3d_normalisation():
    """Section 5.2: a1 = 7677 normalises the two-Gaussian density on [-1, 1]^3 when
    tau acts as a standard deviation, exp(-r^2 / (2 tau^2))."""
    def mass(tau):
        one = ndtr(1 / tau) - ndtr(-1 / tau)
        return (2 * np.pi * tau ** 2) ** 1.5 * one ** 3
    a1 = 1.0 / (mass(0.02) + 1e-5 * mass(0.3))
    assert abs(a1 - 7677) / 7677 < 3e-4
    # the literal exp(-r^2 / tau^2) form would need a1 ~ 2.17e4
    a1_lit = 1.0 / ((np.pi * 0.02 ** 2) ** 1.5 + 1e-5 * (np.pi * 0.09) ** 1.5 *
                    (erf(1 / 0.3)) ** 3)
    assert a1_lit > 2e4
