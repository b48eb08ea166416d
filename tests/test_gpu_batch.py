"""Batches of independent beams solved as one block-diagonal problem.

Every beam of a batch must come out exactly as the oracle computes it for that
beam alone: node sets, leaf ranges and stencil neighbour lists bit-exact, and
rho, phi, node derivatives and particle fields within the FP64 form's 1e-10
relative L2.  Every beam of a batch stops at its own relative residual rtol
(converged beams are frozen at each restart), so rtol = 1e-13 leaves the same
margin as the single-beam parity tests.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1603_04039_gb300 import inputs

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _batch(nb, depth, c, n_lo, n_hi, seed, **kw):
    from paper_1603_04039_gb300 import APCloud
    x, y, z, q, offs, params = inputs.beam_batch(nb, seed, n_lo, n_hi)
    ap = APCloud(max_depth=depth, c_refine=c, **kw)
    ap.build_octree_batched(_t(x), _t(y), _t(z), offs)
    return ap, (x, y, z, q, offs, params)


def _split(ap):
    """Per beam: interior node indices and boundary node indices, in node order."""
    beam = ap.get_node_beams().cpu().numpy()
    idx = np.arange(ap.n_nodes)
    out = []
    for b in range(beam.max() + 1):
        sel = idx[beam == b]
        out.append((sel[sel < ap.n_int], sel[sel >= ap.n_int]))
    return out


@pytest.mark.parametrize("nb,depth,c,seed,pdeg", [(5, 6, 0.3, 1, 1), (9, 5, 0.5, 2, 1), (3, 7, 0.15, 3, 1),
                                                  (5, 6, 0.3, 1, 8), (9, 5, 0.5, 2, 8)])
def test_batch_matches_oracle_per_beam(nb, depth, c, seed, pdeg):
    """pdeg 1: one shared Krylov space with converged beams frozen at restarts;
    pdeg 8: an independent Krylov space per beam (FP64 polynomial form)."""
    ap, (x, y, z, q, offs, params) = _batch(nb, depth, c, 2000, 30000, seed, poly_degree=pdeg, poly_omega=1.0)
    ap.stencils()
    rho, ir = ap.deposit(q=_t(q), rtol=1e-13)
    phi, ip = ap.solve(rtol=1e-13)
    php, ex, ey, ez = ap.gather_field()
    assert ir["status"] == 0 and ip["status"] == 0
    g_nodes = ap.get_nodes()
    g_xyz, g_lvl, g_kind = (g_nodes[k].cpu().numpy() for k in ("xyz", "level", "kind"))
    gl = {k: v.cpu().numpy() for k, v in ap.get_leaves().items()}
    gs = {k: v.cpu().numpy() for k, v in ap.get_stencils().items()}
    rm = ap.get_rho_m().cpu().numpy()
    rho, phi = rho.cpu().numpy(), phi.cpu().numpy()
    dphi = ap.get_derivatives().cpu().numpy()
    php, ex, ey, ez = (a.cpu().numpy() for a in (php, ex, ey, ez))
    parts = _split(ap)
    assert len(parts) == nb
    for b in range(nb):
        s, e = offs[b], offs[b + 1]
        o = oracle.Oracle(max_depth=depth, c_refine=c)
        ref = o.run(x[s:e], y[s:e], z[s:e], q=q[s:e], rtol=1e-13)
        ii, bb = parts[b]
        assert (len(ii), len(bb)) == (o.n_int, o.n_bnd), b
        nodes = np.concatenate([ii, bb])
        w = o.nodes()
        assert np.array_equal(g_xyz[nodes], w["xyz"])
        assert np.array_equal(g_lvl[nodes], w["level"])
        assert np.array_equal(g_kind[nodes], w["kind"])
        key, first, count = o.leaves()
        L = depth
        lvl = g_lvl[ii].astype(np.uint64)
        gkey = gl["key"][ii].astype(np.uint64)
        beam_bits = gkey >> (np.uint64(3) * lvl)
        assert np.all(beam_bits == b)
        assert np.array_equal(gkey & ((np.uint64(1) << (np.uint64(3) * lvl)) - np.uint64(1)), key)
        assert np.array_equal(gl["first"][ii] - s, first)
        assert np.array_equal(gl["count"][ii], count)
        # stencil neighbour lists: global node ids map back to the beam's own numbering
        loc = np.full(ap.n_nodes, -1)
        loc[nodes] = np.arange(len(nodes))
        ws = o.stencils()
        assert np.array_equal(gs["m"][ii], ws["m"])
        nbr = gs["nbr"][ii]
        mapped = np.where(nbr >= 0, loc[np.maximum(nbr, 0)], -1)
        assert np.array_equal(mapped, ws["nbr"])
        # rho_M = Q_j / h^3 with Q_j a sum of N'_j charges in another order:
        # |dQ| <= (N'_j - 1) u sum|q| on either side (u = 2^-53)
        tol = 2.0 * 1.12e-16 * (count.max() + 1)
        assert np.allclose(rm[nodes], ref["rhoM"], rtol=tol, atol=0)
        assert _rel(rho[nodes], ref["rho"]) < 1e-10
        assert _rel(phi[nodes], ref["phi"]) < 1e-10
        assert _rel(dphi[ii], ref["dphi"]) < 1e-10
        assert _rel(php[s:e], ref["phi_p"]) < 1e-10
        for a, r in ((ex, ref["ex"]), (ey, ref["ey"]), (ez, ref["ez"])):
            assert _rel(a[s:e], r) < 1e-10


def test_single_beam_batch_is_the_plain_build():
    from paper_1603_04039_gb300 import APCloud
    x, y, z, q = inputs.beam_with_halo(40000, 4)
    out = []
    for batched in (False, True):
        ap = APCloud(max_depth=6, c_refine=0.4)
        if batched:
            ap.build_octree_batched(_t(x), _t(y), _t(z), [0, len(x)])
        else:
            ap.build_octree(_t(x), _t(y), _t(z))
        ap.stencils()
        ap.deposit(q_uniform=1.0 / len(x), rtol=1e-12)
        phi, info = ap.solve(rtol=1e-12)
        php, ex, ey, ez = ap.gather_field()
        out.append((phi.cpu().numpy(), php.cpu().numpy(), ex.cpu().numpy(), info["iters"]))
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


def test_batch_with_empty_and_tiny_beams():
    """Empty beams keep their roots as single leaves (six boundary nodes each);
    a beam of three particles refines as the oracle refines it alone."""
    from paper_1603_04039_gb300 import APCloud
    rng = np.random.default_rng(5)
    xa, ya, za, _ = inputs.beam_with_halo(20000, 6)
    tiny = rng.uniform(-0.5, 0.5, size=(3, 3))
    x = np.concatenate([xa, tiny[:, 0]])
    y = np.concatenate([ya, tiny[:, 1]])
    z = np.concatenate([za, tiny[:, 2]])
    offs = [0, 0, 20000, 20000, 20003]
    ap = APCloud(max_depth=5, c_refine=0.5)
    ni, nbnd = ap.build_octree_batched(_t(x), _t(y), _t(z), offs)
    beam = ap.get_node_beams().cpu().numpy()
    xyz = ap.get_nodes()["xyz"].cpu().numpy()
    refs = {}
    for b, (px, py, pz) in ((1, (xa, ya, za)), (3, (tiny[:, 0].copy(), tiny[:, 1].copy(), tiny[:, 2].copy()))):
        o = oracle.Oracle(max_depth=5, c_refine=0.5)
        o.build(px, py, pz)
        refs[b] = o
        sel = np.concatenate([np.where(beam[:ni] == b)[0], ni + np.where(beam[ni:] == b)[0]])
        assert np.array_equal(xyz[sel], o.nodes()["xyz"])
    assert np.array_equal(np.bincount(beam[:ni], minlength=4), [1, refs[1].n_int, 1, refs[3].n_int])
    assert nbnd == refs[1].n_bnd + refs[3].n_bnd + 12
    root = xyz[np.where(beam[:ni] == 0)[0][0]]
    assert np.array_equal(root, [0.0, 0.0, 0.0])


def test_batch_rejects_bad_offsets():
    from paper_1603_04039_gb300 import APCloud, APCloudError
    ap = APCloud(max_depth=4, c_refine=1.0)
    x = _t(np.zeros(10))
    for offs in ([0, 5, 3, 10], [1, 10]):
        with pytest.raises(APCloudError) as e:
            ap.build_octree_batched(x, x, x, offs)
        assert e.value.status == -1
    with pytest.raises(ValueError):
        ap.build_octree_batched(x, x, x, [0, 9])


def test_batch_mixed_precision_within_1e6_of_fp64():
    """The mixed form on a batch: every beam's fields within 1e-6 relative L2
    of the FP64 form of the same batch."""
    res = []
    for prec in ("fp64", "mixed"):
        ap, (x, y, z, q, offs, params) = _batch(6, 6, 0.2, 3000, 60000, 7, precision=prec, poly_degree=16,
                                                poly_omega=1.0)
        ap.stencils()
        ap.deposit(q=_t(q), rtol=1e-10)
        ap.solve(rtol=1e-10)
        php, ex, ey, ez = ap.gather_field()
        res.append((offs, php.cpu().numpy(), ex.cpu().numpy(), ey.cpu().numpy(), ez.cpu().numpy()))
    offs = res[0][0]
    for b in range(len(offs) - 1):
        s, e = offs[b], offs[b + 1]
        for k in range(1, 5):
            assert _rel(res[1][k][s:e], res[0][k][s:e]) < 1e-6, (b, k)
