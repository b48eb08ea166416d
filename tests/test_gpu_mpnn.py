"""The learned preconditioner on the GPU against its CPU oracle (oracle/mpnn.py).

  * node features (FP32 arithmetic on both sides): relative 1e-5;
  * forward pass: the head pre-activations t recovered from s and gamma,
    BF16 weights and activations with FP32 accumulation against FP64:
    relative L2 3e-2 (BF16 keeps 8 significant bits, about 4e-3 per
    rounding, over three layers);
  * gradients: every parameter block within relative L2 5e-2 and cosine
    similarity above 0.995 of the FP64 gradient, for the same weights
    (BF16-representable), the same system and the same right-hand side;
  * training: the network learns on the GPU with its own kernels, lowers the
    loss on held-out systems, and cuts Jacobi-GMRES iterations without
    changing the solution beyond the solver tolerance.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import mpnn as om
from paper_1603_04039_gb300 import inputs

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _bf16(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float32).numpy()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _system(n, depth, c, seed, **kw):
    from paper_1603_04039_gb300 import APCloud
    x, y, z, q = inputs.beam_with_halo(n, seed)
    ap = APCloud(max_depth=depth, c_refine=c, **kw)
    ap.build_octree(_t(x), _t(y), _t(z))
    ap.stencils()
    ap.deposit(q=_t(q), rtol=1e-12)
    return ap, (x, y, z, q)


def _oracle_system(x, y, z, q, depth, c):
    o = oracle.Oracle(max_depth=depth, c_refine=c)
    o.build(x, y, z)
    o.stencils()
    rhs, _, _ = o.density_rhs(q)
    rho, *_ = o.solve_density(rhs, rtol=1e-12)
    b = o.poisson_rhs(rho)
    Ah = om.scaled_matrix(*o.matrix("A"))
    nd = o.nodes()
    F, P = om.features(Ah, nd["xyz"], nd["level"], nd["kind"].astype(np.float64), b, 2.0)
    return Ah, F, P, b


def _test_params(seed):
    """Random BF16-representable parameters with a small non-zero head."""
    rng = np.random.default_rng(seed)
    p = om.unflatten(om.init_params(seed))
    for l in range(3):
        p["b%d" % l] = rng.normal(scale=0.05, size=p["b%d" % l].shape)
    p["Wo"] = rng.normal(scale=0.01, size=p["Wo"].shape)
    p["bo"] = np.array([0.02, -0.03])
    th = om.flatten(p)
    return _bf16(th).astype(np.float64)


@pytest.fixture(scope="module")
def pair():
    ap, (x, y, z, q) = _system(20000, 5, 0.3, 41)
    Ah, F, P, b = _oracle_system(x, y, z, q, 5, 0.3)
    assert Ah.shape[0] == ap.n_nodes
    return ap, Ah, F, P, b


def test_features_match_oracle(pair):
    from paper_1603_04039_gb300 import MPNN
    ap, Ah, F, P, b = pair
    net = MPNN(seed=1)
    out = net.outputs(ap)
    Fg = out["features"].cpu().numpy().astype(np.float64)
    for k in range(16):
        scale = max(np.abs(F[:, k]).max(), 1e-30)
        assert np.abs(Fg[:, k] - F[:, k]).max() <= 1e-5 * scale, k
    # untrained network: exactly Jacobi and the plain guess
    assert np.all(out["s"].cpu().numpy() == 1.0) and np.all(out["gamma"].cpu().numpy() == 1.0)


def test_forward_matches_oracle(pair):
    from paper_1603_04039_gb300 import MPNN
    ap, Ah, F, P, b = pair
    th = _test_params(2)
    net = MPNN(theta=th.astype(np.float32))
    out = net.outputs(ap)
    s = out["s"].cpu().numpy().astype(np.float64)
    g = out["gamma"].cpu().numpy().astype(np.float64)
    fw = om.forward(th, F, P)
    inter = fw["interior"]
    assert np.all(s[~inter] == 1.0)
    t0 = np.arctanh(np.log(s[inter]) / om.ALPHA)
    t1 = np.arctanh(np.log(g))
    assert _rel(t0, fw["t"][inter, 0]) < 3e-2
    assert _rel(t1, fw["t"][:, 1]) < 3e-2


def test_gradients_match_oracle(pair):
    from paper_1603_04039_gb300 import MPNN
    ap, Ah, F, P, b = pair
    th = _test_params(3)
    net = MPNN(theta=th.astype(np.float32))
    lg = net.loss(ap, backward=True)
    _, gg = net.params()
    (L, Lp, Lg), gw, _ = om.loss_and_grad(th, Ah, F, P, b)
    assert abs(lg["Lp"] - Lp) <= 2e-2 * abs(Lp)
    assert abs(lg["Lg"] - Lg) <= 2e-2 * abs(Lg)
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in om.SHAPES])
    report = {}
    for k, (name, _) in enumerate(om.SHAPES):
        a = gg[offs[k]:offs[k + 1]].astype(np.float64)
        w = gw[offs[k]:offs[k + 1]]
        cos = float(a @ w / (np.linalg.norm(a) * np.linalg.norm(w) + 1e-300))
        report[name] = (_rel(a, w), cos)
    for name, (r, cos) in report.items():
        assert r < 5e-2 and cos > 0.995, report


def test_training_cuts_jacobi_iterations():
    from paper_1603_04039_gb300 import MPNN
    train = [_system(20000, 6, 0.3, 100 + k)[0] for k in range(12)]
    net = MPNN(seed=7)
    held, _ = _system(30000, 6, 0.3, 900, poly_degree=1)
    before = net.loss(held)
    for step in range(360):
        ap = train[step % len(train)]
        net.loss(ap, backward=True)
        net.adam(ap, lr=2e-3)
    after = net.loss(held)
    # the closed-form minimiser of Lp reaches 0.75 of Jacobi's on this system
    assert after["Lp"] < 0.8 * before["Lp"], (before, after)
    phi0, i0 = held.solve_learned(net, use=0, rtol=1e-10)
    phi1, i1 = held.solve_learned(net, use=3, rtol=1e-10)
    phi4, i4 = held.solve_learned(net, use=4, rtol=1e-10)   # closed-form diagonal
    assert i0["status"] == 0 and i1["status"] == 0 and i4["status"] == 0
    assert i1["iters"] < 0.9 * i0["iters"], (i0, i1, i4)
    assert _rel(phi4.cpu().numpy(), phi0.cpu().numpy()) < 1e-8
    a, b = phi1.cpu().numpy(), phi0.cpu().numpy()
    assert _rel(a, b) < 1e-8
    # the plain path afterwards is untouched: same iterations as before
    phi2, i2 = held.solve_learned(net, use=0, rtol=1e-10)
    assert i2["iters"] == i0["iters"] and np.array_equal(phi2.cpu().numpy(), b)


def test_rebuilt_context_uses_the_new_graph():
    """A context rebuilt for another particle set gives the network the new
    system's graph (same loss as a fresh context), even when the node count
    repeats."""
    from paper_1603_04039_gb300 import APCloud, MPNN
    net = MPNN(theta=_test_params(4).astype(np.float32))
    x, y, z, q = inputs.beam_with_halo(20000, 51)
    ap = APCloud(max_depth=5, c_refine=0.3)
    ap.build_octree(_t(x), _t(y), _t(z))
    ap.stencils()
    ap.deposit(q=_t(q), rtol=1e-12)
    net.loss(ap)
    # the same particles mirrored: the same node count, another node order
    ap.build_octree(_t(-x), _t(y), _t(z))
    ap.stencils()
    ap.deposit(q=_t(q), rtol=1e-12)
    again = net.loss(ap)
    fresh = APCloud(max_depth=5, c_refine=0.3)
    fresh.build_octree(_t(-x), _t(y), _t(z))
    fresh.stencils()
    fresh.deposit(q=_t(q), rtol=1e-12)
    assert again == net.loss(fresh)
