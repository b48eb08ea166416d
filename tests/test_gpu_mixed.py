"""The mixed-precision form against the FP64 oracle.

FP32 stencils (with FP64 refactorisation of blocks whose FP32 condition
estimate min|R_ii|/max|R_ii| is below fp32_rcond_min, 1e-3 by default) and
FP32 GMRES iterations inside an FP64 iterative-refinement
loop.  Integer results stay bit-exact (the selection is integer arithmetic
and the accept/reject tests agree unless a value sits on a threshold); the
fields must match the FP64 oracle within a relative L2 of 1e-6 (FP32
weights perturb the operator by ~1e-7 relative and the rows stay exactly
consistent, so the solution moves by ~1e-7).
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


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("n,depth,c,seed", [(100000, 6, 1.0, 1), (100000, 6, 0.5, 2), (20000, 5, 0.3, 3)])
def test_mixed_matches_fp64_oracle(n, depth, c, seed):
    from paper_1603_04039_gb300 import APCloud
    x, y, z, q = inputs.beam_with_halo(n, seed)
    ap = APCloud(max_depth=depth, c_refine=c, precision="mixed")
    ap.build_octree(_t(x), _t(y), _t(z))
    ap.stencils()
    o = oracle.Oracle(max_depth=depth, c_refine=c)
    o.build(x, y, z)
    w = o.stencils()
    g = {k: v.cpu().numpy() for k, v in ap.get_stencils().items()}
    assert np.array_equal(g["nbr"], w["nbr"]) and np.array_equal(g["m"], w["m"])
    scale = np.abs(w["lap"]).max(axis=1, keepdims=True)
    assert np.all(np.abs(g["lap"] - w["lap"]) <= 1e-5 * scale)
    rho, ir = ap.deposit(q=_t(q), rtol=1e-10)
    phi, ip = ap.solve(rtol=1e-10)
    php, ex, ey, ez = ap.gather_field()
    assert ir["status"] == 0 and ip["status"] == 0 and ip["relres"] <= 1e-10
    ref = o.run(x, y, z, q=q, rtol=1e-12)
    assert rel(rho.cpu().numpy(), ref["rho"]) < 1e-6
    assert rel(phi.cpu().numpy(), ref["phi"]) < 1e-6
    assert rel(php.cpu().numpy(), ref["phi_p"]) < 1e-6
    for a, b in ((ex, ref["ex"]), (ey, ref["ey"]), (ez, ref["ez"])):
        assert rel(a.cpu().numpy(), b) < 1e-6


def test_mixed_refinement_reaches_fp64_residual():
    """Iterative refinement drives the FP64 residual of the (FP32-built)
    system to 1e-12, beyond what FP32 iterations alone can reach."""
    from paper_1603_04039_gb300 import APCloud
    x, y, z, q = inputs.beam_with_halo(100000, 4)
    ap = APCloud(max_depth=6, c_refine=0.7, precision="mixed")
    ap.build_octree(_t(x), _t(y), _t(z))
    ap.stencils()
    b = torch.from_numpy(np.random.default_rng(0).normal(size=ap.n_nodes)).to(DEV)
    xs, info = ap.solve_system("A", b, rtol=1e-12, max_iter=50000)
    assert info["status"] == 0 and info["relres"] <= 1e-12
    r = (b - ap.matvec("A", xs)).cpu().numpy()
    assert np.linalg.norm(r) <= 2e-12 * np.linalg.norm(b.cpu().numpy())


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-6)])
def test_polynomial_preconditioner_matches_oracle(precision, tol):
    """The Jacobi-Neumann polynomial preconditioner changes the Krylov path, not
    the solution: the fields still match the oracle's plain Jacobi solve."""
    from paper_1603_04039_gb300 import APCloud
    n = 100000
    x, y, z, q = inputs.beam_with_halo(n, 5)
    ap = APCloud(max_depth=6, c_refine=0.5, precision=precision, poly_degree=16, poly_omega=1.0)
    ap.build_octree(_t(x), _t(y), _t(z))
    ap.stencils()
    rtol = 1e-13 if precision == "fp64" else 1e-10
    rho, ir = ap.deposit(q=_t(q), rtol=rtol)
    phi, ip = ap.solve(rtol=rtol)
    php, ex, ey, ez = ap.gather_field()
    assert ip["status"] == 0 and ip["relres"] <= rtol
    ref = oracle.Oracle(max_depth=6, c_refine=0.5).run(x, y, z, q=q, rtol=1e-13)
    assert rel(phi.cpu().numpy(), ref["phi"]) < tol
    assert rel(php.cpu().numpy(), ref["phi_p"]) < tol
    assert rel(ex.cpu().numpy(), ref["ex"]) < tol
    # and it needs far fewer Arnoldi steps than Jacobi alone
    ap1 = APCloud(max_depth=6, c_refine=0.5, precision=precision)
    ap1.build_octree(_t(x), _t(y), _t(z))
    ap1.stencils()
    ap1.deposit(q=_t(q), rtol=rtol)
    _, ip1 = ap1.solve(rtol=rtol)
    assert ip["iters"] * 4 < ip1["iters"]


@pytest.mark.parametrize("restart", [8, 30, 40])
def test_gram_schmidt_forms_match_oracle(restart):
    """The mixed polynomial form orthogonalises by DCGS2 (one reduction per
    Arnoldi step, the second projection delayed a step) while a restart cycle
    fits its 2 j + 3 partial sums in 64 slots (restart <= 31), by CGS2 above
    that: short and long cycles of both reach the oracle's fields, and the two
    forms need about the same number of Arnoldi steps."""
    from paper_1603_04039_gb300 import APCloud
    x, y, z, q = inputs.beam_with_halo(100000, 6)
    ap = APCloud(max_depth=6, c_refine=0.5, precision="mixed", poly_degree=16, poly_omega=1.0, restart=restart)
    ap.build_octree(_t(x), _t(y), _t(z))
    ap.stencils()
    rho, ir = ap.deposit(q=_t(q), rtol=1e-10)
    phi, ip = ap.solve(rtol=1e-10)
    php, ex, ey, ez = ap.gather_field()
    assert ir["status"] == 0 and ip["status"] == 0 and ip["relres"] <= 1e-10
    ref = oracle.Oracle(max_depth=6, c_refine=0.5).run(x, y, z, q=q, rtol=1e-13)
    for a, k in ((phi, "phi"), (php, "phi_p"), (ex, "ex"), (ey, "ey"), (ez, "ez")):
        assert rel(a.cpu().numpy(), ref[k]) < 1e-6, k
    # the same cycles at restart 40 (CGS2) and 30 (DCGS2) need about as many steps
    if restart == 40:
        ap30 = APCloud(max_depth=6, c_refine=0.5, precision="mixed", poly_degree=16, poly_omega=1.0, restart=30)
        ap30.build_octree(_t(x), _t(y), _t(z))
        ap30.stencils()
        ap30.deposit(q=_t(q), rtol=1e-10)
        _, ip30 = ap30.solve(rtol=1e-10)
        assert 0.7 * ip30["iters"] <= ip["iters"] <= 1.5 * ip30["iters"] + 4


@pytest.mark.parametrize("rcond_min", [0.05, 2.0])
def test_fp64_refactorisation_of_uncertified_blocks(rcond_min):
    """Mixed form: a block whose FP32 condition estimate falls below
    fp32_rcond_min is refactorised in FP64.  Raising the limit from 1e-3 sends
    some (0.05) or every (2, above any ratio) block down that branch; each such
    row then carries FP64 accuracy (1e-11 of the row's largest weight, like
    the FP64 form) where FP32 rows agree only to ~1e-6, and the fields still
    match the FP64 oracle within 1e-6."""
    from paper_1603_04039_gb300 import APCloud
    n, depth, c = 100000, 6, 0.5
    x, y, z, q = inputs.beam_with_halo(n, 2)
    ap = APCloud(max_depth=depth, c_refine=c, precision="mixed", fp32_rcond_min=rcond_min)
    ap.build_octree(_t(x), _t(y), _t(z))
    ap.stencils()
    nfp64 = ap.sizes()["fp64_stencils"]
    o = oracle.Oracle(max_depth=depth, c_refine=c)
    o.build(x, y, z)
    w = o.stencils()
    g = {k: v.cpu().numpy() for k, v in ap.get_stencils().items()}
    assert np.array_equal(g["nbr"], w["nbr"]) and np.array_equal(g["m"], w["m"])
    dscale = np.abs(w["D"]).max(axis=(1, 2))
    derr = np.abs(g["D"] - w["D"]).max(axis=(1, 2)) / dscale
    exact = int(np.sum(derr <= 1e-11))
    if rcond_min >= 1.0:
        assert nfp64 == ap.n_int and exact == ap.n_int
    else:
        assert 0 < nfp64 < ap.n_int
        assert exact >= nfp64
        assert np.all(derr <= 1e-5)
    rho, ir = ap.deposit(q=_t(q), rtol=1e-10)
    phi, ip = ap.solve(rtol=1e-10)
    php, ex, ey, ez = ap.gather_field()
    ref = o.run(x, y, z, q=q, rtol=1e-12)
    assert rel(phi.cpu().numpy(), ref["phi"]) < 1e-6
    assert rel(php.cpu().numpy(), ref["phi_p"]) < 1e-6
    for a, b in ((ex, ref["ex"]), (ey, ref["ey"]), (ez, ref["ez"])):
        assert rel(a.cpu().numpy(), b) < 1e-6
