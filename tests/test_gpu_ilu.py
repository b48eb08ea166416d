"""ILU(0)-preconditioned GMRES, the comparison baseline of the learned
preconditioner, on the GPU (FP64 form).  The Poisson system of a small beam is
solved to rtol 1e-12: the true residual, computed with the oracle-checked
matrix product, meets the tolerance; the solution agrees with the Jacobi
solve of the same system; ILU(0) needs fewer Arnoldi steps than Jacobi; the
mixed form and batches are refused."""
import numpy as np
import pytest
import torch

from paper_1603_04039_gb300 import inputs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("n,depth,c,seed", [(20000, 5, 0.3, 3), (100000, 6, 0.5, 2)])
def test_ilu0_gmres_solves_the_poisson_system(n, depth, c, seed):
    from paper_1603_04039_gb300 import APCloud
    x, y, z, q = inputs.beam_with_halo(n, seed)
    ap = APCloud(max_depth=depth, c_refine=c, precision="fp64", poly_degree=1)
    ap.build_octree(_t(x), _t(y), _t(z))
    ap.stencils()
    b = _t(np.random.default_rng(seed).normal(size=ap.n_nodes))
    xj, ij = ap.solve_system("A", b, rtol=1e-12, max_iter=200000)
    xi, ii = ap.solve_system_ilu0("A", b, rtol=1e-12, max_iter=200000)
    assert ij["status"] == 0 and ii["status"] == 0 and ii["relres"] <= 1e-12
    bn = np.linalg.norm(b.cpu().numpy())
    r = (b - ap.matvec("A", xi)).cpu().numpy()
    assert np.linalg.norm(r) <= 2e-12 * bn
    assert float(torch.linalg.norm(xi - xj) / torch.linalg.norm(xj)) < 1e-6
    assert ii["iters"] < ij["iters"]
    assert ii["levels_lower"] >= 1 and ii["levels_upper"] >= 1 and ii["nnz"] > ap.n_nodes
    # the density system too
    xd, idn = ap.solve_system_ilu0("B", b, rtol=1e-12, max_iter=200000)
    rd = (b - ap.matvec("B", xd)).cpu().numpy()
    assert idn["status"] == 0 and np.linalg.norm(rd) <= 2e-12 * bn
    ap.close()


def test_ilu0_refuses_mixed_form_and_batches():
    from paper_1603_04039_gb300 import APCloud, APCloudError
    x, y, z, q = inputs.beam_with_halo(20000, 4)
    ap = APCloud(max_depth=5, c_refine=0.3, precision="mixed")
    ap.build_octree(_t(x), _t(y), _t(z))
    ap.stencils()
    b = torch.ones(ap.n_nodes, dtype=torch.float64, device=DEV)
    with pytest.raises(APCloudError):
        ap.solve_system_ilu0("A", b)
    ap.close()
    xs, ys, zs, qs, offs, _ = inputs.beam_batch(3, 5, n_lo=2000, n_hi=4000)
    ab = APCloud(max_depth=5, c_refine=0.3, precision="fp64")
    ab.build_octree_batched(_t(xs), _t(ys), _t(zs), offs)
    ab.stencils()
    with pytest.raises(APCloudError):
        ab.solve_system_ilu0("A", torch.ones(ab.n_nodes, dtype=torch.float64, device=DEV))
    ab.close()
