"""Failure paths of the C ABI, made on the host (no GPU fault is provoked).

  * A Krylov solve that reaches max_iter returns the warning
    APCLOUD_W_NOT_CONVERGED with its iteration count and the recomputed
    relative residual filled in; its outputs stay usable.
  * A device allocator that fails on its k-th call makes the call that
    needed the memory return APCLOUD_E_NOMEM (apcloud_create included), and
    destroying the context afterwards returns every byte it had taken.
  * The binding's default allocator is PyTorch's caching allocator: the
    context's buffers come from the same pool as the caller's tensors.
"""
import numpy as np
import pytest
import torch

from paper_1603_04039_gb300 import inputs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _pipeline(ap, x, y, z, q, precision):
    ap.build_octree(_t(x), _t(y), _t(z))
    ap.stencils()
    ap.deposit(q=_t(q), rtol=1e-10)
    ap.solve(rtol=1e-10)
    ap.gather_field()


@pytest.mark.parametrize("precision,pdeg", [("fp64", 1), ("mixed", 16)])
def test_max_iter_reached_is_a_warning(precision, pdeg):
    from paper_1603_04039_gb300 import APCloud
    x, y, z, q = inputs.beam_with_halo(50000, 3)
    ap = APCloud(max_depth=6, c_refine=0.6, precision=precision, poly_degree=pdeg, poly_omega=1.0)
    ap.build_octree(_t(x), _t(y), _t(z))
    ap.stencils()
    rho, ir = ap.deposit(q=_t(q), rtol=1e-10)
    assert ir["status"] == 0
    phi, ip = ap.solve(rtol=1e-14, max_iter=1)
    assert ip["status"] == 1                          # APCLOUD_W_NOT_CONVERGED
    assert ip["iters"] == 1 and ip["restarts"] >= 1
    assert 1e-14 < ip["relres"] < 1.0                 # one Arnoldi step reduces the residual somewhat
    assert torch.isfinite(phi).all()
    # the reported residual is that of the returned iterate: b = c rho~ on
    # interior rows (c = 1), g = 0 on boundary rows
    b = rho.clone()
    b[ap.n_int:] = 0.0
    r = b - ap.matvec("A", phi)
    assert abs(float(torch.linalg.norm(r) / torch.linalg.norm(b)) - ip["relres"]) <= 1e-6 * ip["relres"]
    # the context stays usable: the same solve to convergence
    phi2, ip2 = ap.solve(rtol=1e-10, max_iter=100000)
    assert ip2["status"] == 0 and ip2["relres"] <= 1e-10
    ap.gather_field()


def test_allocation_failure_returns_nomem_without_leaks():
    from paper_1603_04039_gb300 import APCloud, APCloudError
    from paper_1603_04039_gb300._binding import TorchAllocator
    x, y, z, q = inputs.beam_with_halo(20000, 5)
    for precision in ("fp64", "mixed"):
        pdeg = 16 if precision == "mixed" else 1
        # allocations of a whole pipeline, then a failure at a spread of them
        counter = TorchAllocator(DEV)
        ap = APCloud(max_depth=5, c_refine=0.5, precision=precision, poly_degree=pdeg, poly_omega=1.0,
                     allocator=counter)
        _pipeline(ap, x, y, z, q, precision)
        total = counter.allocs
        ap.close()
        assert counter.live == {} and counter.frees == counter.allocs
        assert total > 10
        ks = sorted(set([1, 2, 3, 4, 5] + list(np.linspace(6, total, 12).astype(int))))
        for k in ks:
            alloc = TorchAllocator(DEV, fail_at=k)
            ap = None
            with pytest.raises(APCloudError) as e:
                ap = APCloud(max_depth=5, c_refine=0.5, precision=precision, poly_degree=pdeg, poly_omega=1.0,
                             allocator=alloc)
                _pipeline(ap, x, y, z, q, precision)
            assert e.value.status == -5, (precision, k, str(e.value))
            if ap is not None:
                ap.close()
            torch.cuda.synchronize()
            assert alloc.live == {}, (precision, k, alloc.live)


def test_default_allocator_is_torch_pool():
    from paper_1603_04039_gb300 import APCloud
    from paper_1603_04039_gb300._binding import TorchAllocator
    x, y, z, q = inputs.beam_with_halo(20000, 6)
    before = torch.cuda.memory_allocated(DEV)
    ap = APCloud(max_depth=5, c_refine=0.5)
    assert isinstance(ap.allocator, TorchAllocator)
    _pipeline(ap, x, y, z, q, "fp64")
    held = torch.cuda.memory_allocated(DEV) - before
    assert held >= ap.allocator.live_bytes > 0
    ap.close()
    assert ap.allocator.live == {}
