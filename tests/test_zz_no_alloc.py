"""The allocation-free GMRES entry point agrees with the allocating one.

apcloud_solve_system_noalloc is for callers that cannot allocate device
memory once their setup is done: a host that hands out all device memory up
front (a fixed budget, or a memory manager that owns the device and refuses
cudaMalloc), or a real-time loop that cannot afford a pool growing mid-run.
Its Krylov scratch is a fixed 20 MiB device array inside the library.  This
file runs last so that a failure here never hides another test; it passes
both alone in a fresh process and after the rest of the suite (the shared
array keeps the previous call's contents).
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_1603_04039_gb300 import inputs

pytestmark = pytest.mark.gpu


def _context(**kw):
    from paper_1603_04039_gb300 import APCloud
    from paper_1603_04039_gb300._binding import TorchAllocator
    dev = torch.device("cuda:0")
    x, y, z, q = inputs.beam_with_halo(100000, 1)
    alloc = TorchAllocator(dev)
    ap = APCloud(max_depth=6, c_refine=1.0, allocator=alloc, **kw)
    ap.build_octree(*(torch.from_numpy(a).to(dev) for a in (x, y, z)))
    ap.stencils()
    return ap, alloc, dev


def _noalloc(ap, which, b, x):
    from paper_1603_04039_gb300._binding import SolveInfo, load
    lib = load()
    info = SolveInfo()
    st = lib.apcloud_solve_system_noalloc(ap._ctx, 1 if which == "A" else 0, C.c_void_p(b.data_ptr()),
                                          C.c_void_p(x.data_ptr()), 1e-12, 20000, C.byref(info))
    return st, info, lib.apcloud_last_error(ap._ctx).decode()


def test_noalloc_matches_allocating_solve_twice():
    ap, alloc, dev = _context()
    n = ap.n_nodes
    assert n <= 65536
    rng = np.random.default_rng(5)
    # calls in a row on different systems and data; the first one on a device
    # also looks up the scratch array's address, so the check that nothing is
    # allocated covers the calls after it
    for call, which in enumerate(("A", "B", "A")):
        b = torch.from_numpy(rng.normal(size=n)).to(dev)
        x0 = torch.from_numpy(rng.normal(size=n) * 0.1).to(dev)
        want, winfo = ap.solve_system(which, b, x0=x0, rtol=1e-12, max_iter=20000)
        x = x0.clone()
        torch.cuda.synchronize()
        # nothing may be allocated by the call: not through the context's
        # allocator, not through PyTorch's pool, not by cudaMalloc
        n_alloc = alloc.allocs
        torch_allocs = torch.cuda.memory_stats(dev).get("allocation.all.allocated", 0)
        free0, _ = torch.cuda.mem_get_info(dev)
        st, info, msg = _noalloc(ap, which, b, x)
        assert st == 0, msg
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info(dev)
        if call > 0:
            assert alloc.allocs == n_alloc
            assert torch.cuda.memory_stats(dev).get("allocation.all.allocated", 0) == torch_allocs
            assert free1 == free0
        got = x.cpu().numpy()
        ref = want.cpu().numpy()
        assert info.iters == winfo["iters"] and info.relres <= 1e-12
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref), call


@pytest.mark.parametrize("form", [dict(precision="mixed"), dict(poly_degree=8, poly_omega=1.0)])
def test_noalloc_refuses_other_solver_forms(form):
    """It runs FP64 Jacobi GMRES only; a context set up for another form is
    refused instead of being solved by a different algorithm."""
    ap, _, dev = _context(**form)
    b = torch.ones(ap.n_nodes, dtype=torch.float64, device=dev)
    x = torch.zeros_like(b)
    st, _, msg = _noalloc(ap, "A", b, x)
    assert st == -1 and "FP64 Jacobi" in msg


def test_noalloc_refuses_batch():
    from paper_1603_04039_gb300 import APCloud
    dev = torch.device("cuda:0")
    x, y, z, q, offs, _ = inputs.beam_batch(3, 4, n_lo=2000, n_hi=6000)
    ap = APCloud(max_depth=5, c_refine=1.0)
    ap.build_octree_batched(*(torch.from_numpy(a).to(dev) for a in (x, y, z)), offs)
    ap.stencils()
    assert ap.n_nodes <= 65536
    b = torch.ones(ap.n_nodes, dtype=torch.float64, device=dev)
    xx = torch.zeros_like(b)
    st, _, msg = _noalloc(ap, "A", b, xx)
    assert st == -1 and "single-beam" in msg


def test_noalloc_rejects_oversized_problem():
    from paper_1603_04039_gb300 import APCloud
    from paper_1603_04039_gb300._binding import APCloudError
    dev = torch.device("cuda:0")
    x, y, z, q = inputs.beam_with_halo(1000000, 2)
    ap = APCloud(max_depth=8, c_refine=0.08)          # ~1.1e5 nodes
    ap.build_octree(*(torch.from_numpy(a).to(dev) for a in (x, y, z)))
    ap.stencils()
    assert ap.n_nodes > 65536
    b = torch.ones(ap.n_nodes, dtype=torch.float64, device=dev)
    xx = torch.zeros_like(b)
    with pytest.raises(APCloudError) as e:
        ap.solve_system_noalloc("A", b, xx)
    assert e.value.status == -1 and "limit" in str(e.value)
