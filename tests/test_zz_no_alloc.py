"""The allocation-free GMRES entry point agrees with the allocating one.

apcloud_solve_system_noalloc serves callers that may not allocate device
memory after setup (stream capture, fixed-budget or externally managed
memory): its Krylov scratch is a fixed 20 MiB device array inside the
library.  This file runs last so that a failure here never hides another
test; it passes both alone in a fresh process and after the rest of the
suite (the shared array keeps the previous call's contents).
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_1603_04039_gb300 import inputs

pytestmark = pytest.mark.gpu


def _problem():
    from paper_1603_04039_gb300 import APCloud
    dev = torch.device("cuda:0")
    x, y, z, q = inputs.beam_with_halo(100000, 1)
    ap = APCloud(max_depth=6, c_refine=1.0)
    ap.build_octree(*(torch.from_numpy(a).to(dev) for a in (x, y, z)))
    ap.stencils()
    return ap, dev


def test_noalloc_matches_allocating_solve_twice():
    from paper_1603_04039_gb300._binding import SolveInfo, load
    lib = load()
    ap, dev = _problem()
    n = ap.n_nodes
    assert n <= 65536
    rng = np.random.default_rng(5)
    for call, which in enumerate(("A", "B")):          # two calls in a row, different systems and data
        b = torch.from_numpy(rng.normal(size=n)).to(dev)
        x0 = torch.from_numpy(rng.normal(size=n) * 0.1).to(dev)
        want, winfo = ap.solve_system(which, b, x0=x0, rtol=1e-12, max_iter=20000)
        x = x0.clone()
        info = SolveInfo()
        st = lib.apcloud_solve_system_noalloc(ap._ctx, 1 if which == "A" else 0, C.c_void_p(b.data_ptr()),
                                              C.c_void_p(x.data_ptr()), 1e-12, 20000, C.byref(info))
        assert st == 0, lib.apcloud_last_error(ap._ctx).decode()
        torch.cuda.synchronize()
        got = x.cpu().numpy()
        ref = want.cpu().numpy()
        assert info.iters == winfo["iters"] and info.relres <= 1e-12
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref), call


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
