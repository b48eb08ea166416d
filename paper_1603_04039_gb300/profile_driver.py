"""Small, bounded runs of the library for profilers (ncu): one workload, a
fixed amount of work, exit 0.  Usage:

    python -m paper_1603_04039_gb300.profile_driver solve  [iters] [fp64|mixed] [sorted]
    python -m paper_1603_04039_gb300.profile_driver mpnn   [steps]
    python -m paper_1603_04039_gb300.profile_driver batch  [iters] [sorted]

`solve`: the 1e7-particle depth-10 beam (1.05e6 nodes), tree, stencils,
deposit, then `iters` Arnoldi steps of the Poisson solve (GMRES(30),
polynomial preconditioner degree 16); `sorted` runs the sweeps on the
width-sorted matrix with the shape the autotuner picks for it (128 threads,
two 4-entry chunks in flight; 2 nodes per stencil block).  `mpnn`: `steps` training steps of the
learned preconditioner on a 2e5-particle depth-8 beam.  `batch`: the 64-beam
depth-9 batch, then `iters` Arnoldi steps (`sorted`: width-sorted sweeps at
the autotuner's batch shape, 512 threads, one chunk in flight).
"""
from __future__ import annotations

import sys

import torch

from . import APCloud, MPNN, inputs


def _put(*arrays):
    return [torch.from_numpy(a).to("cuda:0") for a in arrays]


def solve(iters=400, precision="mixed", sorted_sweeps=False):
    x, y, z, q = inputs.beam_with_halo(10_000_000, 1)
    tx, ty, tz, tq = _put(x, y, z, q)
    ap = APCloud(max_depth=10, c_refine=0.043, precision=precision, poly_degree=16, poly_omega=1.0)
    if sorted_sweeps:
        ap.set_launch_shape(spmv_block=128, wls_warps=2, spmv_unroll=4, sweep_sorted=1)
    ap.build_octree(tx, ty, tz)
    ap.stencils()
    ap.deposit(q=tq, rtol=1e-10)
    ap.solve(rtol=1e-30, max_iter=iters)
    torch.cuda.synchronize()


def mpnn(steps=3):
    x, y, z, q = inputs.beam_with_halo(200_000, 3)
    tx, ty, tz, tq = _put(x, y, z, q)
    ap = APCloud(max_depth=8, c_refine=0.1)
    ap.build_octree(tx, ty, tz)
    ap.stencils()
    ap.deposit(q=tq, rtol=1e-10)
    net = MPNN(seed=1)
    for _ in range(steps):
        net.loss(ap, backward=True)
        net.adam(ap, 1e-3)
    torch.cuda.synchronize()


def batch(iters=300, sorted_sweeps=False):
    x, y, z, q, offs, _ = inputs.beam_batch(64, 1)
    tx, ty, tz, tq = _put(x, y, z, q)
    ap = APCloud(max_depth=9, c_refine=0.05, precision="mixed", poly_degree=16, poly_omega=1.0)
    if sorted_sweeps:
        ap.set_launch_shape(spmv_block=512, wls_warps=8, spmv_unroll=1, sweep_sorted=1)
    ap.build_octree_batched(tx, ty, tz, offs)
    ap.stencils()
    ap.deposit(q=tq, rtol=1e-10)
    ap.solve(rtol=1e-30, max_iter=iters)
    torch.cuda.synchronize()


if __name__ == "__main__":
    what = sys.argv[1] if len(sys.argv) > 1 else "solve"
    rest = sys.argv[2:]
    if what == "solve":
        solve(int(rest[0]) if rest else 400, rest[1] if len(rest) > 1 else "mixed",
              len(rest) > 2 and rest[2] == "sorted")
    elif what == "mpnn":
        mpnn(int(rest[0]) if rest else 3)
    elif what == "batch":
        batch(int(rest[0]) if rest else 300, len(rest) > 1 and rest[1] == "sorted")
    else:
        raise SystemExit("unknown run %r" % what)
