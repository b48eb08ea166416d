"""Oracle side of the full-size parity checks -- TEST INFRASTRUCTURE ONLY.

Given one problem's particles and what the CUDA library produced for it (node
geometry, leaf particle ranges, stencil neighbour lists in the problem's own
node numbering, rho~ and phi at the nodes), this module builds the same
problem with the CPU oracle and reports:

  * whether node geometry, leaves and neighbour lists are bit-identical;
  * the relative residuals of the library's rho~ and phi in the oracle's own
    FP64 systems (Section 3.2): ||rho_M - B rho~|| / ||rho_M|| and
    ||b - A phi|| / ||b||, with b built from the oracle's own solve of the
    density system.  One sparse product per system stands in for an oracle
    Poisson solve, which would take minutes at a million nodes.

A plain function of numpy arrays, so a spawn-started process pool can run one
problem per worker.  Only the test suite and the benchmark's CPU leg use it.
"""
from __future__ import annotations

import time

import numpy as np

from . import Oracle


def _csr_mv(rp, col, val, x):
    return np.add.reduceat(val * x[col], rp[:-1])


def _relres(rp, col, val, x, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(b - _csr_mv(rp, col, val, x)) / nb) if nb > 0 else 0.0


def check(x, y, z, q, max_depth, c_refine, gpu, rtol_rho=1e-13):
    """gpu: dict with any of xyz [n][3], level [n], kind [n], key/first/count
    [n_int] (leaf key without beam bits, first particle relative to this
    problem), nbr [n_int][32] (this problem's numbering), m [n_int], and
    rho, phi_list (a list of potentials [n]).  Returns a dict of results."""
    t0 = time.perf_counter()
    o = Oracle(max_depth=max_depth, c_refine=c_refine)
    o.build(x, y, z)
    out = {"n_int": o.n_int, "n_bnd": o.n_bnd}
    same_size = "xyz" not in gpu or len(gpu["xyz"]) == o.n_nodes
    out["sizes_equal"] = bool(same_size)
    if not same_size:
        return out
    nd = o.nodes()
    if "xyz" in gpu:
        out["nodes_equal"] = bool(np.array_equal(gpu["xyz"], nd["xyz"]) and
                                  np.array_equal(gpu["level"], nd["level"]) and
                                  np.array_equal(gpu["kind"], nd["kind"]))
    if "key" in gpu:
        key, first, count = o.leaves()
        out["leaves_equal"] = bool(np.array_equal(gpu["key"], key) and np.array_equal(gpu["first"], first) and
                                   np.array_equal(gpu["count"], count))
    st = o.stencils()
    if "nbr" in gpu:
        out["nbr_equal"] = bool(np.array_equal(gpu["m"], st["m"]) and np.array_equal(gpu["nbr"], st["nbr"]))
        out["max_ring"] = int(st["ring"].max())
        out["m_hist"] = {int(k): int(v) for k, v in zip(*np.unique(st["m"], return_counts=True))}
    rhs, _, _ = o.density_rhs(q)
    if "rho" in gpu:
        out["relres_rho"] = _relres(*o.matrix("B"), gpu["rho"], rhs)
    if "phi_list" in gpu:
        rho, _, rr, _ = o.solve_density(rhs, rtol=rtol_rho)
        b = o.poisson_rhs(rho)
        A = o.matrix("A")
        out["relres_phi"] = [_relres(*A, p, b) for p in gpu["phi_list"]]
    out["seconds"] = time.perf_counter() - t0
    return out


def check_star(args):
    """check(*args): the form a process pool's map wants."""
    return check(*args)
