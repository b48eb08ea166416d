"""Converged oracle solves of the benchmark workloads -- TEST INFRASTRUCTURE ONLY.

Runs the CPU oracle's whole electrostatic solve (tree, stencils, density
system, Poisson system by GMRES(30) with Jacobi to relative residual 1e-10,
derivatives and gather) on a benchmark workload and records, per workload,
the Krylov iteration counts it needed, the residuals it reached and the time
each stage took.  The benchmark's CPU baseline times a bounded sample of the
same oracle run (the whole pipeline with one GMRES restart cycle of the
Poisson solve) and scales the sampled cycle to these counts; this file is
where those counts come from, so they are the oracle's own.

    python -m oracle.solve_counts beam_halo_1e7_depth10 [seed]

writes oracle/solve_counts.json (merged with the entries already there).
A solve of the 1.05e6-node system takes several minutes on one core.
"""
from __future__ import annotations

import json
import os
import platform
import sys
import time

import numpy as np

from . import Oracle

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "solve_counts.json")
RTOL = 1e-10
# name: (particles, max_depth, c_refine); the beam-with-halo law of the benchmark
WORKLOADS = {
    "beam_halo_1e7_depth10": (10_000_000, 10, 0.043),
    "beam_halo_1e5_depth6": (100_000, 6, 1.0),
}


def run(workload: str, seed: int = 1) -> dict:
    sys.path.insert(0, os.path.dirname(HERE))
    from paper_1603_04039_gb300 import inputs
    npart, depth, c = WORKLOADS[workload]
    x, y, z, q = inputs.beam_with_halo(npart, seed)
    o = Oracle(max_depth=depth, c_refine=c)
    t = {}
    t0 = time.perf_counter(); o.build(x, y, z); t["build"] = time.perf_counter() - t0
    t0 = time.perf_counter(); o.stencils(); t["stencils"] = time.perf_counter() - t0
    t0 = time.perf_counter(); rhs, _, _ = o.density_rhs(q); t["deposit"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    rho, it_r, rr_r, st_r = o.solve_density(rhs, rtol=RTOL, max_iter=200000)
    t["solve_rho"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    phi, it_p, rr_p, st_p = o.solve_poisson(rho, rtol=RTOL, max_iter=200000)
    t["solve_phi"] = time.perf_counter() - t0
    t0 = time.perf_counter(); o.gather(phi); t["gather"] = time.perf_counter() - t0
    return {"workload": workload, "seed": seed, "n_interior": o.n_int, "n_boundary": o.n_bnd, "rtol": RTOL,
            "restart": 30, "iters_rho": it_r, "relres_rho": rr_r, "status_rho": st_r,
            "iters_phi": it_p, "relres_phi": rr_p, "status_phi": st_p,
            "stage_s": {k: round(v, 3) for k, v in t.items()},
            "host": "%s %s" % (platform.machine(), platform.processor() or platform.platform()),
            "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}


def load() -> dict:
    try:
        with open(OUT) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def main(argv):
    workload = argv[1] if len(argv) > 1 else "beam_halo_1e7_depth10"
    seed = int(argv[2]) if len(argv) > 2 else 1
    rec = run(workload, seed)
    data = load()
    data["%s/seed%d" % (workload, seed)] = rec
    tmp = OUT + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, OUT)
    print(json.dumps(rec))


if __name__ == "__main__":
    main(sys.argv)
