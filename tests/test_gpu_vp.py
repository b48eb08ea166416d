"""Vlasov-Poisson leapfrog: 10 kick-drift-kick steps on the GPU against the same
steps driven by the CPU oracle's fields.

The reference integrator below is the textbook velocity Verlet written in
numpy; every field evaluation in it is a full oracle solve (tree, stencils,
density and Poisson systems, gather) for the current positions.  The GPU run
warm-starts each solve from the previous potential, which changes the Krylov
path but not the converged field.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1603_04039_gb300 import inputs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
N, DEPTH, C, DT, STEPS = 20000, 5, 0.5, 2e-3, 10


def _reference(x, y, z, vx, vy, vz):
    x, y, z, vx, vy, vz = (a.copy() for a in (x, y, z, vx, vy, vz))

    def field():
        o = oracle.Oracle(max_depth=DEPTH, c_refine=C)
        r = o.run(x, y, z, q_uniform=1.0 / N, rtol=1e-13)
        h = 2.0 / 2.0 ** o.nodes()["level"][: o.n_int].astype(float)
        w = 0.5 * float(((r["dphi"][:, :3] ** 2).sum(1) * h ** 3).sum())
        return (r["ex"], r["ey"], r["ez"]), w

    def drift(p, v):
        p += DT * v
        hi, lo = p > 1.0, p < -1.0
        p[hi] = 2.0 - p[hi]; v[hi] = -v[hi]
        p[lo] = -2.0 - p[lo]; v[lo] = -v[lo]
        np.clip(p, -1.0, 1.0, out=p)

    E, w = field()
    energies = [w]
    for _ in range(STEPS):
        for v, e in zip((vx, vy, vz), E):
            v += 0.5 * DT * e
        for p, v in zip((x, y, z), (vx, vy, vz)):
            drift(p, v)
        E, w = field()
        for v, e in zip((vx, vy, vz), E):
            v += 0.5 * DT * e
        energies.append(w)
    return (x, y, z, vx, vy, vz), np.array(energies)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 1e-5)])
def test_leapfrog_matches_oracle_steps(precision, tol):
    from paper_1603_04039_gb300 import VlasovPoisson
    x, y, z, q = inputs.beam_with_halo(N, 21)
    vx, vy, vz = inputs.thermal_velocities(N, 21, 0.01)
    ref_state, ref_w = _reference(x, y, z, vx, vy, vz)
    t = [torch.from_numpy(a.copy()).to(DEV) for a in (x, y, z, vx, vy, vz)]
    rtol = 1e-13 if precision == "fp64" else 1e-10
    vp = VlasovPoisson(*t, qm=1.0, rtol=rtol, max_depth=DEPTH, c_refine=C, precision=precision)
    energies = [vp.energies()[0]]
    for _ in range(STEPS):
        vp.step(DT)
        energies.append(vp.energies()[0])
    got = [a.cpu().numpy() for a in t]
    # positions and velocities after 10 steps
    for g, r in zip(got, ref_state):
        assert np.abs(g - r).max() <= tol * max(1.0, np.abs(r).max()), np.abs(g - r).max()
    assert np.allclose(energies, ref_w, rtol=tol, atol=0)
    # the particles did move and the warm start kept the solves cheap
    assert np.abs(got[0] - x).max() > 1e-5
    assert vp.info["relres_phi"] <= rtol
