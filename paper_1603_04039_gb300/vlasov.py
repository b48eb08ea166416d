"""Vlasov-Poisson time stepping with the AP-Cloud field solve.

The paper's title problem: particles move in their own electrostatic field.
It prescribes no integrator; this driver uses the kick-drift-kick leapfrog
(velocity Verlet), and every step rebuilds the octree, stencils and both
linear systems for the moved particles (Section 4 onward), as the method
requires.  Two library contexts alternate so that the new solve is
warm-started from the previous potential interpolated onto the new nodes.

Orchestration only: the push, the interpolation, the field energy and the
whole field solve run in the library's CUDA kernels.
"""
from __future__ import annotations

import torch

from ._binding import APCloud


class VlasovPoisson:
    """Particles (device FP64 tensors, updated in place) with charge q (tensor or
    uniform scalar) and charge-to-mass ratio qm.  Field convention of the paper:
    Lap phi = c rho, E = grad phi, so the acceleration is qm * E."""

    def __init__(self, x, y, z, vx, vy, vz, q=None, q_uniform=None, qm=1.0, rtol=1e-10, max_iter=100000,
                 warm_start=True, net=None, net_use=1, **params):
        self.x, self.y, self.z, self.vx, self.vy, self.vz = x, y, z, vx, vy, vz
        self.q = q
        self.q_uniform = (1.0 / x.numel()) if (q is None and q_uniform is None) else q_uniform
        self.qm = qm
        self.rtol, self.max_iter = rtol, max_iter
        self.warm_start = warm_start
        # learned preconditioner for the Poisson solves (bits of apcloud_solve_learned's `use`)
        self.net, self.net_use = net, net_use
        self.ctx = [APCloud(**params), APCloud(**params)]
        self.cur = 0
        n = x.numel()
        self.E = tuple(torch.empty(n, dtype=torch.float64, device=x.device) for _ in range(3))
        self.phi_p = torch.empty(n, dtype=torch.float64, device=x.device)
        self.info = {}
        self._solve(warm=False)

    @property
    def ap(self):
        return self.ctx[self.cur]

    def _solve(self, warm):
        ap = self.ap
        ap.build_octree(self.x, self.y, self.z)
        ap.stencils()
        _, ir = ap.deposit(q=self.q, q_uniform=self.q_uniform, rtol=self.rtol, max_iter=self.max_iter)
        phi0 = None
        if warm and self.warm_start:
            xyz = ap.get_nodes()["xyz"]
            px, py, pz = (xyz[:, d].contiguous() for d in range(3))
            phi0 = self.ctx[1 - self.cur].interpolate_potential(px, py, pz)
            phi0[ap.n_int:] = 0.0          # Dirichlet data g = 0 on the boundary nodes
        if self.net is not None:
            _, ip = ap.solve_learned(self.net, use=self.net_use, phi0=phi0, rtol=self.rtol, max_iter=self.max_iter)
        else:
            _, ip = ap.solve(phi0=phi0, rtol=self.rtol, max_iter=self.max_iter)
        ap.gather_field((self.phi_p,) + self.E)
        self.info = {"iters_rho": ir["iters"], "iters_phi": ip["iters"], "relres_phi": ip["relres"],
                     "n_nodes": ap.n_nodes}

    def step(self, dt):
        """v += qm dt/2 E; x += dt v; new field; v += qm dt/2 E."""
        self.ap.push_particles(self.x, self.y, self.z, self.vx, self.vy, self.vz, self.E, self.qm * dt / 2, dt)
        self.cur = 1 - self.cur
        self._solve(warm=True)
        self.ap.push_particles(self.x, self.y, self.z, self.vx, self.vy, self.vz, self.E, self.qm * dt / 2, 0.0)

    def energies(self):
        """(field energy 1/2 sum |grad phi|^2 h^3, kinetic energy 1/2 sum m v^2)."""
        w = self.ap.field_energy()
        m = (self.q if self.q is not None else self.q_uniform) / self.qm
        v2 = self.vx * self.vx + self.vy * self.vy + self.vz * self.vz
        k = 0.5 * float((m * v2).sum()) if torch.is_tensor(m) else 0.5 * m * float(v2.sum())
        return w, k
