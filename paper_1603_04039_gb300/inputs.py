"""Seeded synthetic particle sets for the electrostatic solve.

This module holds random-number plumbing and sampling laws only; none of the
AP-Cloud arithmetic lives here.  Both the CUDA path and the CPU oracle read the
same arrays produced by these functions.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) used in counter form, output k of stream s is
mix(base_s + (k + 1) * gamma).  Uniform doubles take the top 53 bits.
Normals use the Box-Muller transform.

Beam-with-halo law (the accelerator-beam workload of Section 5): a Gaussian
core holding ``1 - halo_frac`` of the particles with standard deviation
``sigma`` in every coordinate, redrawn when a draw falls outside the domain,
and a halo of ``halo_frac`` of the particles spread uniformly in volume over
the spherical shell ``r0 <= r <= r1``.  Every particle carries charge 1/N so
that N q = 1 (Section 2).  Particles are returned in a seeded random order, the
order a caller would hand them over in.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def _base(seed: int, stream: int) -> np.uint64:
    s = _mix(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]
    return _mix(np.array([s ^ np.uint64(stream * 0x632BE59BD9B4E019 & 0xFFFFFFFFFFFFFFFF)],
                         dtype=np.uint64))[0]


def uniforms(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n uniform doubles in [0, 1) from counters offset..offset+n-1 of a stream."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = _mix(_base(seed, stream) + k * _GAMMA)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _normals(seed: int, stream: int, n: int, offset: int) -> np.ndarray:
    """n standard normals (Box-Muller), drawing 2*ceil(n/2) uniforms."""
    npair = (n + 1) // 2
    u = uniforms(seed, stream, 2 * npair, offset)
    u1 = 1.0 - u[0::2]          # (0, 1]
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    out = np.empty(2 * npair)
    out[0::2] = rad * np.cos(ang)
    out[1::2] = rad * np.sin(ang)
    return out[:n]


def beam_with_halo(n: int, seed: int, sigma: float = 0.05, halo_frac: float = 0.1,
                   r0: float = 0.3, r1: float = 0.5, lo: float = -1.0, hi: float = 1.0):
    """Return (x, y, z, q) float64 arrays of length n for the beam-with-halo law."""
    n = int(n)
    n_halo = int(round(halo_frac * n))
    n_core = n - n_halo
    core = np.empty((n_core, 3))
    todo = np.arange(n_core)
    offset = 0
    while todo.size:
        g = _normals(seed, 1, 3 * todo.size, offset).reshape(-1, 3) * sigma
        offset += 3 * todo.size + 1
        core[todo] = g
        inside = np.all((g >= lo) & (g <= hi), axis=1)
        todo = todo[~inside]
    u = uniforms(seed, 2, 3 * n_halo).reshape(-1, 3) if n_halo else np.zeros((0, 3))
    rad = np.cbrt(r0 ** 3 + u[:, 0] * (r1 ** 3 - r0 ** 3))
    cz = 2.0 * u[:, 1] - 1.0
    ph = 2.0 * np.pi * u[:, 2]
    st = np.sqrt(np.maximum(0.0, 1.0 - cz * cz))
    halo = np.stack([rad * st * np.cos(ph), rad * st * np.sin(ph), rad * cz], axis=1)
    pts = np.concatenate([core, halo], axis=0)
    order = np.argsort(uniforms(seed, 3, n), kind="stable")
    pts = np.clip(pts[order], lo, hi)
    q = np.full(n, 1.0 / n) if n else np.zeros(0)
    return (np.ascontiguousarray(pts[:, 0]), np.ascontiguousarray(pts[:, 1]),
            np.ascontiguousarray(pts[:, 2]), q)


def uniform_box(n: int, seed: int, lo: float = -1.0, hi: float = 1.0):
    """n points uniform in the cube [lo, hi]^3 with charge 1/n each."""
    u = uniforms(seed, 4, 3 * n).reshape(-1, 3)
    pts = lo + (hi - lo) * u
    q = np.full(n, 1.0 / n) if n else np.zeros(0)
    return (np.ascontiguousarray(pts[:, 0]), np.ascontiguousarray(pts[:, 1]),
            np.ascontiguousarray(pts[:, 2]), q)


def grid_points(depth: int, lo: float = -1.0, hi: float = 1.0):
    """One point at the centre of every cell of the uniform 2^depth grid."""
    k = 1 << depth
    c = lo + (np.arange(k) + 0.5) * ((hi - lo) / k)
    gx, gy, gz = np.meshgrid(c, c, c, indexing="ij")
    n = k ** 3
    return (gx.ravel().copy(), gy.ravel().copy(), gz.ravel().copy(), np.full(n, 1.0 / n))


def thermal_velocities(n: int, seed: int, sigma_v: float = 0.01):
    """(vx, vy, vz): independent N(0, sigma_v^2) components (stream 5)."""
    g = _normals(seed, 5, 3 * int(n), 0).reshape(-1, 3) * sigma_v if n else np.zeros((0, 3))
    return tuple(np.ascontiguousarray(g[:, d]) for d in range(3))
