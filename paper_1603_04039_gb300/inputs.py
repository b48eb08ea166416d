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


def beam_with_halo_device(n: int, seed: int, device, sigma: float = 0.05, halo_frac: float = 0.1,
                          r0: float = 0.3, r1: float = 0.5, lo: float = -1.0, hi: float = 1.0):
    """The beam-with-halo law drawn on a CUDA device with torch's generator
    (a training-set sampler: a million-node system per draw without a host
    round trip).  Same law as beam_with_halo, another random stream: core
    draws outside the domain are clamped instead of redrawn (the core's
    sigma puts the walls 20 sigma away) and the particles come core first,
    halo second (the tree build orders them itself).  Returns torch float64
    tensors (x, y, z, q) on the device."""
    import torch
    n = int(n)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    n_halo = int(round(halo_frac * n))
    core = torch.randn(n - n_halo, 3, generator=g, device=device, dtype=torch.float64) * sigma
    u = torch.rand(n_halo, 3, generator=g, device=device, dtype=torch.float64)
    rad = torch.pow(r0 ** 3 + u[:, 0] * (r1 ** 3 - r0 ** 3), 1.0 / 3.0)
    cz = 2.0 * u[:, 1] - 1.0
    ph = 2.0 * np.pi * u[:, 2]
    st = torch.sqrt(torch.clamp(1.0 - cz * cz, min=0.0))
    halo = torch.stack([rad * st * torch.cos(ph), rad * st * torch.sin(ph), rad * cz], dim=1)
    pts = torch.clamp(torch.cat([core, halo], dim=0), lo, hi)
    q = torch.full((n,), 1.0 / n, device=device, dtype=torch.float64)
    return pts[:, 0].contiguous(), pts[:, 1].contiguous(), pts[:, 2].contiguous(), q


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


def beam_batch_params(n_beams: int, seed: int = 1, n_lo: float = 1e4, n_hi: float = 1e6):
    """Laws of a batch of independent beams (stream 6 of ``seed``, five uniforms
    per beam): particle count log-uniform in [n_lo, n_hi], core sigma uniform
    in [0.02, 0.1], halo fraction uniform in [0.01, 0.2], halo shell radii
    uniform in [0.2, 0.8] (sorted).  Beam b draws its particles with seed b + 1.
    """
    u = uniforms(seed, 6, 5 * int(n_beams)).reshape(-1, 5)
    out = []
    for b in range(int(n_beams)):
        r = sorted((0.2 + 0.6 * u[b, 3], 0.2 + 0.6 * u[b, 4]))
        out.append(dict(n=int(round(n_lo * (n_hi / n_lo) ** u[b, 0])), sigma=0.02 + 0.08 * u[b, 1],
                        halo_frac=0.01 + 0.19 * u[b, 2], r0=r[0], r1=r[1], seed=b + 1))
    return out


def beam_batch(n_beams: int, seed: int = 1, n_lo: float = 1e4, n_hi: float = 1e6):
    """Concatenated particles of a beam batch: (x, y, z, q, offsets, params).
    Beam b occupies offsets[b]:offsets[b+1] and carries charge 1/N_b per
    particle, so every beam has total charge 1."""
    params = beam_batch_params(n_beams, seed, n_lo, n_hi)
    xs, ys, zs, qs = [], [], [], []
    offsets = [0]
    for p in params:
        x, y, z, q = beam_with_halo(p["n"], p["seed"], sigma=p["sigma"], halo_frac=p["halo_frac"],
                                    r0=p["r0"], r1=p["r1"])
        xs.append(x); ys.append(y); zs.append(z); qs.append(q)
        offsets.append(offsets[-1] + p["n"])
    cat = lambda a: np.ascontiguousarray(np.concatenate(a)) if a else np.zeros(0)
    return cat(xs), cat(ys), cat(zs), cat(qs), np.array(offsets, dtype=np.int64), params
