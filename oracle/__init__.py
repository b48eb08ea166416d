"""CPU oracle for the AP-Cloud electrostatic solve -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it and
shares no code with it.  The arithmetic lives in ``apcloud_oracle.c`` (plain
C, FP64, single thread); this module only marshals numpy arrays through
ctypes and compiles the C file with gcc when the shared object is missing.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "apcloud_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

NCOL = 9
MMAX = 32          # widest stencil the oracle stores


def build(force: bool = False) -> str:
    """Compile the oracle (gcc -O2, no FMA contraction so x86 and Arm agree)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        P = C.c_void_p
        D = C.c_double
        I = C.c_int
        L = C.c_int64
        sig = {
            "or_create": (P, [P, P, I, D, I, I, D, D]),
            "or_destroy": (None, [P]),
            "or_last_error": (C.c_char_p, [P]),
            "or_build": (I, [P, P, P, P, L]),
            "or_n_interior": (L, [P]),
            "or_n_boundary": (L, [P]),
            "or_n_cells": (L, [P]),
            "or_get_nodes": (None, [P, P, P, P, P]),
            "or_get_leaves": (None, [P, P, P, P]),
            "or_get_boundary": (None, [P, P, P]),
            "or_get_order": (None, [P, P]),
            "or_get_cells": (None, [P, P, P, P, P]),
            "or_adjacency_size": (L, [P]),
            "or_get_adjacency": (None, [P, P, P]),
            "or_criterion_opens": (I, [L, I, I, D, D, D]),
            "or_wls": (I, [I, P, D, D, P, P, P, P]),
            "or_select": (I, [I, P, P, I, P]),
            "or_stencils": (I, [P]),
            "or_get_stencils": (None, [P, P, P, P, P, P, P]),
            "or_matrix_nnz": (L, [P]),
            "or_matrix": (None, [P, I, P, P, P]),
            "or_density_rhs": (D, [P, P, D, P, P]),
            "or_gmres": (I, [I, P, P, P, P, P, D, I, I, P, P]),
            "or_solve_density": (I, [P, P, P, D, I, I, P, P]),
            "or_solve_poisson": (I, [P, P, P, P, D, I, I, P, P]),
            "or_poisson_rhs": (None, [P, P, P, P]),
            "or_derivatives": (None, [P, P, P]),
            "or_gather": (None, [P, P, P, P, P, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleError(RuntimeError):
    pass


def criterion_opens(nprime: int, level: int, max_depth: int, lo: float, hi: float, c: float) -> bool:
    """Error-balance test of Section 4.3 for one cell (k = 2)."""
    return bool(_load().or_criterion_opens(int(nprime), int(level), int(max_depth), lo, hi, c))


def wls(dint, unit: float, weight_c: float = 4.0):
    """WLS GFD operator of one stencil from integer offsets (m x 3).

    Returns (P 9 x m, lap m, lapdiag, rmin/rmax) or None when rank deficient.
    """
    dint = np.ascontiguousarray(dint, dtype=np.int64)
    m = dint.shape[0]
    P = np.zeros((NCOL, m))
    lap = np.zeros(m)
    ld = C.c_double()
    rr = C.c_double()
    bad = _load().or_wls(m, _p(dint), unit, weight_c, _p(P), _p(lap), C.byref(ld), C.byref(rr))
    if bad:
        return None
    return P, lap, ld.value, rr.value


def select_neighbours(dint, idx, m_target: int):
    """Stencil of one node from its ring candidates (Section 3.1, two nearest per
    octant, then the nearest up to m_target, then the ties at the cut; at most
    MMAX): integer offsets dint (nc x 3) and node indices idx in, the chosen
    indices in rank order out."""
    dint = np.ascontiguousarray(dint, dtype=np.int64).reshape(-1, 3)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    sel = np.zeros(MMAX, dtype=np.int32)
    m = _load().or_select(len(idx), _p(dint), _p(idx), int(m_target), _p(sel))
    if m < 0:
        raise OracleError("or_select: out of memory")
    return sel[:m].copy()


def gmres(rowptr, col, val, b, x0=None, rtol=1e-10, max_iter=10000, restart=30):
    n = len(b)
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = _f64(val)
    b = _f64(b)
    x = np.zeros(n) if x0 is None else _f64(x0).copy()
    it = C.c_int()
    rr = C.c_double()
    s = _load().or_gmres(n, _p(rowptr), _p(col), _p(val), _p(b), _p(x), rtol, max_iter, restart,
                         C.byref(it), C.byref(rr))
    return x, it.value, rr.value, s


class Oracle:
    """One AP-Cloud problem on the CPU: tree, nodes, stencils, systems, fields."""

    def __init__(self, lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0), max_depth=6, c_refine=1.0,
                 m_target=20, ring_max=5, weight_c=4.0, poisson_c=1.0):
        lib = _load()
        self._lib = lib
        self.lo = np.array(lo, dtype=np.float64)
        self.hi = np.array(hi, dtype=np.float64)
        self.max_depth = max_depth
        self.m_target = m_target
        self.poisson_c = poisson_c
        self._ctx = lib.or_create(_p(self.lo), _p(self.hi), max_depth, c_refine, m_target, ring_max,
                                  weight_c, poisson_c)

    def __del__(self):
        if getattr(self, "_ctx", None):
            self._lib.or_destroy(self._ctx)
            self._ctx = None

    def _check(self, status):
        if status < 0:
            raise OracleError("oracle status %d: %s" % (status, self._lib.or_last_error(self._ctx).decode()))
        return status

    # -- Section 4: tree and nodes -------------------------------------------
    def build(self, x, y, z):
        self.x, self.y, self.z = _f64(x), _f64(y), _f64(z)
        self._check(self._lib.or_build(self._ctx, _p(self.x), _p(self.y), _p(self.z), len(self.x)))
        self.n_int = int(self._lib.or_n_interior(self._ctx))
        self.n_bnd = int(self._lib.or_n_boundary(self._ctx))
        return self.n_int, self.n_bnd

    @property
    def n_nodes(self):
        return self.n_int + self.n_bnd

    def nodes(self):
        nt = self.n_nodes
        ic = np.zeros((nt, 3), dtype=np.int32)
        lv = np.zeros(nt, dtype=np.int8)
        kd = np.zeros(nt, dtype=np.int8)
        xyz = np.zeros((nt, 3))
        self._lib.or_get_nodes(self._ctx, _p(ic), _p(lv), _p(kd), _p(xyz))
        return dict(icoord=ic, level=lv, kind=kd, xyz=xyz)

    def leaves(self):
        n = self.n_int
        key = np.zeros(n, dtype=np.uint64)
        first = np.zeros(n, dtype=np.int32)
        count = np.zeros(n, dtype=np.int32)
        self._lib.or_get_leaves(self._ctx, _p(key), _p(first), _p(count))
        return key, first, count

    def boundary(self):
        owner = np.zeros(self.n_bnd, dtype=np.int32)
        face = np.zeros(self.n_bnd, dtype=np.int8)
        self._lib.or_get_boundary(self._ctx, _p(owner), _p(face))
        return owner, face

    def order(self):
        o = np.zeros(len(self.x), dtype=np.int32)
        self._lib.or_get_order(self._ctx, _p(o))
        return o

    def cells(self):
        nc = int(self._lib.or_n_cells(self._ctx))
        key = np.zeros(nc, dtype=np.uint64)
        lv = np.zeros(nc, dtype=np.int8)
        op = np.zeros(nc, dtype=np.int8)
        cnt = np.zeros(nc, dtype=np.int32)
        self._lib.or_get_cells(self._ctx, _p(key), _p(lv), _p(op), _p(cnt))
        return key, lv, op, cnt

    def adjacency(self):
        na = int(self._lib.or_adjacency_size(self._ctx))
        off = np.zeros(self.n_nodes + 1, dtype=np.int32)
        adj = np.zeros(na, dtype=np.int32)
        self._lib.or_get_adjacency(self._ctx, _p(off), _p(adj))
        return off, adj

    # -- Section 3.1 / 4.3: stencils -----------------------------------------
    def stencils(self):
        self._check(self._lib.or_stencils(self._ctx))
        n, M = self.n_int, MMAX
        nbr = np.zeros((n, M), dtype=np.int32)
        msz = np.zeros(n, dtype=np.int32)
        ring = np.zeros(n, dtype=np.int32)
        lap = np.zeros((n, M))
        lapd = np.zeros(n)
        D = np.zeros((n, NCOL, M))
        self._lib.or_get_stencils(self._ctx, _p(nbr), _p(msz), _p(ring), _p(lap), _p(lapd), _p(D))
        self.st = dict(nbr=nbr, m=msz, ring=ring, lap=lap, lapd=lapd, D=D)
        return self.st

    def matrix(self, which: str):
        """CSR (rowptr, col, val) of 'B' (density) or 'A' (Poisson)."""
        nnz = int(self._lib.or_matrix_nnz(self._ctx))
        rp = np.zeros(self.n_nodes + 1, dtype=np.int64)
        col = np.zeros(nnz, dtype=np.int32)
        val = np.zeros(nnz)
        self._lib.or_matrix(self._ctx, 0 if which == "B" else 1, _p(rp), _p(col), _p(val))
        return rp, col, val

    # -- Section 3.2: the three steps ----------------------------------------
    def density_rhs(self, q=None, q_uniform=0.0):
        rhs = np.zeros(self.n_nodes)
        Qc = np.zeros(self.n_int)
        qa = None if q is None else _f64(q)
        total = self._lib.or_density_rhs(self._ctx, _p(qa), q_uniform, _p(rhs), _p(Qc))
        return rhs, Qc, total

    def solve_density(self, rhs, rtol=1e-12, max_iter=20000, restart=30, x0=None):
        rho = np.zeros(self.n_nodes) if x0 is None else _f64(x0).copy()
        it = C.c_int()
        rr = C.c_double()
        s = self._check(self._lib.or_solve_density(self._ctx, _p(_f64(rhs)), _p(rho), rtol, max_iter, restart,
                                                   C.byref(it), C.byref(rr)))
        return rho, it.value, rr.value, s

    def poisson_rhs(self, rho, g=None):
        rhs = np.zeros(self.n_nodes)
        ga = None if g is None else _f64(g)
        self._lib.or_poisson_rhs(self._ctx, _p(_f64(rho)), _p(ga), _p(rhs))
        return rhs

    def solve_poisson(self, rho, g=None, rtol=1e-12, max_iter=50000, restart=30, x0=None):
        phi = np.zeros(self.n_nodes) if x0 is None else _f64(x0).copy()
        ga = None if g is None else _f64(g)
        it = C.c_int()
        rr = C.c_double()
        s = self._check(self._lib.or_solve_poisson(self._ctx, _p(_f64(rho)), _p(ga), _p(phi), rtol, max_iter,
                                                   restart, C.byref(it), C.byref(rr)))
        return phi, it.value, rr.value, s

    def derivatives(self, phi):
        d = np.zeros((self.n_int, NCOL))
        self._lib.or_derivatives(self._ctx, _p(_f64(phi)), _p(d))
        return d

    def gather(self, phi, dphi=None):
        if dphi is None:
            dphi = self.derivatives(phi)
        N = len(self.x)
        out = [np.zeros(N) for _ in range(4)]
        self._lib.or_gather(self._ctx, _p(_f64(phi)), _p(_f64(dphi)), *[_p(o) for o in out])
        return tuple(out)

    def run(self, x, y, z, q=None, q_uniform=None, g=None, rtol=1e-12, restart=30, max_iter=50000):
        """Whole electrostatic solve: returns dict with phi at nodes and particles, E."""
        self.build(x, y, z)
        self.stencils()
        if q is None and q_uniform is None:
            q_uniform = 1.0 / max(1, len(self.x))
        rhs, Qc, total = self.density_rhs(q, 0.0 if q_uniform is None else q_uniform)
        rho, it_r, rr_r, _ = self.solve_density(rhs, rtol=rtol, restart=restart, max_iter=max_iter)
        phi, it_p, rr_p, _ = self.solve_poisson(rho, g, rtol=rtol, restart=restart, max_iter=max_iter)
        dphi = self.derivatives(phi)
        php, ex, ey, ez = self.gather(phi, dphi)
        return dict(rhoM=rhs, Q=Qc, total_charge=total, rho=rho, phi=phi, dphi=dphi, phi_p=php,
                    ex=ex, ey=ey, ez=ez, iters=(it_r, it_p), relres=(rr_r, rr_p))
