"""ctypes binding of libapcloud.so: argument marshalling only.

Every function here forwards to the C ABI of include/apcloud.h with the same
name; device arrays are CUDA tensors (float64 unless stated), the stream is
the current torch stream of the tensor's device.  All computation happens in
the library's CUDA kernels.  A missing library raises immediately: there is
no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
import sys
import threading

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libapcloud.so")

NUM_KINDS = 19
MMAX = 32
NCOL = 9

STATUS = {0: "OK", 1: "W_NOT_CONVERGED", -1: "E_INVALID", -2: "E_DOMAIN", -3: "E_STENCIL", -4: "E_CUDA",
          -5: "E_NOMEM", -6: "E_TIMEOUT", -7: "E_STATE", -8: "E_NUMERIC"}

_lock = threading.Lock()
_lib = None


class APCloudError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s (%d): %s" % (STATUS.get(status, "?"), status, message))
        self.status = status


class Params(C.Structure):
    _fields_ = [("lo", C.c_double * 3), ("hi", C.c_double * 3), ("max_depth", C.c_int), ("c_refine", C.c_double),
                ("m_target", C.c_int), ("ring_max", C.c_int), ("weight_c", C.c_double),
                ("poisson_c", C.c_double), ("restart", C.c_int), ("precision", C.c_int),
                ("poly_degree", C.c_int), ("poly_omega", C.c_double), ("fp32_rcond_min", C.c_double),
                ("stencil_slots", C.c_int)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int), ("restarts", C.c_int), ("relres", C.c_double)]

    def as_dict(self):
        return {"iters": self.iters, "restarts": self.restarts, "relres": self.relres}


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    """apcloud_allocator: alloc(bytes, stream, user) / free(ptr, stream, user)."""
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("user", C.c_void_p)]


class TorchAllocator:
    """The context's device allocator backed by PyTorch's caching allocator, so
    the library's buffers come from (and return to) the same pool as the
    caller's tensors, on the context's stream.  Counts its calls; `fail_at`
    (1-based) makes that allocation call report failure instead (tests of the
    out-of-memory path)."""

    def __init__(self, device, fail_at=None):
        self.device = torch.device(device).index or 0
        self.fail_at = fail_at
        self.allocs = 0
        self.frees = 0
        self.live = {}
        self._cb_alloc = _ALLOC_FN(self._alloc)
        self._cb_free = _FREE_FN(self._free)
        self.struct = Allocator(self._cb_alloc, self._cb_free, None)

    @property
    def live_bytes(self):
        return sum(self.live.values())

    def _alloc(self, nbytes, stream, user):
        self.allocs += 1
        if self.fail_at is not None and self.allocs == self.fail_at:
            return None
        try:
            p = torch.cuda.caching_allocator_alloc(int(nbytes), device=self.device, stream=int(stream or 0))
        except Exception:   # out of memory: the library reports APCLOUD_E_NOMEM
            return None
        self.live[p] = int(nbytes)
        return p

    def _free(self, ptr, stream, user):
        if not ptr:
            return
        self.frees += 1
        self.live.pop(ptr, None)
        try:
            torch.cuda.caching_allocator_delete(ptr)
        except Exception:
            pass


def load():
    """Load libapcloud.so (built by paper_1603_04039_gb300.build)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libapcloud.so is not built: run `python -c \"import __graft_entry__ as g; "
                               "g.build()\"` (or paper_1603_04039_gb300.build.build())")
        lib = C.CDLL(LIB_PATH)
        P, I, D, L = C.c_void_p, C.c_int, C.c_double, C.c_int64
        sig = {
            "apcloud_default_params": (None, [C.POINTER(Params)]),
            "apcloud_create": (I, [C.POINTER(Params), P, P, C.POINTER(P)]),
            "apcloud_destroy": (None, [P]),
            "apcloud_last_error": (C.c_char_p, [P]),
            "apcloud_build_octree": (I, [P, P, P, P, L, C.POINTER(L), C.POINTER(L)]),
            "apcloud_build_octree_batched": (I, [P, P, P, P, C.POINTER(L), I, C.POINTER(L), C.POINTER(L)]),
            "apcloud_get_node_beams": (I, [P, P]),
            "apcloud_get_nodes": (I, [P, P, P, P]),
            "apcloud_get_leaves": (I, [P, P, P, P]),
            "apcloud_stencils": (I, [P]),
            "apcloud_get_stencils": (I, [P, P, P, P, P, P]),
            "apcloud_deposit": (I, [P, P, D, D, I, P, C.POINTER(SolveInfo)]),
            "apcloud_get_rho_m": (I, [P, P]),
            "apcloud_solve": (I, [P, P, P, D, I, P, C.POINTER(SolveInfo)]),
            "apcloud_gather_field": (I, [P, P, P, P, P]),
            "apcloud_get_derivatives": (I, [P, P]),
            "apcloud_matvec": (I, [P, I, P, P]),
            "apcloud_solve_system": (I, [P, I, P, P, D, I, C.POINTER(SolveInfo)]),
            "apcloud_solve_system_noalloc": (I, [P, I, P, P, D, I, C.POINTER(SolveInfo)]),
            "apcloud_solve_system_ilu0": (I, [P, I, P, P, D, I, C.POINTER(SolveInfo), P]),
            "apcloud_ilu0_factor_host": (I, [L, P, P, P]),
            "apcloud_field_host": (I, [P, P, P, P, P, D, L, D, I, P, P, P, P, C.POINTER(SolveInfo),
                                       C.POINTER(SolveInfo)]),
            "apcloud_field_host_batched": (I, [P, P, P, P, P, D, C.POINTER(L), I, D, I, P, P, P, P,
                                               C.POINTER(SolveInfo), C.POINTER(SolveInfo)]),
            "apcloud_set_timing": (I, [P, C.c_uint]),
            "apcloud_set_graphs": (I, [P, I]),
            "apcloud_autotune": (I, [P, C.c_uint, C.POINTER(I), C.POINTER(I), C.POINTER(I), C.POINTER(I), P]),
            "apcloud_set_launch_shape": (I, [P, I, I, I, I]),
            "apcloud_set_sweep_l2_keep": (I, [P, L]),
            "apcloud_set_dependent_launch": (I, [P, I]),
            "apcloud_get_sweep_l2_keep": (I, [P, C.POINTER(L)]),
            "apcloud_graph_stats": (I, [P, C.POINTER(L), C.POINTER(L)]),
            "apcloud_get_timing": (I, [P, P, P, P, P, I]),
            "apcloud_kernel_name": (C.c_char_p, [I]),
            "apcloud_launch_count": (L, [P]),
            "apcloud_host_sync_count": (L, [P]),
            "apcloud_get_sizes": (I, [P, P]),
            "apcloud_interpolate_potential": (I, [P, P, P, P, L, P]),
            "apcloud_push_particles": (I, [P, P, P, P, P, P, P, L, P, P, P, D, D]),
            "apcloud_field_energy": (I, [P, C.POINTER(D)]),
            "apcloud_measure_fma_peak": (I, [C.POINTER(D), C.POINTER(D)]),
            "apcloud_mpnn_num_params": (I, []),
            "apcloud_mpnn_create": (I, [P, C.c_uint64, C.POINTER(P)]),
            "apcloud_mpnn_destroy": (None, [P]),
            "apcloud_mpnn_get_params": (I, [P, P, P]),
            "apcloud_mpnn_set_params": (I, [P, P]),
            "apcloud_mpnn_loss": (I, [P, P, I, P]),
            "apcloud_mpnn_adam": (I, [P, P, C.c_float]),
            "apcloud_mpnn_outputs": (I, [P, P, P, P, P]),
            "apcloud_solve_learned": (I, [P, P, C.c_uint, P, D, I, P, C.POINTER(SolveInfo)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _dptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _f64(t, n=None):
    if t is None:
        return None
    if t.dtype != torch.float64:
        raise TypeError("expected float64, got %s" % t.dtype)
    if n is not None and t.numel() != n:
        raise ValueError("expected %d entries, got %d" % (n, t.numel()))
    return t


def ilu0_factor_host(rowptr, col, val):
    """ILU(0) of a host CSR matrix (columns sorted, diagonal present) through the
    library's host routine; returns the factored values (L strictly below the
    diagonal with a unit diagonal implied, U on and above it)."""
    lib = load()
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    cj = np.ascontiguousarray(col, dtype=np.int32)
    a = np.array(val, dtype=np.float64, copy=True)
    st = lib.apcloud_ilu0_factor_host(len(rp) - 1, rp.ctypes.data_as(C.c_void_p), cj.ctypes.data_as(C.c_void_p),
                                      a.ctypes.data_as(C.c_void_p))
    if st < 0:
        raise APCloudError(st, "ILU(0) factorisation")
    return a


def measure_fma_peak():
    """(FP64, FP32) FMA throughput of the current CUDA device in TFLOP/s."""
    lib = load()
    d, f = C.c_double(), C.c_double()
    st = lib.apcloud_measure_fma_peak(C.byref(d), C.byref(f))
    if st != 0:
        raise APCloudError(st, "apcloud_measure_fma_peak failed")
    return d.value, f.value


def kernel_names():
    lib = load()
    return [lib.apcloud_kernel_name(k).decode() for k in range(NUM_KINDS)]


class APCloud:
    """One AP-Cloud problem on one GPU (see include/apcloud.h for each call)."""

    def __init__(self, lo=-1.0, hi=1.0, max_depth=6, c_refine=1.0, m_target=20, ring_max=5, weight_c=4.0,
                 poisson_c=1.0, restart=30, precision="fp64", poly_degree=1, poly_omega=0.7, device="cuda:0",
                 stream=None, allocator="torch", fp32_rcond_min=1e-3, stencil_slots=128):
        """allocator: "torch" (default) gives the context PyTorch's caching
        allocator; None selects the library's own cudaMallocAsync pool; a
        TorchAllocator instance is used as given."""
        lib = load()
        self._lib = lib
        self.device = torch.device(device)
        p = Params()
        lib.apcloud_default_params(C.byref(p))
        for d in range(3):
            p.lo[d] = float(lo)
            p.hi[d] = float(hi)
        p.max_depth, p.c_refine, p.m_target, p.ring_max = int(max_depth), float(c_refine), int(m_target), int(ring_max)
        p.weight_c, p.poisson_c, p.restart = float(weight_c), float(poisson_c), int(restart)
        p.precision = {"fp64": 0, "mixed": 1}[precision]
        p.poly_degree, p.poly_omega = int(poly_degree), float(poly_omega)
        p.fp32_rcond_min = float(fp32_rcond_min)
        p.stencil_slots = int(stencil_slots)
        self.params = p
        with torch.cuda.device(self.device):
            s = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.stream = s
            ctx = C.c_void_p()
            if allocator == "torch":
                allocator = TorchAllocator(self.device)
            self.allocator = allocator   # keeps the callbacks alive as long as the context
            a = C.byref(allocator.struct) if allocator is not None else None
            st = lib.apcloud_create(C.byref(p), a, C.c_void_p(s.cuda_stream), C.byref(ctx))
        if st != 0:
            raise APCloudError(st, "apcloud_create failed")
        self._ctx = ctx
        self.n_int = self.n_bnd = 0
        self.n = 0

    def close(self):
        if getattr(self, "_ctx", None):
            with torch.cuda.device(self.device):
                self._lib.apcloud_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        # at interpreter exit the allocator's Python callbacks may be gone: leave
        # the buffers to the process teardown
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st < 0:
            raise APCloudError(st, self._lib.apcloud_last_error(self._ctx).decode())
        return st

    def _empty(self, *shape, dtype=torch.float64):
        return torch.empty(*shape, dtype=dtype, device=self.device)

    @property
    def n_nodes(self):
        return self.n_int + self.n_bnd

    # -- entry points ---------------------------------------------------------
    def build_octree(self, x, y, z):
        n = x.numel()
        for t in (x, y, z):
            _f64(t, n)
        self._pos = (x, y, z)   # the library keeps these pointers until the next build
        ni, nb = C.c_int64(), C.c_int64()
        with torch.cuda.device(self.device):
            self._check(self._lib.apcloud_build_octree(self._ctx, _dptr(x), _dptr(y), _dptr(z), n, C.byref(ni),
                                                       C.byref(nb)))
        self.n, self.n_int, self.n_bnd = n, ni.value, nb.value
        return self.n_int, self.n_bnd

    def build_octree_batched(self, x, y, z, offsets):
        """Independent beams: beam b holds particles offsets[b]:offsets[b+1]."""
        n = x.numel()
        for t in (x, y, z):
            _f64(t, n)
        offs = [int(o) for o in offsets]
        if len(offs) < 2 or offs[-1] != n:
            raise ValueError("offsets must have n_beams + 1 entries ending at the particle count")
        arr = (C.c_int64 * len(offs))(*offs)
        self._pos = (x, y, z)
        ni, nb = C.c_int64(), C.c_int64()
        with torch.cuda.device(self.device):
            self._check(self._lib.apcloud_build_octree_batched(self._ctx, _dptr(x), _dptr(y), _dptr(z), arr,
                                                               len(offs) - 1, C.byref(ni), C.byref(nb)))
        self.n, self.n_int, self.n_bnd = n, ni.value, nb.value
        return self.n_int, self.n_bnd

    def get_node_beams(self):
        out = self._empty(self.n_nodes, dtype=torch.int32)
        with torch.cuda.device(self.device):
            self._check(self._lib.apcloud_get_node_beams(self._ctx, _dptr(out)))
        return out

    def get_nodes(self):
        xyz = self._empty(self.n_nodes, 3)
        lv = self._empty(self.n_nodes, dtype=torch.int8)
        kd = self._empty(self.n_nodes, dtype=torch.int8)
        with torch.cuda.device(self.device):
            self._check(self._lib.apcloud_get_nodes(self._ctx, _dptr(xyz), _dptr(lv), _dptr(kd)))
        return {"xyz": xyz, "level": lv, "kind": kd}

    def get_leaves(self):
        key = self._empty(self.n_int, dtype=torch.int64)
        first = self._empty(self.n_int, dtype=torch.int32)
        count = self._empty(self.n_int, dtype=torch.int32)
        with torch.cuda.device(self.device):
            self._check(self._lib.apcloud_get_leaves(self._ctx, _dptr(key), _dptr(first), _dptr(count)))
        return {"key": key, "first": first, "count": count}

    def stencils(self):
        with torch.cuda.device(self.device):
            self._check(self._lib.apcloud_stencils(self._ctx))

    def get_stencils(self):
        n = self.n_int
        out = {"nbr": self._empty(n, MMAX, dtype=torch.int32), "m": self._empty(n, dtype=torch.int32),
               "lap": self._empty(n, MMAX), "lapd": self._empty(n), "D": self._empty(n, NCOL, MMAX)}
        with torch.cuda.device(self.device):
            self._check(self._lib.apcloud_get_stencils(self._ctx, _dptr(out["nbr"]), _dptr(out["m"]),
                                                       _dptr(out["lap"]), _dptr(out["lapd"]), _dptr(out["D"])))
        return out

    def deposit(self, q=None, q_uniform=None, rtol=1e-10, max_iter=100000):
        if q is not None:
            _f64(q, self.n)
        if q is None and q_uniform is None:
            q_uniform = 1.0 / max(1, self.n)
        rho = self._empty(self.n_nodes)
        info = SolveInfo()
        with torch.cuda.device(self.device):
            st = self._check(self._lib.apcloud_deposit(self._ctx, _dptr(q), float(q_uniform or 0.0), rtol,
                                                       int(max_iter), _dptr(rho), C.byref(info)))
        return rho, dict(info.as_dict(), status=st)

    def get_rho_m(self):
        out = self._empty(self.n_nodes)
        with torch.cuda.device(self.device):
            self._check(self._lib.apcloud_get_rho_m(self._ctx, _dptr(out)))
        return out

    def solve(self, g=None, phi0=None, rtol=1e-10, max_iter=100000):
        if g is not None:
            _f64(g, self.n_bnd)
        if phi0 is not None:
            _f64(phi0, self.n_nodes)
        phi = self._empty(self.n_nodes)
        info = SolveInfo()
        with torch.cuda.device(self.device):
            st = self._check(self._lib.apcloud_solve(self._ctx, _dptr(g), _dptr(phi0), rtol, int(max_iter),
                                                     _dptr(phi), C.byref(info)))
        return phi, dict(info.as_dict(), status=st)

    def gather_field(self, out=None):
        if out is None:
            out = tuple(self._empty(self.n) for _ in range(4))
        with torch.cuda.device(self.device):
            self._check(self._lib.apcloud_gather_field(self._ctx, *[_dptr(t) for t in out]))
        return out

    def get_derivatives(self):
        out = self._empty(self.n_int, NCOL)
        with torch.cuda.device(self.device):
            self._check(self._lib.apcloud_get_derivatives(self._ctx, _dptr(out)))
        return out

    def matvec(self, which, x):
        _f64(x, self.n_nodes)
        y = self._empty(self.n_nodes)
        with torch.cuda.device(self.device):
            self._check(self._lib.apcloud_matvec(self._ctx, 1 if which == "A" else 0, _dptr(x), _dptr(y)))
        return y

    def solve_system(self, which, b, x0=None, rtol=1e-10, max_iter=100000):
        _f64(b, self.n_nodes)
        x = torch.zeros(self.n_nodes, dtype=torch.float64, device=self.device) if x0 is None else x0.clone()
        info = SolveInfo()
        with torch.cuda.device(self.device):
            st = self._check(self._lib.apcloud_solve_system(self._ctx, 1 if which == "A" else 0, _dptr(b), _dptr(x),
                                                            rtol, int(max_iter), C.byref(info)))
        return x, dict(info.as_dict(), status=st)

    def solve_system_ilu0(self, which, b, x0=None, rtol=1e-10, max_iter=100000):
        """GMRES with the ILU(0) right preconditioner (FP64 form, single beam): the
        comparison baseline of the learned preconditioner."""
        _f64(b, self.n_nodes)
        x = torch.zeros(self.n_nodes, dtype=torch.float64, device=self.device) if x0 is None else x0.clone()
        info = SolveInfo()
        stats = np.zeros(4)
        with torch.cuda.device(self.device):
            st = self._check(self._lib.apcloud_solve_system_ilu0(self._ctx, 1 if which == "A" else 0, _dptr(b),
                                                                 _dptr(x), rtol, int(max_iter), C.byref(info),
                                                                 stats.ctypes.data_as(C.c_void_p)))
        return x, dict(info.as_dict(), status=st, setup_ms=float(stats[0]), levels_lower=int(stats[1]),
                       levels_upper=int(stats[2]), nnz=int(stats[3]))

    def solve_system_noalloc(self, which, b, x, rtol=1e-10, max_iter=100000):
        """apcloud_solve_system_noalloc on caller-owned tensors: x holds the
        initial guess and receives the solution; the library allocates nothing."""
        _f64(b, self.n_nodes)
        _f64(x, self.n_nodes)
        info = SolveInfo()
        with torch.cuda.device(self.device):
            st = self._check(self._lib.apcloud_solve_system_noalloc(self._ctx, 1 if which == "A" else 0, _dptr(b),
                                                                    _dptr(x), rtol, int(max_iter), C.byref(info)))
        return dict(info.as_dict(), status=st)

    def field_host(self, x, y, z, q=None, q_uniform=None, rtol=1e-10, max_iter=100000, out=None, offsets=None):
        """Whole solve on host numpy arrays (pinned tensors are also accepted);
        ``offsets`` (n_beams + 1 entries) makes it a batch of beams."""
        def hp(a):
            if a is None:
                return None
            if isinstance(a, torch.Tensor):
                assert not a.is_cuda and a.dtype == torch.float64 and a.is_contiguous()
                return C.c_void_p(a.data_ptr())
            a = np.ascontiguousarray(a, dtype=np.float64)
            return a.ctypes.data_as(C.c_void_p)
        n = len(x)
        if out is None:
            out = tuple(np.empty(n) for _ in range(4))
        if q is None and q_uniform is None:
            q_uniform = 1.0 / max(1, n)
        keep = [np.ascontiguousarray(a, dtype=np.float64) if isinstance(a, np.ndarray) else a for a in (x, y, z, q)]
        ir, ip = SolveInfo(), SolveInfo()
        with torch.cuda.device(self.device):
            if offsets is None:
                st = self._check(self._lib.apcloud_field_host(self._ctx, hp(keep[0]), hp(keep[1]), hp(keep[2]),
                                                              hp(keep[3]), float(q_uniform or 0.0), n, rtol,
                                                              int(max_iter), *[hp(o) for o in out], C.byref(ir),
                                                              C.byref(ip)))
            else:
                offs = [int(o) for o in offsets]
                if len(offs) < 2 or offs[0] != 0 or offs[-1] != n:
                    raise ValueError("offsets must run from 0 to the particle count")
                arr = (C.c_int64 * len(offs))(*offs)
                st = self._check(self._lib.apcloud_field_host_batched(
                    self._ctx, hp(keep[0]), hp(keep[1]), hp(keep[2]), hp(keep[3]), float(q_uniform or 0.0), arr,
                    len(offs) - 1, rtol, int(max_iter), *[hp(o) for o in out], C.byref(ir), C.byref(ip)))
        self.n = n
        return out, {"rho": ir.as_dict(), "phi": ip.as_dict(), "status": st}

    def interpolate_potential(self, x, y, z, out=None):
        n = x.numel()
        out = self._empty(n) if out is None else out
        with torch.cuda.device(self.device):
            self._check(self._lib.apcloud_interpolate_potential(self._ctx, _dptr(x), _dptr(y), _dptr(z), n,
                                                                _dptr(out)))
        return out

    def push_particles(self, x, y, z, vx, vy, vz, field=None, qm_dt=0.0, dt=0.0):
        n = x.numel()
        ex, ey, ez = field if field is not None else (None, None, None)
        with torch.cuda.device(self.device):
            self._check(self._lib.apcloud_push_particles(self._ctx, _dptr(x), _dptr(y), _dptr(z), _dptr(vx),
                                                         _dptr(vy), _dptr(vz), n, _dptr(ex), _dptr(ey), _dptr(ez),
                                                         float(qm_dt), float(dt)))

    def field_energy(self):
        e = C.c_double()
        with torch.cuda.device(self.device):
            self._check(self._lib.apcloud_field_energy(self._ctx, C.byref(e)))
        return e.value

    def autotune(self, spmv=True, stencils=True):
        """Times the launch shapes and keeps the fastest; returns the choice and timings:
        spmv_ms = ms of one Poisson solve (synthetic right-hand side) per product shape,
        wls_ms = ms of one stencil build per nodes-per-block."""
        bs, un, so, ww = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        ms = np.zeros(19)
        what = (1 if spmv else 0) | (2 if stencils else 0)
        with torch.cuda.device(self.device):
            self._check(self._lib.apcloud_autotune(self._ctx, what, C.byref(bs), C.byref(un), C.byref(so),
                                                   C.byref(ww), ms.ctypes.data_as(C.c_void_p)))
        keys = ["%s%d/u%d" % (lay, b, u) for lay in ("ell", "sorted") for u in (1, 4) for b in (64, 128, 256, 512)]
        sp = {k: v for k, v in zip(keys, ms[:16].round(4).tolist()) if v > 0}
        return {"spmv_block": bs.value, "spmv_unroll": un.value, "sweep_sorted": so.value, "wls_warps": ww.value,
                "spmv_ms": sp if spmv else None,
                "wls_ms": dict(zip((2, 4, 8), ms[16:].round(3).tolist())) if stencils else None}

    def set_launch_shape(self, spmv_block=256, wls_warps=4, spmv_unroll=1, sweep_sorted=0):
        self._check(self._lib.apcloud_set_launch_shape(self._ctx, int(spmv_block), int(spmv_unroll),
                                                       int(sweep_sorted), int(wls_warps)))

    def set_dependent_launch(self, enable):
        self._check(self._lib.apcloud_set_dependent_launch(self._ctx, 1 if enable else 0))

    def set_sweep_l2_keep(self, keep_bytes=-1):
        self._check(self._lib.apcloud_set_sweep_l2_keep(self._ctx, int(keep_bytes)))

    def sweep_l2_keep(self):
        v = C.c_int64()
        self._check(self._lib.apcloud_get_sweep_l2_keep(self._ctx, C.byref(v)))
        return v.value

    def solve_learned(self, net, use=3, rtol=1e-10, max_iter=100000, phi0=None):
        """Poisson solve with the network's column scaling (use bit 0), guess (bit 1)
        or the closed-form diagonal (bit 2); without bit 1 it starts from phi0 (or 0)."""
        phi = self._empty(self.n_nodes)
        info = SolveInfo()
        if phi0 is not None:
            _f64(phi0, self.n_nodes)
        with torch.cuda.device(self.device):
            st = self._check(self._lib.apcloud_solve_learned(self._ctx, net._net, int(use), _dptr(phi0), rtol,
                                                             int(max_iter), _dptr(phi), C.byref(info)))
        return phi, dict(info.as_dict(), status=st)

    def set_graphs(self, enable):
        with torch.cuda.device(self.device):
            self._check(self._lib.apcloud_set_graphs(self._ctx, 1 if enable else 0))

    def graph_stats(self):
        r, g = C.c_int64(), C.c_int64()
        self._check(self._lib.apcloud_graph_stats(self._ctx, C.byref(r), C.byref(g)))
        return {"replays": r.value, "cached": g.value}

    def set_timing(self, mask):
        self._check(self._lib.apcloud_set_timing(self._ctx, int(mask)))

    def get_timing(self, reset=True):
        """{kernel: (ms, launches, algorithmic bytes, algorithmic flops)} since the last reset."""
        ms = np.zeros(NUM_KINDS)
        cnt = np.zeros(NUM_KINDS, dtype=np.int64)
        by = np.zeros(NUM_KINDS)
        fl = np.zeros(NUM_KINDS)
        self._check(self._lib.apcloud_get_timing(self._ctx, ms.ctypes.data_as(C.c_void_p),
                                                 cnt.ctypes.data_as(C.c_void_p), by.ctypes.data_as(C.c_void_p),
                                                 fl.ctypes.data_as(C.c_void_p), 1 if reset else 0))
        return {name: (float(ms[k]), int(cnt[k]), float(by[k]), float(fl[k]))
                for k, name in enumerate(kernel_names())}

    def sizes(self):
        h = np.zeros(9, dtype=np.int64)
        self._check(self._lib.apcloud_get_sizes(self._ctx, h.ctypes.data_as(C.c_void_p)))
        keys = ("particles", "n_interior", "n_boundary", "nnz", "ell_entries", "sum_m", "slices", "depth",
                "fp64_stencils")
        return dict(zip(keys, (int(v) for v in h)))

    def launch_count(self):
        return int(self._lib.apcloud_launch_count(self._ctx))

    def host_sync_count(self):
        return int(self._lib.apcloud_host_sync_count(self._ctx))


class MPNN:
    """The learned preconditioner network (see include/apcloud.h)."""

    def __init__(self, theta=None, seed=0, device="cuda:0"):
        lib = load()
        self._lib = lib
        self.device = torch.device(device)
        self.n_params = lib.apcloud_mpnn_num_params()
        net = C.c_void_p()
        arr = None
        if theta is not None:
            arr = np.ascontiguousarray(theta, dtype=np.float32)
            assert arr.size == self.n_params
        with torch.cuda.device(self.device):
            st = lib.apcloud_mpnn_create(arr.ctypes.data_as(C.c_void_p) if arr is not None else None, int(seed),
                                         C.byref(net))
        if st != 0:
            raise APCloudError(st, "apcloud_mpnn_create failed")
        self._net = net

    def close(self):
        if getattr(self, "_net", None):
            with torch.cuda.device(self.device):
                self._lib.apcloud_mpnn_destroy(self._net)
            self._net = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        th = np.zeros(self.n_params, dtype=np.float32)
        g = np.zeros(self.n_params, dtype=np.float32)
        with torch.cuda.device(self.device):
            st = self._lib.apcloud_mpnn_get_params(self._net, th.ctypes.data_as(C.c_void_p), g.ctypes.data_as(C.c_void_p))
        if st != 0:
            raise APCloudError(st, "apcloud_mpnn_get_params failed")
        return th, g

    def set_params(self, theta):
        arr = np.ascontiguousarray(theta, dtype=np.float32)
        with torch.cuda.device(self.device):
            st = self._lib.apcloud_mpnn_set_params(self._net, arr.ctypes.data_as(C.c_void_p))
        if st != 0:
            raise APCloudError(st, "apcloud_mpnn_set_params failed")

    def loss(self, ap, backward=False):
        out = np.zeros(3)
        with torch.cuda.device(self.device):
            ap._check(self._lib.apcloud_mpnn_loss(ap._ctx, self._net, 1 if backward else 0,
                                                  out.ctypes.data_as(C.c_void_p)))
        return {"L": out[0], "Lp": out[1], "Lg": out[2]}

    def adam(self, ap, lr=1e-3):
        with torch.cuda.device(self.device):
            ap._check(self._lib.apcloud_mpnn_adam(ap._ctx, self._net, C.c_float(lr)))

    def outputs(self, ap):
        n = ap.n_nodes
        s = torch.empty(n, dtype=torch.float32, device=ap.device)
        g = torch.empty(n, dtype=torch.float32, device=ap.device)
        f = torch.empty(n, 16, dtype=torch.float32, device=ap.device)
        with torch.cuda.device(self.device):
            ap._check(self._lib.apcloud_mpnn_outputs(ap._ctx, self._net, _dptr(s), _dptr(g), _dptr(f)))
        return {"s": s, "gamma": g, "features": f}

