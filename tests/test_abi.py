"""The C-ABI library builds, loads without a GPU and exports every symbol the
public header declares; host-side validation needs no device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(apcloud_[a-z_]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1603_04039_gb300 import build
    path = build.build()
    return C.CDLL(path)


def test_header_declares_the_five_steps():
    names = _declared()
    for n in ("apcloud_build_octree", "apcloud_stencils", "apcloud_deposit", "apcloud_solve",
              "apcloud_gather_field"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in sorted(_declared()):
        assert hasattr(lib, name), name


def test_param_validation_without_gpu(lib):
    from paper_1603_04039_gb300 import _binding as B
    l = B.load()
    p = B.Params()
    l.apcloud_default_params(C.byref(p))
    assert (p.max_depth, p.m_target, p.ring_max, p.restart) == (6, 20, 5, 30)
    assert p.weight_c == 4.0 and p.poisson_c == 1.0 and p.c_refine == 1.0
    ctx = C.c_void_p()
    for field, bad in (("max_depth", 22), ("m_target", 8), ("m_target", 33), ("ring_max", 1), ("restart", 0),
                       ("precision", 2), ("stencil_slots", 15), ("stencil_slots", 129)):
        q = B.Params()
        l.apcloud_default_params(C.byref(q))
        setattr(q, field, bad)
        assert l.apcloud_create(C.byref(q), None, None, C.byref(ctx)) == -1, field
    q = B.Params()
    l.apcloud_default_params(C.byref(q))
    q.hi[2] = 2.0                        # not a cube
    assert l.apcloud_create(C.byref(q), None, None, C.byref(ctx)) == -1
    keep = C.c_int64()
    assert l.apcloud_set_sweep_l2_keep(None, 0) == -1          # no context
    assert l.apcloud_get_sweep_l2_keep(None, C.byref(keep)) == -1
    assert l.apcloud_kernel_name(7) == b"spmv"
    assert l.apcloud_kernel_name(99) == b"unknown"
