"""GB300-native AP-Cloud electrostatic solve (arXiv 1603.04039).

The computation lives in libapcloud.so (hand-written CUDA for sm_103a behind
the C ABI of include/apcloud.h).  ``APCloud`` is the thin ctypes binding;
``inputs`` holds the seeded synthetic particle laws.  Importing the package
does not load the library; creating an ``APCloud`` does, and fails loudly if
it has not been built.
"""
from . import inputs  # noqa: F401


def __getattr__(name):
    if name in ("APCloud", "APCloudError", "MPNN", "kernel_names", "load", "ilu0_factor_host"):
        from . import _binding
        return getattr(_binding, name)
    if name == "VlasovPoisson":
        from .vlasov import VlasovPoisson
        return VlasovPoisson
    raise AttributeError(name)
