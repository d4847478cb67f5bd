"""GB300 (sm_103a) spherical harmonics after arXiv 2302.08381 (sphericart).

The compute path is the CUDA library ``libsphericart_gb300.so`` behind the
C-ABI declared in ``include/sphericart_gb300.h``; this package marshals
arguments to it (``_capi``: ctypes, same names as the C-ABI; ``api``: torch
tensors) and wraps it for autograd (``autograd``). Importing the package does
not load the library; the first call does, and fails loudly if it is missing.
"""

__version__ = "1.0.0"


def __getattr__(name):
    if name in ("spherical_harmonics", "backward", "double_backward", "materialized_backward", "device_status"):
        from . import api

        return getattr(api, name)
    if name in ("SphericalHarmonicsFn", "spherical_harmonics_autograd"):
        from . import autograd

        return getattr(autograd, name)
    raise AttributeError(name)
