"""GB300 (sm_103a) spherical harmonics after arXiv 2302.08381 (sphericart).

The compute path is the CUDA library ``libsphericart_gb300.so`` behind the
C-ABI declared in ``include/sphericart_gb300.h``; this package only marshals
arguments to it (``_capi``) and wraps it for torch autograd.
"""
