"""FP64 CPU oracle for the real spherical harmonics (test infrastructure only).

This package is the independent checker of the CUDA path. It is NOT part of the
product: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` may import it. It shares no code, tables or
constants with ``paper_2302_08381_gb300`` and never imports it.

Parity status of each oracle function is stated in ``sph_oracle``'s header.
"""

from .sph_oracle import (  # noqa: F401
    prefactor,
    prefactor_table,
    legendre_table,
    legendre_derivative_table,
    spherical_harmonics,
    spherical_harmonics_grad,
    spherical_harmonics_hessian,
    spherical_harmonics_hessian_fd,
    backward,
    double_backward,
    column,
    expansion,
)
