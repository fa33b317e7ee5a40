"""FP64 CPU oracle of the ALI hot path (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the bench's CPU-baseline and
reference legs may import this package. The CUDA library never calls it.
"""
from .oracle import (  # noqa: F401
    Oracle, healpix_dirs, antipodes, gauss_hermite, build_oracle, lib_path,
    CONST, planck, line_width_nu, first_order,
)
