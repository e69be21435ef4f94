"""CPU oracle for the 3D C2C DFT and the PME reciprocal-space convolution (test
infrastructure; see ``oracle.direct_dft`` and ``oracle.convolution``).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference legs may import this package.  The CUDA library never does.
"""

from .direct_dft import (  # noqa: F401
    BACKWARD,
    FORWARD,
    backward,
    dft3,
    dft3_at,
    dft3_bruteforce,
    dft_along_axis,
    dft_matrix,
    forward,
    rel_l2,
)
from .convolution import convolve  # noqa: F401,E402
