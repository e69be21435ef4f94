"""FP64 CPU oracle for the reciprocal-space convolution of the PME method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code, tables or constants with the CUDA library.

What it computes.  The paper's motivating application (Sec. 1) is the
particle-mesh Ewald (PME) method, where the charge grid goes through a forward
3D FFT, is multiplied point by point by a real influence function G(k), and
comes back through a backward 3D FFT.  With F the forward transform of Eq. (1)
and B the backward transform of Eq. (2) read unnormalised (see
``oracle.direct_dft``):

    convolve(X, G) = B(G * F(X)).

By the convolution theorem this equals the circular convolution of X with
h = B(G) (no 1/N factor anywhere):  out(j) = sum_m X(m) h((j - m) mod n).

How: the definition as written - the oracle's own forward transform, an
elementwise product with G upcast exactly to float64, the oracle's backward
transform.  No fusion, no reordering.
"""

from __future__ import annotations

import numpy as np

from .direct_dft import backward, forward

__all__ = ["convolve"]


def convolve(x: np.ndarray, g: np.ndarray) -> np.ndarray:
    """B(G * F(x)) for a (nx, ny, nz) grid x and a real (nx, ny, nz) influence function g."""
    x = np.asarray(x)
    g = np.asarray(g)
    if g.shape != x.shape:
        raise ValueError(f"influence function shape {g.shape} != grid shape {x.shape}")
    if np.iscomplexobj(g):
        raise ValueError("the influence function is real")
    y = forward(x)
    y = y * g.astype(np.float64)
    return backward(y)
