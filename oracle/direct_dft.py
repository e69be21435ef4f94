"""FP64 CPU oracle for the unnormalised 3D complex-to-complex DFT.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code, tables or constants with the CUDA library.

What it computes (paper Sec. 2.1):

* Forward, Eq. (1):
  ``Y(kx,ky,kz) = sum_j X(jx,jy,jz) exp(-2 pi i (kx jx/Nx + ky jy/Ny + kz jz/Nz))``.
* Backward, Eq. (2) with the sign ``+``.  Eq. (2) prints a ``1/(Nx Ny Nz)``
  factor, while Sec. 5.3 describes a backward pass used without any
  normalisation; this library's reading is *unnormalised in both directions*,
  so ``backward(forward(X)) = Nx Ny Nz * X``.  A caller who wants Eq. (2)
  literally divides by ``Nx Ny Nz``.

How (the plain definition, no fast algorithm):

* The exponent of Eq. (1) is a sum over the three axes, so the triple sum
  factors into three one-axis DFTs (the separability the paper builds on,
  Sec. 2.1 last paragraph and Sec. 4).  ``dft3`` applies the dense
  ``n x n`` DFT matrix along z, then y, then x (the same axis order as the
  GPU passes; the exact result does not depend on the order).
* DFT matrix entries ``W[k, j] = exp(s 2 pi i r / n)`` with ``r = (j k) mod n``
  reduced in int64 before the float conversion, so every angle is below 2 pi.
* ``dft3_bruteforce`` multiplies by the full ``N x N`` matrix of Eq. (1)
  (N = Nx Ny Nz); it is an independent check of the factorisation on tiny
  grids.
* ``dft3_at`` evaluates single outputs Y(k) of Eq. (1) directly, for sampled
  checks on grids too large for ``dft3``.

Everything is float64 / complex128.  Inputs are upcast exactly.
"""

from __future__ import annotations

import numpy as np

FORWARD = -1   # exponent sign of Eq. (1)
BACKWARD = +1  # exponent sign of Eq. (2)

__all__ = [
    "FORWARD",
    "BACKWARD",
    "dft_matrix",
    "dft_along_axis",
    "dft3",
    "forward",
    "backward",
    "dft3_bruteforce",
    "dft3_at",
    "rel_l2",
]


def _check_sign(sign: int) -> int:
    if sign not in (FORWARD, BACKWARD):
        raise ValueError("sign must be -1 (forward, Eq. 1) or +1 (backward, Eq. 2)")
    return sign


def dft_matrix(n: int, sign: int) -> np.ndarray:
    """n x n DFT matrix W[k, j] = exp(sign * 2 pi i * ((j*k) mod n) / n)  (Eq. 1 / Eq. 2 per axis)."""
    _check_sign(sign)
    idx = np.arange(n, dtype=np.int64)
    r = np.outer(idx, idx) % n  # row k, column j
    return np.exp(sign * 2j * np.pi * (r.astype(np.float64) / n))


def dft_along_axis(x: np.ndarray, axis: int, sign: int) -> np.ndarray:
    """One-axis DFT: out[..., k, ...] = sum_j W[k, j] x[..., j, ...] along ``axis``."""
    n = x.shape[axis]
    w = dft_matrix(n, sign)
    xm = np.moveaxis(x, axis, -1)           # (..., j)
    ym = np.matmul(xm, w.T)                 # (..., k) = sum_j x[..., j] W[k, j]
    return np.moveaxis(ym, -1, axis)


def dft3(x: np.ndarray, sign: int) -> np.ndarray:
    """Unnormalised 3D DFT of a (nx, ny, nz) array: Eq. (1) for sign=-1, Eq. (2) without 1/N for sign=+1."""
    _check_sign(sign)
    y = np.asarray(x).astype(np.complex128)
    if y.ndim != 3:
        raise ValueError("expected a 3D array (nx, ny, nz)")
    for axis in (2, 1, 0):                   # z, then y, then x
        y = dft_along_axis(y, axis, sign)
    return y


def forward(x: np.ndarray) -> np.ndarray:
    """Eq. (1)."""
    return dft3(x, FORWARD)


def backward(x: np.ndarray) -> np.ndarray:
    """Eq. (2) with the exponent sign +, unnormalised."""
    return dft3(x, BACKWARD)


def dft3_bruteforce(x: np.ndarray, sign: int) -> np.ndarray:
    """Eq. (1)/(2) as one dense N x N matrix-vector product (tiny grids only).

    Phase of entry (k, j) = (kx jx mod Nx)/Nx + (ky jy mod Ny)/Ny + (kz jz mod Nz)/Nz.
    """
    _check_sign(sign)
    x = np.asarray(x).astype(np.complex128)
    nx, ny, nz = x.shape
    n_total = nx * ny * nz
    if n_total > 4096:
        raise ValueError("brute force is for tiny grids (N <= 4096)")
    jx, jy, jz = np.meshgrid(np.arange(nx, dtype=np.int64), np.arange(ny, dtype=np.int64),
                             np.arange(nz, dtype=np.int64), indexing="ij")
    jx, jy, jz = jx.ravel(), jy.ravel(), jz.ravel()
    phase = (np.outer(jx, jx) % nx) / nx + (np.outer(jy, jy) % ny) / ny + (np.outer(jz, jz) % nz) / nz
    f = np.exp(sign * 2j * np.pi * phase)   # symmetric: row = k, column = j
    return (f @ x.ravel()).reshape(nx, ny, nz)


def dft3_at(x: np.ndarray, ks, sign: int) -> np.ndarray:
    """Selected outputs Y(k) of Eq. (1)/(2), each summed over the whole grid.

    ``ks`` is an (S, 3) integer array of output indices.  For each k the triple
    sum is contracted axis by axis (z, then y, then x) with the 1D phase
    vectors exp(sign 2 pi i (k_a j_a mod N_a)/N_a); cost O(N) per sample.
    """
    _check_sign(sign)
    x = np.asarray(x)
    nx, ny, nz = x.shape
    ks = np.asarray(ks, dtype=np.int64).reshape(-1, 3)
    out = np.empty(len(ks), dtype=np.complex128)

    def phase_vec(k, n):
        j = np.arange(n, dtype=np.int64)
        return np.exp(sign * 2j * np.pi * (((k * j) % n).astype(np.float64) / n))

    # group samples by kz so the O(N) z-contraction is shared
    order = np.argsort(ks[:, 2], kind="stable")
    i = 0
    while i < len(order):
        kz = ks[order[i], 2]
        grp = [order[i]]
        i += 1
        while i < len(order) and ks[order[i], 2] == kz:
            grp.append(order[i])
            i += 1
        ez = phase_vec(kz, nz)
        # z-contraction over the complex64 input, upcast in slabs of x to bound memory
        plane = np.empty((nx, ny), dtype=np.complex128)
        step = max(1, (1 << 24) // max(1, ny * nz))
        for x0 in range(0, nx, step):
            plane[x0:x0 + step] = x[x0:x0 + step].astype(np.complex128) @ ez
        for g in grp:
            kx, ky, _ = ks[g]
            out[g] = phase_vec(kx, nx) @ (plane @ phase_vec(ky, ny))
    return out


def rel_l2(y: np.ndarray, y_ref: np.ndarray) -> float:
    """||y - y_ref||_2 / ||y_ref||_2, accumulated in float64."""
    y = np.asarray(y).astype(np.complex128).ravel()
    y_ref = np.asarray(y_ref).astype(np.complex128).ravel()
    den = np.sqrt(np.sum(np.abs(y_ref) ** 2))
    num = np.sqrt(np.sum(np.abs(y - y_ref) ** 2))
    return float(num / den) if den > 0 else float(num)
