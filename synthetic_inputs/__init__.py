"""Seeded synthetic inputs for the 3D complex-to-complex DFT.

This module is shared by the CPU oracle (``oracle/``) and the CUDA path
(tests, ``bench.py``).  It holds no arithmetic of the transform itself: it only
draws random numbers and spreads point charges onto a mesh, the way a
particle-mesh Ewald (PME) code fills the grid it hands to the forward 3D FFT
(the motivating application of the paper, Sec. 1).

Every generator works in float64 and casts to complex64 at the very end, so the
GPU and the oracle receive bit-identical complex64 buffers.

Grid layout everywhere: array shape ``(nx, ny, nz)``, C order, ``z`` contiguous.

Recipes (one per workload):

* ``white_noise(shape, seed)``: real and imaginary parts iid uniform[-1, 1)
  drawn as one ``(nx, ny, nz, 2)`` array from ``numpy.random.default_rng(seed)``.
* ``pme_charge_grid(shape, n_charges, rng)``: ``n_charges`` point charges at
  iid uniform positions in the unit cube (drawn first, as an ``(M, 3)`` array),
  charges +1/-1 in equal numbers in a random order (drawn second, as a
  permutation), spread with the order-4 cardinal B-spline (64 mesh points per
  charge).  The imaginary part is zero.
* ``pme_batch(count, seed)``: the batch of uneven grids (each axis length
  drawn from a fixed menu, 2 * U{10000..100000} charges per grid).
* ``pme_influence(shape)``: the real reciprocal-space influence function that
  a smooth-PME code multiplies the transformed charge grid by before the
  backward transform (no random draws; a fixed function of the mesh).
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "white_noise",
    "bspline4_weights",
    "pme_charge_grid",
    "pme_batch",
    "config_input",
    "pme_influence",
    "BATCH_AXIS_CHOICES",
]

# Axis lengths of the per-system PME meshes in the batched workload.
BATCH_AXIS_CHOICES = (48, 60, 64, 72, 80, 96, 120, 128)


def white_noise(shape, seed: int) -> np.ndarray:
    """complex64 grid with real/imag parts iid uniform[-1, 1) (one draw)."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(-1.0, 1.0, tuple(shape) + (2,))
    return (a[..., 0] + 1j * a[..., 1]).astype(np.complex64)


def bspline4_weights(w: np.ndarray) -> np.ndarray:
    """Uniform cubic (order-4 cardinal) B-spline weights for fractional offset w.

    For a charge at mesh coordinate ``u`` with ``i0 = floor(u)`` and
    ``w = u - i0`` the four weights land on mesh points ``i0-1 .. i0+2``.
    Returns an array of shape ``w.shape + (4,)``; the four weights sum to 1.
    """
    w = np.asarray(w, dtype=np.float64)
    w2 = w * w
    w3 = w2 * w
    b0 = (1.0 - w) ** 3 / 6.0
    b1 = (3.0 * w3 - 6.0 * w2 + 4.0) / 6.0
    b2 = (-3.0 * w3 + 3.0 * w2 + 3.0 * w + 1.0) / 6.0
    b3 = w3 / 6.0
    return np.stack([b0, b1, b2, b3], axis=-1)


def _draw_charges(rng: np.random.Generator, n_charges: int):
    if n_charges % 2:
        raise ValueError("n_charges must be even (net-zero +1/-1 charges)")
    pos = rng.random((n_charges, 3))
    half = n_charges // 2
    q = rng.permutation(np.concatenate([np.ones(half), -np.ones(half)]))
    return pos, q


def spread_charges(shape, pos: np.ndarray, q: np.ndarray, chunk: int = 1 << 19) -> np.ndarray:
    """Spread charges onto a float64 mesh with order-4 B-splines.

    Deterministic: charges are accumulated chunk by chunk in input order with
    ``numpy.bincount`` (a sequential sum), so the same inputs always give the
    same bits.
    """
    nx, ny, nz = (int(s) for s in shape)
    n_total = nx * ny * nz
    grid = np.zeros(n_total, dtype=np.float64)
    dims = np.array([nx, ny, nz], dtype=np.int64)
    for s in range(0, len(q), chunk):
        p = pos[s:s + chunk]
        qq = q[s:s + chunk]
        u = p * dims  # mesh coordinates, (C, 3)
        i0 = np.floor(u).astype(np.int64)
        w = u - i0
        wts = bspline4_weights(w)  # (C, 3, 4)
        offs = np.arange(-1, 3, dtype=np.int64)
        idx = (i0[:, :, None] + offs[None, None, :]) % dims[None, :, None]  # (C, 3, 4)
        flat = ((idx[:, 0, :, None, None] * ny + idx[:, 1, None, :, None]) * nz
                + idx[:, 2, None, None, :])
        val = (qq[:, None, None, None] * wts[:, 0, :, None, None]
               * wts[:, 1, None, :, None] * wts[:, 2, None, None, :])
        grid += np.bincount(flat.ravel(), weights=val.ravel(), minlength=n_total)
    return grid.reshape(nx, ny, nz)


def pme_charge_grid(shape, n_charges: int, rng: np.random.Generator) -> np.ndarray:
    """PME-shaped complex64 grid: B-spline-spread +-1 charges, imag part zero."""
    pos, q = _draw_charges(rng, n_charges)
    g = spread_charges(shape, pos, q)
    return g.astype(np.complex64)


def pme_batch(count: int = 96, seed: int = 3, choices=BATCH_AXIS_CHOICES):
    """The batch of uneven PME meshes: returns (dims list, list of complex64 grids).

    Draw order: all dims, then all charge counts, then per grid in order its
    positions and its charge permutation.
    """
    rng = np.random.default_rng(seed)
    dims = rng.choice(np.asarray(choices, dtype=np.int64), size=(count, 3))
    m = 2 * rng.integers(10000, 100001, size=count)
    grids = []
    for g in range(count):
        grids.append(pme_charge_grid(tuple(int(d) for d in dims[g]), int(m[g]), rng))
    return [tuple(int(d) for d in row) for row in dims], grids


def pme_influence(shape, spacing: float = 0.1, beta: float = 3.12, dtype=np.float32) -> np.ndarray:
    """Smooth-PME influence function G(k) on an (nx, ny, nz) mesh, indexed like the transform's output.

    Orthorhombic box with mesh spacing ``spacing`` on every axis (box side
    L_a = K_a * spacing) and Ewald splitting parameter ``beta`` (1/length).
    With the signed frequency m_a = k_a (k_a <= K_a/2) or k_a - K_a, the
    reciprocal vector f_a = m_a / L_a and V = L_x L_y L_z:

        G(k) = exp(-pi^2 |f|^2 / beta^2) / (pi V |f|^2) * prod_a |b_a(k_a)|^2,   G(0) = 0,

    where 1 / |b_a(k)|^2 = |sum_{t=0..2} M4(t+1) exp(2 pi i k t / K_a)|^2 with the
    order-4 cardinal B-spline values M4(1) = M4(3) = 1/6, M4(2) = 2/3 (the
    interpolation correction that goes with ``bspline4_weights``).  G is real
    and even (G(-k) = G(k)).  Computed in float64, cast to ``dtype`` at the end.
    """
    shape = tuple(int(s) for s in shape)
    axes_f2 = []
    axes_b2 = []
    for k_len in shape:
        k = np.arange(k_len, dtype=np.int64)
        m = np.where(k <= k_len // 2, k, k - k_len).astype(np.float64)
        axes_f2.append((m / (k_len * spacing)) ** 2)
        ph = 2.0 * np.pi * k.astype(np.float64) / k_len
        den = (1.0 / 6.0) + (2.0 / 3.0) * np.exp(1j * ph) + (1.0 / 6.0) * np.exp(2j * ph)
        axes_b2.append(1.0 / np.abs(den) ** 2)
    f2 = axes_f2[0][:, None, None] + axes_f2[1][None, :, None] + axes_f2[2][None, None, :]
    b2 = axes_b2[0][:, None, None] * axes_b2[1][None, :, None] * axes_b2[2][None, None, :]
    vol = float(np.prod([k_len * spacing for k_len in shape]))
    with np.errstate(divide="ignore", invalid="ignore"):
        g = np.exp(-(np.pi ** 2) * f2 / beta ** 2) / (np.pi * vol * f2) * b2
    g[0, 0, 0] = 0.0
    return g.astype(dtype)


def config_input(name: str):
    """Named workloads.  Returns a complex64 grid (or a list for multi-grid ones).

    * ``"noise32"``     : 32x32x32 white noise, seed 0.
    * ``"pme256"``      : 256^3, 200k charges, seed 1.
    * ``"pme480"`` / ``"pme384x360x320"``: one seed-2 stream, 2M charges each,
      480^3 drawn first.
    * ``"pme512"``      : 512^3, 8M charges, seed 4.
    """
    if name == "noise32":
        return white_noise((32, 32, 32), 0)
    if name == "pme256":
        return pme_charge_grid((256, 256, 256), 200_000, np.random.default_rng(1))
    if name in ("pme480", "pme384x360x320"):
        rng = np.random.default_rng(2)
        if name == "pme480":
            return pme_charge_grid((480, 480, 480), 2_000_000, rng)
        _draw_charges(rng, 2_000_000)  # the 480^3 grid's draws come first
        return pme_charge_grid((384, 360, 320), 2_000_000, rng)
    if name == "pme512":
        return pme_charge_grid((512, 512, 512), 8_000_000, np.random.default_rng(4))
    raise KeyError(name)
