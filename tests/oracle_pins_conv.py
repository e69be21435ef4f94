"""Pins that tie the convolution oracle (``oracle.convolution``) to facts outside itself.

``convolve(X, G) = B(G * F(X))`` is the reciprocal-space step of the PME
method (paper Sec. 1) built from Eq. (1) and the unnormalised Eq. (2).  Each
``pin_*`` takes a module with a ``convolve`` function (the real one or a copy
with a planted mistake) and raises ``AssertionError`` on disagreement with:

* closed forms: G = 1 gives N X; G = a single mode k0 gives one plane wave whose
  amplitude is the k0-th Fourier coefficient of X, summed here term by term;
* the convolution theorem: the output is the circular convolution of X with
  h = B(G), both evaluated here by explicit sums on tiny grids;
* invariants: circular shift equivariance, linearity in G, a real output for
  real X and a real even G, and the energy identity
  <X, convolve(X, G)> = sum_k G(k) |F(X)(k)|^2 (the PME reciprocal energy form);
* a library routine: numpy's pocketfft, N * ifftn(G * fftn(X)).
"""

from __future__ import annotations

import numpy as np

SHAPES_TINY = [(1, 1, 1), (2, 3, 4), (3, 1, 5), (4, 4, 2), (1, 6, 5), (5, 3, 3)]


def _cnoise(shape, seed):
    r = np.random.default_rng(seed)
    return r.standard_normal(shape) + 1j * r.standard_normal(shape)


def _rnoise(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def _close(a, b, rtol, what):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    assert a.shape == b.shape, f"{what}: shape {a.shape} != {b.shape}"
    scale = max(1.0, float(np.max(np.abs(b))) if b.size else 1.0)
    err = float(np.max(np.abs(a - b))) if a.size else 0.0
    assert err <= rtol * scale, f"{what}: max err {err:.3e} > {rtol:.1e} * {scale:.3e}"


def _phase(kvec, jvec, shape):
    """sum_a (k_a j_a mod n_a) / n_a for integer index arrays (broadcast)."""
    return sum(((kvec[a] * jvec[a]) % shape[a]) / shape[a] for a in range(3))


def pin_conv_identity(c):
    """G = 1 everywhere: B(F(X)) = N X under the unnormalised reading of Eq. (2)."""
    for i, shape in enumerate(SHAPES_TINY + [(8, 6, 10)]):
        x = _cnoise(shape, 300 + i)
        _close(c.convolve(x, np.ones(shape)), np.prod(shape) * x, 1e-12, f"identity {shape}")


def pin_conv_single_mode(c):
    """G = indicator of k0: out(j) = Xhat(k0) exp(+2 pi i k0.j / n), Xhat(k0) = sum_m X(m) exp(-2 pi i k0.m / n)."""
    shape = (4, 6, 5)
    x = _cnoise(shape, 310)
    j = np.indices(shape).reshape(3, -1).astype(np.int64)
    for k0 in [(0, 0, 0), (1, 2, 3), (3, 5, 4), (2, 0, 1)]:
        g = np.zeros(shape)
        g[k0] = 1.0
        kv = [np.int64(v) for v in k0]
        xhat = np.sum(x.ravel() * np.exp(-2j * np.pi * _phase(kv, j, shape)))
        want = (xhat * np.exp(2j * np.pi * _phase(kv, j, shape))).reshape(shape)
        _close(c.convolve(x, g), want, 1e-12, f"single mode {k0}")


def pin_conv_circular(c):
    """Convolution theorem on tiny grids: out(j) = sum_m X(m) h(j - m mod n), h(r) = sum_k G(k) exp(+2 pi i k.r / n)."""
    for i, shape in enumerate(SHAPES_TINY):
        x = _cnoise(shape, 320 + i)
        g = _rnoise(shape, 330 + i)
        idx = np.indices(shape).reshape(3, -1).astype(np.int64)  # all grid points, (3, N)
        n_tot = idx.shape[1]
        h = np.empty(n_tot, dtype=np.complex128)
        for r in range(n_tot):
            h[r] = np.sum(g.ravel() * np.exp(2j * np.pi * _phase(idx, idx[:, r:r + 1], shape)))
        h = h.reshape(shape)
        out = np.zeros(shape, dtype=np.complex128)
        for m in range(n_tot):
            mx, my, mz = idx[:, m]
            shifted = np.roll(h, (mx, my, mz), axis=(0, 1, 2))  # shifted[j] = h[j - m]
            out += x[mx, my, mz] * shifted
        _close(c.convolve(x, g), out, 1e-11, f"circular convolution {shape}")


def pin_conv_numpy(c):
    """numpy's pocketfft in float64: N * ifftn(G * fftn(X))."""
    for i, shape in enumerate([(8, 8, 8), (6, 10, 4), (16, 12, 9), (2, 1, 30)]):
        x = _cnoise(shape, 340 + i)
        g = _rnoise(shape, 350 + i)
        want = np.fft.ifftn(g * np.fft.fftn(x)) * np.prod(shape)
        _close(c.convolve(x, g), want, 1e-12, f"numpy {shape}")


def pin_conv_energy(c):
    """<X, convolve(X, G)> = sum_k G(k) |Xhat(k)|^2 (Xhat from numpy's fftn)."""
    shape = (6, 8, 10)
    x = _cnoise(shape, 360)
    g = _rnoise(shape, 361)
    lhs = np.vdot(x, c.convolve(x, g))
    rhs = np.sum(g * np.abs(np.fft.fftn(x)) ** 2)
    assert abs(lhs - rhs) <= 1e-11 * abs(rhs), f"energy {lhs} vs {rhs}"


def pin_conv_shift(c):
    """Circular shift of X shifts the output by the same amount."""
    shape = (5, 6, 4)
    x = _cnoise(shape, 370)
    g = _rnoise(shape, 371)
    s = (2, 5, 1)
    _close(c.convolve(np.roll(x, s, axis=(0, 1, 2)), g), np.roll(c.convolve(x, g), s, axis=(0, 1, 2)), 1e-12, "shift")


def pin_conv_linear_in_g(c):
    shape = (4, 5, 6)
    x = _cnoise(shape, 380)
    g1, g2 = _rnoise(shape, 381), _rnoise(shape, 382)
    _close(c.convolve(x, 2.0 * g1 - 0.5 * g2), 2.0 * c.convolve(x, g1) - 0.5 * c.convolve(x, g2), 1e-12, "linear in G")


def pin_conv_real_even(c):
    """Real X and the PME influence function (real, even, zero at k = 0): real output, zero mean."""
    from synthetic_inputs import pme_influence
    shape = (8, 6, 10)
    g = pme_influence(shape, dtype=np.float64)
    neg = g[np.ix_(*[(-np.arange(n)) % n for n in shape])]
    assert np.allclose(neg, g, rtol=1e-13, atol=0), "influence function is not even"
    assert g[0, 0, 0] == 0.0 and np.all(g[g != 0] > 0)
    x = _rnoise(shape, 390)
    y = c.convolve(x, g)
    assert np.max(np.abs(y.imag)) <= 1e-12 * np.max(np.abs(y.real)), "imaginary part of a real even convolution"
    assert abs(np.sum(y)) <= 1e-12 * np.sum(np.abs(y)), "G(0) = 0 must remove the mean"


ALL_CONV_PINS = [
    pin_conv_identity, pin_conv_single_mode, pin_conv_circular, pin_conv_numpy, pin_conv_energy,
    pin_conv_shift, pin_conv_linear_in_g, pin_conv_real_even,
]
