"""Pins that tie the FP64 oracle to facts fixed by the DFT's definition (Eq. 1, Eq. 2).

Each ``pin_*`` takes an oracle *module* (the real ``oracle.direct_dft`` or a copy with
a planted mistake) and raises ``AssertionError`` when the module disagrees with
an expectation that does not come from the module itself:

* closed forms of Eq. (1) for special inputs (delta, constant, plane wave,
  hand-derived small transforms),
* invariants of the exact transform (Parseval, linearity, circular shift,
  Hermitian symmetry of real input, backward(forward(x)) = N x under the
  unnormalised reading of Eq. (2)),
* an independent formulation (the dense N x N matrix of Eq. (1) on tiny grids,
  single-output sums),
* a library routine (numpy's pocketfft in float64) standing in for the FFTW3
  cross-check of Sec. 5.3.

The pins are chosen so that a plausible slip anywhere in the oracle (a wrong
sign, a dropped term or axis, a wrong index, a stray normalisation, a
conjugation) fails at least one of them; ``test_oracle_mutations.py`` plants
such slips and checks exactly that.
"""

from __future__ import annotations

import numpy as np

SHAPES_SMALL = [(1, 1, 1), (2, 2, 2), (2, 3, 5), (8, 6, 4), (3, 1, 4), (5, 4, 3), (1, 7, 2),
                (4, 4, 4), (6, 5, 2), (8, 8, 8)]


def _rng(seed):
    return np.random.default_rng(seed)


def _cnoise(shape, seed):
    r = _rng(seed)
    return r.standard_normal(shape) + 1j * r.standard_normal(shape)


def _close(a, b, rtol, what):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    assert a.shape == b.shape, f"{what}: shape {a.shape} != {b.shape}"
    scale = max(1.0, float(np.max(np.abs(b))) if b.size else 1.0)
    err = float(np.max(np.abs(a - b))) if a.size else 0.0
    assert err <= rtol * scale, f"{what}: max err {err:.3e} > {rtol:.1e} * {scale:.3e}"


# ---------------------------------------------------------------------------
# hand-derived closed forms (textbook special cases of Eq. 1)
# ---------------------------------------------------------------------------

def pin_textbook_1d(o):
    """1 x 1 x n grids reduce Eq. (1) to the 1D DFT; small cases worked by hand.

    * n = 2: Y = (x0 + x1, x0 - x1).
    * n = 4, x = (1, 2, 3, 4): Y = (10, -2 + 2i, -2, -2 - 2i).
    * n = 3, x = (1, 0, 0) -> all ones; x = (0, 1, 0) -> (1, w, w^2),
      w = exp(-2 pi i / 3) = -1/2 - i sqrt(3)/2.
    * backward of n = 4, x = (1, 2, 3, 4): (10, -2 - 2i, -2, -2 + 2i).
    """
    y = o.forward(np.array([3.0, 5.0]).reshape(1, 1, 2))
    _close(y.ravel(), [8.0, -2.0], 1e-14, "n=2")
    y = o.forward(np.array([1.0, 2.0, 3.0, 4.0]).reshape(1, 1, 4))
    _close(y.ravel(), [10, -2 + 2j, -2, -2 - 2j], 1e-14, "n=4 forward")
    y = o.backward(np.array([1.0, 2.0, 3.0, 4.0]).reshape(1, 1, 4))
    _close(y.ravel(), [10, -2 - 2j, -2, -2 + 2j], 1e-14, "n=4 backward")
    w = complex(-0.5, -np.sqrt(3.0) / 2.0)
    y = o.forward(np.array([0.0, 1.0, 0.0]).reshape(1, 1, 3))
    _close(y.ravel(), [1.0, w, w * w], 1e-14, "n=3 delta at 1")
    # the same along the other two axes (axis handling)
    y = o.forward(np.array([1.0, 2.0, 3.0, 4.0]).reshape(4, 1, 1))
    _close(y.ravel(), [10, -2 + 2j, -2, -2 - 2j], 1e-14, "n=4 along x")
    y = o.forward(np.array([1.0, 2.0, 3.0, 4.0]).reshape(1, 4, 1))
    _close(y.ravel(), [10, -2 + 2j, -2, -2 - 2j], 1e-14, "n=4 along y")


def pin_textbook_2x2x2(o):
    """2x2x2: every phase factor is +-1, so Y(k) = sum_j (-1)^(k.j) X(j) (exact integers)."""
    x = np.arange(1, 9, dtype=np.float64).reshape(2, 2, 2)
    # Hand evaluation: Y(0) = 36; for k != 0 the (+1,-1) sums over the index
    # bits give Y(0,0,1) = -4, Y(0,1,0) = -8, Y(1,0,0) = -16, all others 0.
    expect = np.zeros((2, 2, 2))
    expect[0, 0, 0] = 36
    expect[0, 0, 1] = -4
    expect[0, 1, 0] = -8
    expect[1, 0, 0] = -16
    _close(o.forward(x), expect, 1e-14, "2x2x2 forward")
    _close(o.backward(x), expect, 1e-14, "2x2x2 backward")


def pin_delta(o):
    """X = delta at (a, b, c) -> Y(k) = exp(-2 pi i (kx a/Nx + ky b/Ny + kz c/Nz)); delta at 0 -> ones."""
    for shape, at in [((4, 6, 5), (1, 2, 3)), ((8, 3, 2), (7, 0, 1)), ((5, 5, 5), (0, 0, 0))]:
        x = np.zeros(shape, dtype=np.complex128)
        x[at] = 1.0
        kx, ky, kz = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
        ang = 2 * np.pi * (kx * at[0] / shape[0] + ky * at[1] / shape[1] + kz * at[2] / shape[2])
        _close(o.forward(x), np.cos(ang) - 1j * np.sin(ang), 1e-13, f"delta fwd {shape}")
        _close(o.backward(x), np.cos(ang) + 1j * np.sin(ang), 1e-13, f"delta bwd {shape}")


def pin_constant(o):
    """X = 1 everywhere -> Y = N at k = 0 and 0 elsewhere."""
    for shape in [(4, 6, 5), (3, 3, 8)]:
        x = np.ones(shape)
        expect = np.zeros(shape)
        expect[0, 0, 0] = np.prod(shape)
        _close(o.forward(x), expect, 1e-13, f"constant {shape}")


def pin_plane_wave(o):
    """X(j) = exp(+2 pi i p.j/N) -> forward gives a single spike N at k = p."""
    for shape, p in [((4, 6, 5), (3, 1, 4)), ((6, 4, 9), (5, 3, 2))]:
        jx, jy, jz = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
        ang = 2 * np.pi * (p[0] * jx / shape[0] + p[1] * jy / shape[1] + p[2] * jz / shape[2])
        x = np.cos(ang) + 1j * np.sin(ang)
        expect = np.zeros(shape, dtype=np.complex128)
        expect[p] = np.prod(shape)
        _close(o.forward(x), expect, 1e-12, f"plane wave fwd {shape}")
        expect_b = np.zeros(shape, dtype=np.complex128)
        expect_b[tuple((-np.array(p)) % np.array(shape))] = np.prod(shape)
        _close(o.backward(x), expect_b, 1e-12, f"plane wave bwd {shape}")


# ---------------------------------------------------------------------------
# invariants
# ---------------------------------------------------------------------------

def pin_parseval(o):
    for shape in [(4, 6, 5), (8, 8, 8), (3, 10, 2)]:
        x = _cnoise(shape, 11)
        y = o.forward(x)
        lhs = np.sum(np.abs(y) ** 2)
        rhs = np.prod(shape) * np.sum(np.abs(x) ** 2)
        assert abs(lhs - rhs) <= 1e-12 * rhs, f"Parseval {shape}: {lhs} vs {rhs}"


def pin_linearity(o):
    shape = (6, 4, 5)
    x = _cnoise(shape, 1)
    z = _cnoise(shape, 2)
    a, b = 0.7 - 1.3j, -2.1 + 0.4j
    _close(o.forward(a * x + b * z), a * o.forward(x) + b * o.forward(z), 1e-13, "linearity")


def pin_shift(o):
    """F(X(j - s))(k) = exp(-2 pi i sum_a k_a s_a / N_a) F(X)(k) for a circular shift s."""
    shape = (6, 4, 5)
    s = (2, 3, 1)
    x = _cnoise(shape, 3)
    xs = np.roll(x, shift=s, axis=(0, 1, 2))
    kx, ky, kz = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    ang = 2 * np.pi * (kx * s[0] / shape[0] + ky * s[1] / shape[1] + kz * s[2] / shape[2])
    _close(o.forward(xs), (np.cos(ang) - 1j * np.sin(ang)) * o.forward(x), 1e-13, "shift")


def pin_round_trip(o):
    """backward(forward(X)) = N X (unnormalised Eq. 2; the paper's own check, Sec. 5.3)."""
    for shape in [(4, 6, 5), (8, 8, 8), (1, 3, 16)]:
        x = _cnoise(shape, 4)
        _close(o.backward(o.forward(x)), np.prod(shape) * x, 1e-13, f"round trip {shape}")


def pin_hermitian(o):
    """Real X -> Y(-k mod N) = conj(Y(k))."""
    shape = (6, 5, 4)
    x = _rng(5).standard_normal(shape)
    y = o.forward(x)
    idx = [(-np.arange(n)) % n for n in shape]
    y_neg = y[np.ix_(*idx)]
    _close(y_neg, np.conj(y), 1e-13, "Hermitian")


def pin_pme_dc(o):
    """Net-zero charges spread with B-spline weights (each summing to 1) -> Y(0,0,0) = sum q = 0."""
    from synthetic_inputs import spread_charges
    rng = _rng(6)
    pos = rng.random((1000, 3))
    q = rng.permutation(np.concatenate([np.ones(500), -np.ones(500)]))
    g = spread_charges((8, 6, 10), pos, q)
    y = o.forward(g)
    assert abs(y[0, 0, 0]) <= 1e-11, f"PME DC {y[0, 0, 0]}"
    # and the DC of a positive-only spread is the total charge
    g1 = spread_charges((8, 6, 10), pos, np.ones(1000))
    assert abs(o.forward(g1)[0, 0, 0] - 1000.0) <= 1e-9


# ---------------------------------------------------------------------------
# independent formulations and the library pin
# ---------------------------------------------------------------------------

def pin_bruteforce(o):
    """Per-axis factorisation == the dense N x N matrix of Eq. (1) on every small shape."""
    for i, shape in enumerate(SHAPES_SMALL):
        x = _cnoise(shape, 100 + i)
        for sign in (o.FORWARD, o.BACKWARD):
            _close(o.dft3(x, sign), o.dft3_bruteforce(x, sign), 1e-13, f"brute {shape} {sign}")


def pin_numpy(o):
    """numpy.fft (pocketfft, float64) agrees: fftn == forward, N * ifftn == backward."""
    for i, shape in enumerate([(4, 6, 5), (8, 8, 8), (16, 12, 10), (2, 3, 30)]):
        x = _cnoise(shape, 200 + i)
        _close(o.forward(x), np.fft.fftn(x), 1e-12, f"numpy fwd {shape}")
        _close(o.backward(x), np.fft.ifftn(x) * np.prod(shape), 1e-12, f"numpy bwd {shape}")


def pin_sampled(o):
    """Single-output sums dft3_at agree with the full transform (and with numpy)."""
    shape = (12, 10, 9)
    x = _cnoise(shape, 7).astype(np.complex64)
    ks = np.array([[0, 0, 0], [11, 9, 8], [3, 7, 2], [6, 5, 4], [1, 0, 8]])
    ref = np.fft.fftn(x.astype(np.complex128))
    got = o.dft3_at(x, ks, o.FORWARD)
    _close(got, ref[ks[:, 0], ks[:, 1], ks[:, 2]], 1e-12, "sampled fwd")
    refb = np.fft.ifftn(x.astype(np.complex128)) * np.prod(shape)
    gotb = o.dft3_at(x, ks, o.BACKWARD)
    _close(gotb, refb[ks[:, 0], ks[:, 1], ks[:, 2]], 1e-12, "sampled bwd")


def pin_rel_l2(o):
    a = np.array([3.0, 4.0])
    assert abs(o.rel_l2(a, a) - 0.0) == 0.0
    assert abs(o.rel_l2(np.array([3.0, 6.0]), a) - 0.4) < 1e-15  # |(0,2)| / |(3,4)| = 2/5
    assert abs(o.rel_l2(np.array([3.0 + 2.0j, 4.0]), a) - 0.4) < 1e-15  # complex modulus |2i| = 2


ALL_PINS = [
    pin_textbook_1d, pin_textbook_2x2x2, pin_delta, pin_constant, pin_plane_wave,
    pin_parseval, pin_linearity, pin_shift, pin_round_trip, pin_hermitian, pin_pme_dc,
    pin_bruteforce, pin_numpy, pin_sampled, pin_rel_l2,
]
