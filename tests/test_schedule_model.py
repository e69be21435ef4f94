"""Host model of the pass kernel's Stockham indexing (CPU only).

Replays, in numpy, exactly the index arithmetic of the pass kernels (butterfly
b reads x[b + j n/R], twiddles input j with table entry p-1 + (j-1) p + k,
writes output j to (b-k) R + k + j p) with the library's own radix schedule
and float32 twiddle table, and checks that the result is the length-n DFT of
the oracle and that every index stays in bounds.  This pins the schedule /
twiddle-table layout contract between the planner and the kernels before any
GPU run.
"""

import numpy as np
import pytest

import oracle


def _supported(n):
    m = n
    for p in (2, 3, 5):
        while m % p == 0:
            m //= p
    return m == 1


def stockham_model(x, radices, tw):
    n = x.shape[-1]
    p = 1
    for R in radices:
        nb = n // R
        y = np.zeros_like(x)
        written = np.zeros(n, dtype=np.int64)
        for b in range(nb):
            k = b % p
            src = [b + j * nb for j in range(R)]
            assert max(src) < n
            u = x[..., src].copy()
            for j in range(1, R):
                ti = p - 1 + (j - 1) * p + k
                assert 0 <= ti < n - 1
                u[..., j] *= tw[ti]
            Y = np.fft.fft(u, axis=-1)  # the in-register radix-R DFT
            for j in range(R):
                o = (b - k) * R + k + j * p
                assert 0 <= o < n
                written[o] += 1
                y[..., o] = Y[..., j]
        assert np.all(written == 1)  # every output written exactly once per stage
        x = y
        p *= R
    return x


@pytest.mark.parametrize("n", [n for n in range(2, 1100) if _supported(n)][::3] + [2048, 3888, 4096])
def test_stockham_model_matches_dft(croft_lib, n):
    radices = croft_lib.croft_factorize(n)
    tw = croft_lib.croft_twiddle_table(n, radices).astype(np.complex128)
    rng = np.random.default_rng(n)
    x = rng.standard_normal((2, n)) + 1j * rng.standard_normal((2, n))
    y = stockham_model(x, radices, tw)
    ref = oracle.dft_along_axis(x, 1, oracle.FORWARD)
    err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    assert err < 1e-6, (n, radices, err)  # float32 twiddles, float64 arithmetic
