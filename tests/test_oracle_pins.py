"""The FP64 oracle against facts fixed by Eq. (1)/(2) (CPU only)."""

import numpy as np
import pytest

import oracle.direct_dft as O
from tests import oracle_pins as P


@pytest.mark.parametrize("pin", P.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin(O)


def test_sign_constants():
    assert O.FORWARD == -1 and O.BACKWARD == +1
    with pytest.raises(ValueError):
        O.dft3(np.zeros((2, 2, 2)), 0)


def test_large_angle_reduction():
    """Entries of the 4096-point DFT matrix keep unit modulus and exact symmetry points."""
    w = O.dft_matrix(4096, O.FORWARD)
    assert np.max(np.abs(np.abs(w) - 1.0)) < 1e-15
    # k*j = 1024 (mod 4096) is a quarter turn: exactly -i up to the float64 cos/sin rounding
    assert abs(w[32, 32] - (-1j)) < 1e-15
    # the matrix is symmetric, unitary up to a factor n
    assert np.allclose(w @ np.conj(w).T, 4096 * np.eye(4096), atol=1e-8)
