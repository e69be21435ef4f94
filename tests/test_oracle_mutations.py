"""Plant plausible mistakes in a copy of the oracle and check that the pins catch each one.

The mistakes are planted in the oracle's own source text (on the CPU), the
copy is executed as a fresh module, and the full pin suite must reject it.
"""

import importlib.util
import inspect
import types

import pytest

import oracle.direct_dft as O
from tests import oracle_pins as P

SRC = inspect.getsource(O)

MUTATIONS = {
    "forward_sign_flipped": ("FORWARD = -1 ", "FORWARD = +1 "),
    "dropped_axis_y": ("for axis in (2, 1, 0):", "for axis in (2, 0):"),
    "axis_applied_twice": ("for axis in (2, 1, 0):", "for axis in (2, 2, 0):"),
    "twiddle_index_off_by_one": ("r = np.outer(idx, idx) % n", "r = np.outer(idx, idx + 1) % n"),
    "twiddle_sum_not_product": ("r = np.outer(idx, idx) % n", "r = np.add.outer(idx, idx) % n"),
    "half_angle": ("np.exp(sign * 2j * np.pi * (r.astype", "np.exp(sign * 1j * np.pi * (r.astype"),
    "dropped_first_term": ("ym = np.matmul(xm, w.T)", "ym = np.matmul(xm[..., 1:], w.T[1:, :])"),
    "dropped_last_term": ("ym = np.matmul(xm, w.T)", "ym = np.matmul(xm[..., :-1], w.T[:-1, :])"),
    "input_index_reversed": ("ym = np.matmul(xm, w.T)", "ym = np.matmul(xm[..., ::-1], w.T)"),
    "backward_normalised": ("return dft3(x, BACKWARD)\n", "return dft3(x, BACKWARD) / np.size(x)\n"),
    "input_conjugated": ("y = np.asarray(x).astype(np.complex128)\n    if y.ndim",
                         "y = np.conj(np.asarray(x).astype(np.complex128))\n    if y.ndim"),
    "output_axis_misplaced": ("return np.moveaxis(ym, -1, axis)", "return np.moveaxis(ym, -1, 0)"),
    "brute_phase_wrong_axis": ("(np.outer(jy, jy) % ny) / ny", "(np.outer(jy, jy) % ny) / nx"),
    "sampled_wrong_sign": ("return np.exp(sign * 2j * np.pi * (((k * j) % n)",
                           "return np.exp(-2j * np.pi * (((k * j) % n)"),
    "sampled_ky_kx_swapped": ("out[g] = phase_vec(kx, nx) @ (plane @ phase_vec(ky, ny))",
                              "out[g] = phase_vec(ky, nx) @ (plane @ phase_vec(kx, ny))"),
    "rel_l2_missing_sqrt": ("num = np.sqrt(np.sum(np.abs(y - y_ref) ** 2))",
                            "num = np.sum(np.abs(y - y_ref) ** 2)"),
}


def _mutant(name):
    old, new = MUTATIONS[name]
    assert SRC.count(old) >= 1, f"mutation anchor for {name} not found in the oracle source"
    src = SRC.replace(old, new)
    mod = types.ModuleType(f"oracle_mutant_{name}")
    exec(compile(src, f"<oracle mutant {name}>", "exec"), mod.__dict__)
    return mod


def _pins_reject(mod):
    failures = []
    for pin in P.ALL_PINS:
        try:
            pin(mod)
        except Exception as e:  # noqa: BLE001 - any failure counts as detection
            failures.append((pin.__name__, type(e).__name__))
    return failures


def test_unmutated_oracle_passes_all_pins():
    assert _pins_reject(O) == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name):
    failures = _pins_reject(_mutant(name))
    assert failures, f"no pin caught the planted mistake {name}"
