"""The convolution oracle against its pins, and planted mistakes that the pins must catch (CPU only)."""

import inspect
import types

import numpy as np
import pytest

import oracle.convolution as C
from tests import oracle_pins_conv as P

SRC = inspect.getsource(C).replace("from .direct_dft import", "from oracle.direct_dft import")

MUTATIONS = {
    "g_not_applied": ("y = y * g.astype(np.float64)", "y = y * 1.0"),
    "g_reversed": ("y = y * g.astype(np.float64)", "y = y * g[::-1, ::-1, ::-1].astype(np.float64)"),
    "g_axes_swapped": ("y = y * g.astype(np.float64)", "y = y * np.swapaxes(g, 0, 2).astype(np.float64)"),
    "g_squared": ("y = y * g.astype(np.float64)", "y = y * g.astype(np.float64) ** 2"),
    "forward_twice": ("return backward(y)", "return forward(y)"),
    "backward_first": ("y = forward(x)", "y = backward(x)"),
    "normalised": ("return backward(y)", "return backward(y) / y.size"),
    "input_conjugated": ("y = forward(x)", "y = forward(np.conj(x))"),
}


@pytest.mark.parametrize("pin", P.ALL_CONV_PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin(C)


def test_rejects_bad_influence():
    with pytest.raises(ValueError):
        C.convolve(np.zeros((2, 2, 2)), np.zeros((2, 2, 3)))
    with pytest.raises(ValueError):
        C.convolve(np.zeros((2, 2, 2)), np.zeros((2, 2, 2), dtype=np.complex128))


def _mutant(name):
    old, new = MUTATIONS[name]
    assert SRC.count(old) >= 1, f"mutation anchor for {name} not found"
    mod = types.ModuleType(f"conv_mutant_{name}")
    exec(compile(SRC.replace(old, new), f"<conv mutant {name}>", "exec"), mod.__dict__)
    return mod


def _failures(mod):
    out = []
    for pin in P.ALL_CONV_PINS:
        try:
            pin(mod)
        except Exception as e:  # noqa: BLE001 - any failure counts as detection
            out.append((pin.__name__, type(e).__name__))
    return out


def test_unmutated_copy_passes():
    mod = types.ModuleType("conv_copy")
    exec(compile(SRC, "<conv copy>", "exec"), mod.__dict__)
    assert _failures(mod) == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name):
    assert _failures(_mutant(name)), f"no pin caught the planted mistake {name}"
