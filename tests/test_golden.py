"""Stored fixtures under tests/golden/ (written by tests/golden/make_golden.py from the oracle).

CPU: the fixture inputs regenerate bit for bit and the oracle still reproduces the stored
outputs.  GPU: the CUDA path matches the stored outputs within the transform tolerance.
"""

import math
import os

import numpy as np
import pytest

import oracle

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name, shape):
    x = np.zeros(shape, dtype=np.complex64)
    y = np.zeros(shape, dtype=np.complex128)
    with open(os.path.join(HERE, name)) as f:
        lines = [ln.split() for ln in f if not ln.startswith("#")]
    assert len(lines) == int(np.prod(shape))
    for v in lines:
        i, j, k = int(v[0]), int(v[1]), int(v[2])
        x[i, j, k] = np.float32(v[3]) + 1j * np.float32(v[4])
        y[i, j, k] = float(v[5]) + 1j * float(v[6])
    return x, y


def _load_g(shape):
    g = np.zeros(shape, dtype=np.float32)
    with open(os.path.join(HERE, "convolve_3x4x5_g.txt")) as f:
        for ln in f:
            if ln.startswith("#"):
                continue
            v = ln.split()
            g[int(v[0]), int(v[1]), int(v[2])] = np.float32(v[3])
    return g


def _fixture_inputs():
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.inputs()


def test_fixture_inputs_regenerate_exactly():
    x, xc, g = _fixture_inputs()
    xf, _ = _load("dft3_forward_2x3x5.txt", (2, 3, 5))
    xcf, _ = _load("convolve_3x4x5.txt", (3, 4, 5))
    assert np.array_equal(x, xf) and np.array_equal(xc, xcf) and np.array_equal(g, _load_g((3, 4, 5)))


@pytest.mark.parametrize("name,fn", [("dft3_forward_2x3x5.txt", oracle.forward),
                                     ("dft3_backward_2x3x5.txt", oracle.backward)])
def test_oracle_reproduces_stored_transforms(name, fn):
    x, y = _load(name, (2, 3, 5))
    assert oracle.rel_l2(fn(x), y) <= 1e-15


def test_oracle_reproduces_stored_convolution():
    x, y = _load("convolve_3x4x5.txt", (3, 4, 5))
    assert oracle.rel_l2(oracle.convolve(x, _load_g((3, 4, 5))), y) <= 1e-15


@pytest.mark.gpu
def test_gpu_matches_stored_values(croft_lib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    x, yf = _load("dft3_forward_2x3x5.txt", (2, 3, 5))
    _, yb = _load("dft3_backward_2x3x5.txt", (2, 3, 5))
    tol = 2e-6 * math.log2(x.size)
    d = torch.from_numpy(x).cuda()
    with croft_lib.Plan(2, 3, 5) as p:
        f = p.forward(d).cpu().numpy()
        b = p.backward(d).cpu().numpy()
    assert oracle.rel_l2(f, yf) <= tol and oracle.rel_l2(b, yb) <= tol
    xc, yc = _load("convolve_3x4x5.txt", (3, 4, 5))
    g = torch.from_numpy(_load_g((3, 4, 5))).cuda()
    with croft_lib.Plan(3, 4, 5) as p:
        c = p.convolve(torch.from_numpy(xc).cuda(), g).cpu().numpy()
    assert oracle.rel_l2(c, yc) <= 2 * 2e-6 * math.log2(xc.size)
