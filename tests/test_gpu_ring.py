"""Tensor-copy ring column kernel (croft_ring_kernel.cuh) vs the FP64 oracle (needs a GPU).

The kernel serves the column passes of the lengths whose pencils take 32 threads
(270..512); CROFT_RING=1 selects it for every such column pass (x and y), CROFT_RING=0
(and, as measured so far, the default) for none.  Every length is checked as the x axis and as the y axis,
with a ragged last tile (the column count is not a multiple of 16), forward and
backward, against the oracle at the FP32 bar.
"""

import math
import os

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

RING_LENGTHS = [270, 288, 300, 320, 324, 360, 375, 384, 400, 405, 432, 450, 480, 486, 500, 512]


def tol(shape):
    return 2e-6 * math.log2(int(np.prod(shape)))


class _env:
    def __init__(self, **kv):
        self.kv = kv
        self.old = {}

    def __enter__(self):
        for k, v in self.kv.items():
            self.old[k] = os.environ.get(k)
            os.environ[k] = v

    def __exit__(self, *exc):
        for k, v in self.old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def _check(croft, x, expect_ring):
    d = torch.from_numpy(x).cuda()
    with croft.Plan(*x.shape) as p:
        desc = p.describe()
        yf = p.forward(d)
        yb = p.backward(d)
        torch.cuda.synchronize()
        st = croft.croft_plan_last_device_status(p.handle)
    assert ("+ring" in desc) == expect_ring, desc
    assert st == croft.CROFT_OK
    t = tol(x.shape)
    ef = oracle.rel_l2(yf.cpu().numpy(), oracle.forward(x))
    eb = oracle.rel_l2(yb.cpu().numpy(), oracle.backward(x))
    assert ef <= t and eb <= t, (x.shape, ef, eb, t)
    return ef, eb


def _noise(shape, seed):
    rng = np.random.default_rng(seed)
    return (rng.uniform(-1, 1, shape) + 1j * rng.uniform(-1, 1, shape)).astype(np.complex64)


@pytest.mark.parametrize("n", RING_LENGTHS)
def test_ring_x_pass(croft_lib, n):
    # x stride 2 x 1350 elements = 21.6 KB; 2700 columns = 168 tiles of 16 + a ragged tile of 12
    with _env(CROFT_RING="1"):
        _check(croft_lib, _noise((n, 2, 1350), n), expect_ring=True)


@pytest.mark.parametrize("n", RING_LENGTHS)
def test_ring_y_pass_forced(croft_lib, n):
    # y stride 50 elements (400 B); 50 columns = 3 tiles + 2
    with _env(CROFT_RING="1"):
        _check(croft_lib, _noise((3, n, 50), 1000 + n), expect_ring=True)


def test_ring_off_and_odd_strides_use_the_plain_kernel(croft_lib):
    with _env(CROFT_RING="0"):
        _check(croft_lib, _noise((512, 2, 1350), 7), expect_ring=False)
    # an odd element stride (3375 columns) cannot be described to the tensor copy: plain kernel
    with _env(CROFT_RING="1"):
        _check(croft_lib, _noise((512, 3, 1125), 8), expect_ring=False)


def test_ring_many_tiles_per_cta_in_place(croft_lib):
    """More tiles than the ring's depth on every CTA (each CTA walks ~30 tiles through its three
    buffers, both consumer groups), in place (in == out) and out of place."""
    x = _noise((512, 270, 270), 9)  # 72900 columns = 4556 tiles of 16 + a ragged one of 4
    ref = oracle.forward(x)
    d = torch.from_numpy(x).cuda()
    with _env(CROFT_RING="1"), croft_lib.Plan(*x.shape) as p:
        assert "+ring" in p.describe()
        y = p.forward(d)
        z = d.clone()
        p.forward(z, z)
        torch.cuda.synchronize()
    t = tol(x.shape)
    assert oracle.rel_l2(y.cpu().numpy(), ref) <= t
    assert torch.equal(y.view(torch.float32), z.view(torch.float32))  # in place gives the same bits


def test_ring_deterministic(croft_lib):
    x = torch.from_numpy(_noise((480, 4, 1024), 11)).cuda()
    with _env(CROFT_RING="1"), croft_lib.Plan(*x.shape) as p:
        a = p.forward(x)
        b = p.forward(x)
        torch.cuda.synchronize()
    assert torch.equal(a.view(torch.float32), b.view(torch.float32))
