"""Cluster-pair column kernel (croft_pair_kernel.cuh) vs the FP64 oracle (needs a GPU).

Two CTAs of a 2-CTA cluster share a 16-column tile of an even 270..512-point axis: each
transforms the even or the odd rows at half length, and a radix-2 step across the pair
(one operand read through distributed shared memory) combines them.  By default it runs the
512-point passes across strides of 256 KB or more (the 512^3 x pass); CROFT_PAIR=1 selects it
for every column pass it can serve; tuned plans may pick it.  Every length as x and y,
ragged tiles, forward and backward, in place, determinism.
"""

import math
import os

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

PAIR_LENGTHS = [270, 288, 300, 320, 324, 360, 384, 400, 432, 450, 480, 486, 500, 512]


def tol(shape):
    return 2e-6 * math.log2(int(np.prod(shape)))


@pytest.fixture()
def pair_on():
    old = os.environ.get("CROFT_PAIR")
    os.environ["CROFT_PAIR"] = "1"
    yield
    if old is None:
        os.environ.pop("CROFT_PAIR", None)
    else:
        os.environ["CROFT_PAIR"] = old


def _noise(shape, seed):
    rng = np.random.default_rng(seed)
    return (rng.uniform(-1, 1, shape) + 1j * rng.uniform(-1, 1, shape)).astype(np.complex64)


def _check(croft, x, n_pair_passes):
    d = torch.from_numpy(x).cuda()
    with croft.Plan(*x.shape) as p:
        desc = p.describe()
        yf = p.forward(d)
        yb = p.backward(d)
        torch.cuda.synchronize()
    assert desc.count("+pair") == n_pair_passes, desc
    t = tol(x.shape)
    ef = oracle.rel_l2(yf.cpu().numpy(), oracle.forward(x))
    eb = oracle.rel_l2(yb.cpu().numpy(), oracle.backward(x))
    assert ef <= t and eb <= t, (x.shape, ef, eb, t)


@pytest.mark.parametrize("n", PAIR_LENGTHS)
def test_pair_x_and_y(croft_lib, pair_on, n):
    # x pass across 21.6 KB strides, 2700 columns (ragged last tile of 12); y pass across 400 B, 50 columns
    _check(croft_lib, _noise((n, 2, 1350), n), 1)
    _check(croft_lib, _noise((3, n, 50), 1000 + n), 1)


def test_pair_x_and_y_together_in_place(croft_lib, pair_on):
    x = _noise((480, 300, 40), 5)
    ref = oracle.forward(x)
    d = torch.from_numpy(x).cuda()
    with croft_lib.Plan(*x.shape) as p:
        assert p.describe().count("+pair") == 2
        y = p.forward(d)
        z = d.clone()
        p.forward(z, z)
        w = p.forward(d)
        torch.cuda.synchronize()
    assert oracle.rel_l2(y.cpu().numpy(), ref) <= tol(x.shape)
    assert torch.equal(y.view(torch.float32), z.view(torch.float32))  # in place: same bits
    assert torch.equal(y.view(torch.float32), w.view(torch.float32))  # deterministic


def test_pair_not_for_odd_lengths(croft_lib, pair_on):
    _check(croft_lib, _noise((375, 2, 1350), 3), 0)


def test_pair_default_for_512_point_long_strides(croft_lib):
    """Without CROFT_PAIR: the x pass of a 512 x 256 x 256 grid (512 KB strides) is a pair pass,
    its y pass (2 KB) and a 512 x 128 x 128 grid's x pass (128 KB) are not."""
    x = _noise((512, 256, 256), 11)
    ref = oracle.forward(x)
    d = torch.from_numpy(x).cuda()
    with croft_lib.Plan(*x.shape) as p:
        desc = p.describe()
        y = p.forward(d)
        torch.cuda.synchronize()
    assert desc.count("+pair") == 1 and "x:col+pair" in desc, desc
    assert oracle.rel_l2(y.cpu().numpy(), ref) <= tol(x.shape)
    with croft_lib.Plan(512, 128, 128) as p:
        assert "+pair" not in p.describe()


def test_pair_default_for_486_and_500(croft_lib):
    """Without CROFT_PAIR: 486-point passes pair at every stride (y across 40 bytes, x across
    18 KB), 500-point ones only across 256 KB or more."""
    with croft_lib.Plan(486, 45, 50) as p:
        d = p.describe()
    assert "x:col+pair" in d, d
    x = _noise((3, 486, 50), 21)
    _check(croft_lib, x, 1)
    with croft_lib.Plan(500, 256, 256) as p:
        assert "x:col+pair" in p.describe()
    with croft_lib.Plan(500, 45, 50) as p:
        assert "+pair" not in p.describe()
    with croft_lib.Plan(3, 500, 50) as p:
        assert "+pair" not in p.describe()
