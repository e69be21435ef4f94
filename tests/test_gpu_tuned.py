"""CROFT_SCHEDULE_TUNED plans (needs a GPU): every candidate kernel the tuner may pick runs
correctly, and a measured plan matches the oracle.

The tuner times, per column pass of a 270..512-point axis, the 16- and 8-column tiles with the
near-equal and the radix-16-first power-of-two split, 16-column tiles with 16 threads per pencil,
and the tensor-copy ring kernel, then the schedules, and caches the choice.  The candidates are driven one by one through the cache
file (its last matching line wins): the first plan writes the key, the test appends a line per
forced configuration.
"""

import math
import os

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

LENGTHS = [270, 300, 360, 375, 405, 480, 486, 500, 512]


def tol(shape):
    return 2e-6 * math.log2(int(np.prod(shape)))


def _noise(shape, seed):
    rng = np.random.default_rng(seed)
    return (rng.uniform(-1, 1, shape) + 1j * rng.uniform(-1, 1, shape)).astype(np.complex64)


def _check(croft, x, desc_has=()):
    d = torch.from_numpy(x).cuda()
    with croft.Plan(*x.shape, schedule=croft.CROFT_SCHEDULE_TUNED) as p:
        desc = p.describe()
        yf = p.forward(d)
        yb = p.backward(d)
        torch.cuda.synchronize()
    for s in desc_has:
        assert s in desc, (s, desc)
    t = tol(x.shape)
    assert oracle.rel_l2(yf.cpu().numpy(), oracle.forward(x)) <= t
    assert oracle.rel_l2(yb.cpu().numpy(), oracle.backward(x)) <= t
    return desc


@pytest.fixture()
def cache(tmp_path):
    path = str(tmp_path / "tune.txt")
    old = os.environ.get("CROFT_TUNE_CACHE")
    os.environ["CROFT_TUNE_CACHE"] = path
    yield path
    if old is None:
        os.environ.pop("CROFT_TUNE_CACHE", None)
    else:
        os.environ["CROFT_TUNE_CACHE"] = old


@pytest.mark.parametrize("n", LENGTHS)
def test_every_tuner_candidate_matches_the_oracle(croft_lib, cache, n):
    # x pass across 21.6 KB strides (ragged last tile), y pass across 400 B (ragged)
    for shape, axis in (((n, 2, 1350), 0), ((3, n, 50), 1)):
        x = _noise(shape, n + axis)
        desc = _check(croft_lib, x, ("tuned: ",))  # measured: writes the cache line
        lines = open(cache).read().splitlines()
        key = [ln for ln in lines if ln.startswith(f"plan-v2:{shape[0]}x{shape[1]}x{shape[2]}:0:")][-1].split()[0]
        assert "three_pass=" in desc and "slab_l2=" in desc
        for kind, w, sv, th in ((0, 16, 0, 0), (0, 8, 0, 0), (0, 16, 1, 0), (0, 8, 1, 0), (0, 16, 0, 16),
                                (0, 16, 1, 16), (1, 16, 0, 0)) + (((2, 16, 0, 0),) if n % 2 == 0 else ()):
            ch = [[-1, 0, 0, 0] for _ in range(3)]
            ch[axis] = [kind, w, sv, th]
            with open(cache, "a") as f:
                f.write(f"{key} 1 " + " ".join(str(v) for c in ch for v in c) + " forced\n")
            desc = _check(croft_lib, x, ("tuned (cached)",))
            seg = [s for s in desc.split("|") if s.strip().startswith(("x:", "y:", "z:"))][2 - axis]
            if kind == 1:
                assert "+ring" in seg, seg
            elif kind == 2:
                assert "+pair" in seg, seg
            else:
                assert f" W={w} " in seg and f" T={th or 32} " in seg, seg
                if n == 512:
                    assert ("radix=16x16x2" in seg) == (sv == 1), seg


def test_tuned_config_grids(croft_lib, cache):
    """A measured tuned plan on a config-size grid gives the oracle's result."""
    x = _noise((480, 96, 64), 3)
    desc = _check(croft_lib, x, ("tuned: ",))
    assert "x:" in desc
