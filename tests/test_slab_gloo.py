"""Slab decomposition of one transform over several processes (paper Sec. 2.2.1), on the CPU
with gloo process groups: the partition, the pack / unpack and the all-to-all schedule of
``paper_2002_04896_gb300.slab`` with the local 1D transforms done by the FP64 oracle
(``oracle.dft_along_axis``) instead of libcroft.  The assembled y-slabs must equal the
oracle's full forward transform, and backward must return every process N times its own
x-slab.
"""

import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleOps:
    """The local steps of the slab transform on the CPU: FP64 oracle axis DFTs, numpy transposes."""

    def __init__(self, shape_x, shape_y):
        self.shapes = {"x": shape_x, "y": shape_y}

    def axes(self, which, inp, out, axes, direction, stream=None):
        import oracle
        shape = self.shapes[which]
        a = inp.reshape(shape).numpy().astype(np.complex128)
        for ax in (2, 1, 0):
            if axes & (1 << ax):
                a = oracle.dft_along_axis(a, ax, direction)
        out.reshape(shape).copy_(torch.from_numpy(a.astype(np.complex64)))

    def transpose(self, inp, out, d0, d1, inner, stream=None):
        src = inp.reshape(-1)[: d0 * d1 * inner].reshape(d0, d1, inner)
        out.reshape(-1)[: d0 * d1 * inner].copy_(src.transpose(0, 1).reshape(-1))

    def empty(self, like, n):
        return torch.empty(n, dtype=like.dtype)


def _grid(shape):
    rng = np.random.default_rng(sum(shape))
    return (rng.uniform(-1, 1, shape) + 1j * rng.uniform(-1, 1, shape)).astype(np.complex64)


def _worker(rank, world, port, shape, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    from paper_2002_04896_gb300 import slab
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        x = _grid(shape)
        sx, sy = slab.slab_shapes(shape, world)
        fft = slab.SlabFFT(shape, ops=OracleOps(sx, sy))
        assert (fft.world, fft.rank) == (world, rank)
        xs = torch.from_numpy(x[rank * sx[0]:(rank + 1) * sx[0]].copy())
        ys = torch.empty(sy, dtype=torch.complex64)
        fft.forward(xs.clone(), ys)
        back = torch.empty(sx, dtype=torch.complex64)
        fft.backward(ys.clone(), back)
        out[rank] = (ys.numpy().copy(), back.numpy().copy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("shape,world", [((8, 6, 10), 2), ((6, 9, 4), 3), ((4, 8, 3), 4)])
def test_slab_transform_gloo(shape, world):
    import oracle
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), shape, out), nprocs=world, join=True)
        res = dict(out)
    x = _grid(shape)
    ref = oracle.forward(x)
    nyl = shape[1] // world
    full = np.concatenate([res[r][0] for r in range(world)], axis=1)  # y-slabs side by side
    assert full.shape == ref.shape
    assert oracle.rel_l2(full, ref) <= 1e-6
    for r in range(world):
        np.testing.assert_allclose(res[r][0], ref[:, r * nyl:(r + 1) * nyl], rtol=0, atol=1e-5 * np.abs(ref).max())
        nxl = shape[0] // world
        assert oracle.rel_l2(res[r][1], x.size * x[r * nxl:(r + 1) * nxl].astype(np.complex128)) <= 1e-6


def test_slab_shapes_refuse_uneven_splits():
    from paper_2002_04896_gb300 import slab
    assert slab.slab_shapes((8, 6, 10), 2) == ((4, 6, 10), (8, 3, 10))
    with pytest.raises(ValueError):
        slab.slab_shapes((8, 6, 10), 4)  # 6 % 4 != 0
    with pytest.raises(ValueError):
        slab.slab_shapes((9, 6, 10), 2)


def test_partition_grids_balances_the_pme_batch():
    import math
    from paper_2002_04896_gb300 import slab
    import synthetic_inputs as S  # noqa: F401
    rng = np.random.default_rng(3)
    dims = [tuple(int(v) for v in r) for r in rng.choice(np.asarray(S.BATCH_AXIS_CHOICES), size=(96, 3))]
    cost = [math.prod(d) * math.log2(math.prod(d)) for d in dims]
    for world in (1, 2, 4, 8):
        parts = slab.partition_grids(dims, world)
        assert len(parts) == world
        assert sorted(i for p in parts for i in p) == list(range(96))  # every grid exactly once
        loads = [sum(cost[i] for i in p) for p in parts]
        # LPT's guarantee: the largest load exceeds the mean by at most the largest single cost
        assert max(loads) <= sum(cost) / world + max(cost)
        if world > 1:
            assert max(loads) / min(loads) < 1.1  # 96 grids over <= 8 processes balance well
    assert slab.partition_grids([(2, 2, 2)], 3) == [[0], [], []]
