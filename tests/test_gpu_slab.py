"""Slab-decomposed transform with the real libcroft steps on one GPU (needs a GPU).

The G ranks of a slab job are emulated in one process, stage by stage: every rank's first
stage (croft_exec_axes on its x-slab, croft_transpose_blocks into its send buffer), then the
all-to-all as plain device copies (recv_r[s] = send_s[r]), then every rank's last stage.  No
kernel waits on another rank's kernel.  The assembled y-slabs are checked against the FP64
oracle, and the backward path must return each rank N times its own x-slab.
"""

import math

import numpy as np
import pytest

import oracle
import synthetic_inputs as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def tol(shape):
    return 2e-6 * math.log2(int(np.prod(shape)))


def _emulated_all_to_all(fft_list, sends):
    G = len(fft_list)
    recvs = []
    for r, f in enumerate(fft_list):
        recv = f.buffers(sends[r])[1]
        for s in range(G):
            recv[s * f.block:(s + 1) * f.block].copy_(sends[s][r * f.block:(r + 1) * f.block])
        recvs.append(recv)
    return recvs


@pytest.mark.parametrize("shape,world", [((64, 48, 40), 2), ((60, 48, 50), 4), ((512, 96, 64), 8),
                                         ((30, 27, 8), 3)])
def test_slab_fft_emulated_ranks(croft_lib, shape, world):
    from paper_2002_04896_gb300 import slab
    x = S.white_noise(shape, world)
    ref = oracle.forward(x)
    t = tol(shape)
    ffts = [slab.SlabFFT(shape, world=world, rank=r, exchange=lambda a, b: None) for r in range(world)]
    try:
        nxl = shape[0] // world
        xs = [torch.from_numpy(x[r * nxl:(r + 1) * nxl].copy()).cuda() for r in range(world)]
        sends = [f.forward_send(xs[r].clone()).clone() for r, f in enumerate(ffts)]
        recvs = _emulated_all_to_all(ffts, sends)
        ys = [f.forward_finish(recvs[r], torch.empty(f.shape_y, dtype=torch.complex64, device="cuda"))
              for r, f in enumerate(ffts)]
        torch.cuda.synchronize()
        full = np.concatenate([y.cpu().numpy() for y in ys], axis=1)
        e = oracle.rel_l2(full, ref)
        assert e <= t, (shape, world, e)
        # backward: y-slabs -> x-slabs, N times the input
        sends = [f.backward_send(ys[r].clone()).clone() for r, f in enumerate(ffts)]
        recvs = _emulated_all_to_all(ffts, sends)
        backs = [f.backward_finish(recvs[r], torch.empty(f.shape_x, dtype=torch.complex64, device="cuda"))
                 for r, f in enumerate(ffts)]
        torch.cuda.synchronize()
        for r in range(world):
            er = oracle.rel_l2(backs[r].cpu().numpy(), x.size * x[r * nxl:(r + 1) * nxl].astype(np.complex128))
            assert er <= t, (shape, world, r, er)
    finally:
        for f in ffts:
            f.close()


def test_exec_axes_subsets_match_the_oracle(croft_lib):
    x = S.white_noise((24, 20, 30), 5)
    d = torch.from_numpy(x).cuda()
    with croft_lib.Plan(*x.shape) as p:
        for mask in range(8):
            for direction in (-1, 1):
                out = torch.empty_like(d)
                croft_lib.croft_exec_axes(p.handle, d, out, mask, direction)
                torch.cuda.synchronize()
                ref = x.astype(np.complex128)
                for ax in (2, 1, 0):
                    if mask & (1 << ax):
                        ref = oracle.dft_along_axis(ref, ax, direction)
                assert oracle.rel_l2(out.cpu().numpy(), ref) <= tol(x.shape), (mask, direction)
        # in place, and the same bits as exec_forward for all three axes
        y = p.forward(d)
        z = d.clone()
        croft_lib.croft_exec_axes(p.handle, z, z, 7, -1)
        torch.cuda.synchronize()
        assert torch.equal(y.view(torch.float32), z.view(torch.float32))
    # schedules with more than one launch per axis refuse (256 x 128 x 128: two 16 MiB slabs)
    with croft_lib.Plan(256, 128, 128, schedule=croft_lib.CROFT_SCHEDULE_SLAB_L2) as p:
        assert croft_lib.croft_plan_num_launches(p.handle) > 3
        st = croft_lib.croft_exec_axes_status(p.handle, d, d, 7, -1)
        assert st == croft_lib.CROFT_ERR_INVALID_ARG


def test_transpose_blocks(croft_lib):
    a = torch.arange(5 * 7 * 3, dtype=torch.float32, device="cuda").reshape(5, 7, 3)
    b = torch.empty(7, 5, 3, dtype=torch.float32, device="cuda")
    croft_lib.croft_transpose_blocks(a, b, 5, 7, 3 * 4)
    c = torch.empty(5, 7, 3, dtype=torch.float32, device="cuda")
    croft_lib.croft_transpose_blocks(b, c, 7, 5, 3 * 4)  # the other copy direction (d1 < d0)
    torch.cuda.synchronize()
    assert torch.equal(b, a.transpose(0, 1))
    assert torch.equal(c, a)
    with pytest.raises(croft_lib.CroftError):
        croft_lib.croft_transpose_blocks(a, a, 5, 7, 12)  # overlap refused
