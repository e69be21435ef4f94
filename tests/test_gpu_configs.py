"""Full-size workloads (PME-shaped grids) on the CUDA path vs the FP64 oracle (needs a GPU).

Each grid is checked element by element against the oracle (forward, backward
of the oracle's forward output, and the round trip against N x), plus
properties that hold at any size: Hermitian symmetry of the spectrum of a real
input and a vanishing DC term for a net-neutral charge grid.
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


def _check_grid(croft, x):
    shape = x.shape
    t = tol(shape)
    d = torch.from_numpy(x).cuda()
    with croft.Plan(*shape) as p:
        yf = p.forward(d)
        torch.cuda.synchronize()
        yf_h = yf.cpu().numpy()
        ref_f = oracle.forward(x)
        ef = oracle.rel_l2(yf_h, ref_f)
        ref_f32 = np.ascontiguousarray(ref_f, dtype=np.complex64)
        yb = p.backward(torch.from_numpy(ref_f32).cuda())
        torch.cuda.synchronize()
        eb = oracle.rel_l2(yb.cpu().numpy(), oracle.backward(ref_f32))
        del ref_f
        yr = p.backward(yf)
        torch.cuda.synchronize()
        er = oracle.rel_l2(yr.cpu().numpy(), float(x.size) * x.astype(np.complex128))
    # properties of the GPU spectrum itself: Hermitian (real input), DC = sum of the grid
    idx = [(-np.arange(n)) % n for n in shape]
    herm = np.linalg.norm(yf_h[np.ix_(*idx)] - np.conj(yf_h)) / np.linalg.norm(yf_h)
    dc_ref = complex(np.sum(x.astype(np.complex128)))
    scale = np.linalg.norm(yf_h) / math.sqrt(yf_h.size)
    print(f"{shape}: rel_l2 fwd {ef:.3e} bwd {eb:.3e} roundtrip {er:.3e} hermitian {herm:.2e} (tol {t:.2e})")
    assert ef <= t and eb <= t and er <= t
    assert herm <= t
    assert abs(yf_h[0, 0, 0] - dc_ref) <= 1e-5 * scale * math.sqrt(x.size)


def test_pme256(croft_lib):
    _check_grid(croft_lib, S.config_input("pme256"))


def test_pme480(croft_lib):
    _check_grid(croft_lib, S.config_input("pme480"))


def test_pme384x360x320(croft_lib):
    _check_grid(croft_lib, S.config_input("pme384x360x320"))


def test_pme512_fp32(croft_lib):
    _check_grid(croft_lib, S.config_input("pme512"))
