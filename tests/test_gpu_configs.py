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


def local_error_checks(y, ref, t):
    """Checks that a localised mistake (one wrong tile, a wrong high-frequency block) cannot hide
    under the whole-array rel L2 of a steeply decaying PME spectrum:

    * per element: max |Y - Y_ref| / max |Y_ref| <= t;
    * no outliers: max |Y - Y_ref| <= 40 x the rms error.  Rounding spreads error over every
      output (the largest of N roughly Gaussian errors is ~6 rms at N = 1e8), while one wrong
      tile of T elements puts its whole error there (max ~ sqrt(N / T) rms);
    * the outer half of the spectrum (normalised |k| = sqrt(sum_a (m_a / (K_a / 2))^2) >= 1,
      m_a the signed frequency): its error norm stays within its share of the error budget,
      ||Y - Y_ref||_band <= 2 t ||Y_ref|| sqrt(N_band / N).
    Returns (max_rel, outlier_ratio, band_rel)."""
    nx, ny, nz = ref.shape
    err2 = np.zeros(ref.shape, dtype=np.float64)
    for x0 in range(0, nx, 32):
        d = y[x0:x0 + 32].astype(np.complex128) - ref[x0:x0 + 32]
        err2[x0:x0 + 32] = d.real ** 2 + d.imag ** 2
    ref_abs_max = float(np.sqrt(max(float((r.real ** 2 + r.imag ** 2).max()) for r in ref)))
    ref_norm = float(np.sqrt(sum(float((r.real ** 2 + r.imag ** 2).sum()) for r in ref)))
    max_err = float(np.sqrt(err2.max()))
    rms_err = float(np.sqrt(err2.mean()))

    def f2(k):
        m = np.arange(k, dtype=np.float64)
        m = np.where(m <= k // 2, m, m - k)
        return (m / (k / 2.0)) ** 2

    band = (f2(nx)[:, None, None] + f2(ny)[None, :, None] + f2(nz)[None, None, :]) >= 1.0
    band_err = float(np.sqrt(err2[band].sum()))
    band_bar = 2.0 * t * ref_norm * math.sqrt(band.sum() / band.size)
    max_rel = max_err / ref_abs_max
    outlier = max_err / rms_err if rms_err > 0 else 0.0
    assert max_rel <= t, ("per-element error", max_rel, t)
    assert outlier <= 40.0, ("localised error", outlier)
    assert band_err <= band_bar, ("high-|k| band error", band_err, band_bar)
    return max_rel, outlier, band_err / band_bar


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
        loc = local_error_checks(yf_h, ref_f, t)
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
    print(f"{shape}: rel_l2 fwd {ef:.3e} bwd {eb:.3e} roundtrip {er:.3e} hermitian {herm:.2e} (tol {t:.2e}); "
          f"max-elem {loc[0]:.2e}, max/rms {loc[1]:.1f}, band {loc[2]:.2f} of its bar")
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
