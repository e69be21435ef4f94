"""Tensor-core variants: a radix-16 stage as split-operand tcgen05 GEMMs (needs a GPU).

CROFT_C2C_F32_TC_BF16X3 (bf16 hi + lo) and CROFT_C2C_F32_TC_FP16X3 (fp16 hi + lo, each
butterfly scaled by a power of two).  Bar: relative L2 error <= 3e-5 against the FP64
oracle, for every result.  Every axis length with a factor 16 up to 1024 runs on the
tensor cores, on each axis; longer ones are refused at plan creation.
"""

import numpy as np
import pytest

import oracle
import synthetic_inputs as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TC_TOL = 3e-5


def _run(croft, x, dtype, direction="forward"):
    d = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    with croft.Plan(*x.shape, dtype=dtype) as p:
        desc = p.describe()
        y = getattr(p, direction)(d)
        torch.cuda.synchronize()
        st = croft.croft_plan_last_device_status(p.handle)
    return y.cpu().numpy(), desc, st


@pytest.mark.parametrize("shape", [(4, 6, 256), (3, 512, 5), (512, 3, 2), (16, 256, 256), (2, 48, 512), (512, 1, 1)])
def test_tc_axes_match_oracle(croft_lib, shape):
    x = S.white_noise(shape, sum(shape))
    for direction, ref in (("forward", oracle.forward(x)), ("backward", oracle.backward(x))):
        y, desc, st = _run(croft_lib, x, croft_lib.CROFT_C2C_F32_TC_BF16X3, direction)
        assert st == croft_lib.CROFT_OK
        assert "+tc" in desc, desc
        e = oracle.rel_l2(y, ref)
        print(f"tc {shape} {direction}: rel_l2 {e:.3e}")
        assert e <= TC_TOL, (shape, direction, e)


TC_LENGTHS = [16, 32, 48, 64, 80, 96, 128, 144, 160, 192, 240, 256, 288, 320, 384, 400, 432, 480, 512, 576,
              640, 720, 768, 800, 864, 960, 1024]
PRECS = [("bf16x3", 1), ("fp16x3", 3)]


@pytest.mark.parametrize("n", TC_LENGTHS)
def test_tc_every_length_on_every_axis(croft_lib, n):
    """Each tensor-core length as z (row), y and x (column), ragged batches, both precisions."""
    for shape, axis in (((3, 2, n), 2), ((2, n, 5), 1), ((n, 3, 2), 0)):
        x = S.white_noise(shape, n + axis)
        ref_f, ref_b = oracle.forward(x), oracle.backward(x)
        for name, dt in PRECS:
            d = torch.from_numpy(x).cuda()
            with croft_lib.Plan(*shape, dtype=dt) as p:
                assert croft_lib.croft_plan_tc_axes(p.handle) == 1 << axis, (shape, p.describe())
                yf = p.forward(d)
                yb = p.backward(d)
                torch.cuda.synchronize()
                assert croft_lib.croft_plan_last_device_status(p.handle) == croft_lib.CROFT_OK
            ef = oracle.rel_l2(yf.cpu().numpy(), ref_f)
            eb = oracle.rel_l2(yb.cpu().numpy(), ref_b)
            assert ef <= TC_TOL and eb <= TC_TOL, (shape, name, ef, eb)


def test_tc_refuses_radix16_axes_it_cannot_run(croft_lib):
    """No silent FP32 stand-in: a factor-16 axis longer than 1024 makes a tensor-core plan fail."""
    for _, dt in PRECS:
        for shape in ((2, 2, 2048), (4096, 2, 3), (2, 1600, 3)):
            st, h = croft_lib.croft_plan_create_status(*shape, dt)
            assert st == croft_lib.CROFT_ERR_UNSUPPORTED_SIZE, (shape, dt)
            assert h is None
        # the same shapes plan fine on the FP32 path
        st, h = croft_lib.croft_plan_create_status(2, 2, 2048, croft_lib.CROFT_C2C_F32)
        assert st == croft_lib.CROFT_OK
        croft_lib.croft_plan_destroy(h)


def test_tc_axes_mask(croft_lib):
    for _, dt in PRECS:
        with croft_lib.Plan(512, 60, 256, dtype=dt) as p:  # 60 has no factor 16
            assert croft_lib.croft_plan_tc_axes(p.handle) == 0b101
        with croft_lib.Plan(12, 10, 9, dtype=dt) as p:
            assert croft_lib.croft_plan_tc_axes(p.handle) == 0
    with croft_lib.Plan(512, 512, 512) as p:
        assert croft_lib.croft_plan_tc_axes(p.handle) == 0


def test_fp16x3_scaling_covers_a_wide_dynamic_range(croft_lib):
    """fp16 alone spans 2^-24 .. 65504; per-butterfly power-of-two scaling keeps the split exact
    for inputs far outside that range (and for pencils of very different magnitudes)."""
    rng = np.random.default_rng(3)
    shape = (4, 8, 256)
    a = (rng.uniform(-1, 1, shape) + 1j * rng.uniform(-1, 1, shape))
    a *= np.exp2(rng.integers(-60, 60, size=(4, 8, 1)))  # pencils from 2^-60 to 2^60
    x = a.astype(np.complex64)
    d = torch.from_numpy(x).cuda()
    with croft_lib.Plan(*shape, dtype=croft_lib.CROFT_C2C_F32_TC_FP16X3) as p:
        y = p.forward(d)
        torch.cuda.synchronize()
    yh = y.cpu().numpy()
    ref = oracle.forward(x)
    # per pencil (the z transform of each (x, y) pencil is independent up to the x and y sums, so
    # compare the whole result and the smallest-magnitude pencils' share of it)
    assert np.all(np.isfinite(yh))
    assert oracle.rel_l2(yh, ref) <= TC_TOL


def test_tc_plan_without_radix16_axes_is_fp32(croft_lib):
    x = S.white_noise((12, 10, 9), 1)
    y, desc, st = _run(croft_lib, x, croft_lib.CROFT_C2C_F32_TC_BF16X3)
    assert "+tc" not in desc
    assert oracle.rel_l2(y, oracle.forward(x)) <= 2e-6 * np.log2(x.size)


def test_tc_deterministic(croft_lib):
    x = torch.from_numpy(S.white_noise((8, 256, 512), 2)).cuda()
    with croft_lib.Plan(8, 256, 512, dtype=croft_lib.CROFT_C2C_F32_TC_BF16X3) as p:
        a = p.forward(x)
        b = p.forward(x)
        torch.cuda.synchronize()
    assert torch.equal(a.view(torch.int32), b.view(torch.int32))


def test_pme512_tc_vs_fp32_error_per_result(croft_lib):
    """512^3 PME grid, 8M charges: the tensor-core and FP32 paths on the same input, error of each result."""
    x = S.config_input("pme512")
    n = x.size
    ref_f = oracle.forward(x)
    d = torch.from_numpy(x).cuda()
    errs = {}
    for name, dt in (("fp32", 0), ("tc_bf16x3", 1), ("tc_fp16x3", 3)):
        with croft_lib.Plan(512, 512, 512, dtype=dt) as p:
            yf = p.forward(d)
            yr = p.backward(yf)
            torch.cuda.synchronize()
            assert croft_lib.croft_plan_last_device_status(p.handle) == croft_lib.CROFT_OK
            ef = oracle.rel_l2(yf.cpu().numpy(), ref_f)
            er = oracle.rel_l2(yr.cpu().numpy(), n * x.astype(np.complex128))
        errs[name] = (ef, er)
    print("pme512 rel_l2: " + "; ".join(f"{k} fwd {v[0]:.3e} roundtrip {v[1]:.3e}" for k, v in errs.items()))
    assert errs["fp32"][0] <= 2e-6 * 27 and errs["fp32"][1] <= 2e-6 * 27
    for k in ("tc_bf16x3", "tc_fp16x3"):
        assert errs[k][0] <= TC_TOL and errs[k][1] <= TC_TOL, (k, errs[k])
    # the fp16 split carries ~22 bits: within a few times the FP32 path's error
    assert errs["tc_fp16x3"][0] <= 8 * errs["fp32"][0], errs
