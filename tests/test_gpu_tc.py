"""Tensor-core variant: radix-16 stages as split-bf16 tcgen05 GEMMs (needs a GPU).

Bar: relative L2 error <= 3e-5 against the FP64 oracle, for every result.
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
    for name, dt in (("fp32", 0), ("tc_bf16x3", 1)):
        with croft_lib.Plan(512, 512, 512, dtype=dt) as p:
            yf = p.forward(d)
            yr = p.backward(yf)
            torch.cuda.synchronize()
            assert croft_lib.croft_plan_last_device_status(p.handle) == croft_lib.CROFT_OK
            ef = oracle.rel_l2(yf.cpu().numpy(), ref_f)
            er = oracle.rel_l2(yr.cpu().numpy(), n * x.astype(np.complex128))
        errs[name] = (ef, er)
    print(f"pme512 rel_l2: fp32 fwd {errs['fp32'][0]:.3e} roundtrip {errs['fp32'][1]:.3e}; "
          f"tc fwd {errs['tc_bf16x3'][0]:.3e} roundtrip {errs['tc_bf16x3'][1]:.3e}")
    assert errs["fp32"][0] <= 2e-6 * 27 and errs["fp32"][1] <= 2e-6 * 27
    assert errs["tc_bf16x3"][0] <= TC_TOL and errs["tc_bf16x3"][1] <= TC_TOL
