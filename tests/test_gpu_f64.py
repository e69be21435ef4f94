"""complex128 path (the paper's double complex), against the FP64 oracle (needs a GPU).

Tolerance: relative L2 <= 1e-14 * log2(N) (double-precision rounding of an
O(log N)-deep transform with correctly rounded float64 twiddles).
"""

import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def tol64(shape):
    return 1e-14 * max(1.0, math.log2(int(np.prod(shape))))


def _noise128(shape, seed):
    r = np.random.default_rng(seed)
    return r.uniform(-1, 1, shape) + 1j * r.uniform(-1, 1, shape)


@pytest.mark.parametrize("shape", [(128, 128, 128), (8, 1024, 4), (1024, 3, 2), (2, 5, 1024), (48, 60, 120),
                                   (16, 12, 15), (1, 1, 512), (64, 1, 1), (1, 1, 1)])
def test_f64_forward_backward_roundtrip(croft_lib, shape):
    x = _noise128(shape, sum(shape))
    d = torch.from_numpy(x).cuda()
    with croft_lib.Plan(*shape, dtype=croft_lib.CROFT_C2C_F64) as p:
        yf = p.forward(d)
        yb = p.backward(d)
        yr = p.backward(yf)
        torch.cuda.synchronize()
    ef = oracle.rel_l2(yf.cpu().numpy(), oracle.forward(x))
    eb = oracle.rel_l2(yb.cpu().numpy(), oracle.backward(x))
    er = oracle.rel_l2(yr.cpu().numpy(), x.size * x)
    print(f"f64 {shape}: fwd {ef:.2e} bwd {eb:.2e} roundtrip {er:.2e}")
    assert ef <= tol64(shape) and eb <= tol64(shape) and er <= tol64(shape)


def test_f64_rejections(croft_lib):
    for dims in [(7, 8, 8), (4, 9, 8), (2048, 2, 2)]:
        st, h = croft_lib.croft_plan_create_status(*dims, croft_lib.CROFT_C2C_F64)
        assert st == croft_lib.CROFT_ERR_UNSUPPORTED_SIZE and h is None
    st, h = croft_lib.croft_plan_create_status(4, 32, 32, croft_lib.CROFT_C2C_F64, croft_lib.CROFT_SCHEDULE_PLANE_FUSED)
    assert st == croft_lib.CROFT_ERR_UNSUPPORTED_SIZE
    x = torch.zeros((4, 4, 4), dtype=torch.complex64, device="cuda")
    with croft_lib.Plan(4, 4, 4, dtype=croft_lib.CROFT_C2C_F64) as p:
        with pytest.raises(ValueError):
            p.forward(x)  # complex64 tensor on a complex128 plan
