"""Host-streaming executor: host grids through the GPU with overlapped copies (needs a GPU)."""

import math

import numpy as np
import pytest

import oracle
import synthetic_inputs as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def tol(shape):
    return 2e-6 * math.log2(int(np.prod(shape)))


def _pinned(x):
    return torch.from_numpy(x).pin_memory()


@pytest.mark.parametrize("count", [1, 2, 7])
def test_pipeline_forward_and_roundtrip(croft_lib, count):
    shape = (24, 20, 30)
    xs = [S.white_noise(shape, 40 + i) for i in range(count)]
    hin = [_pinned(x) for x in xs]
    hout = [torch.empty(shape, dtype=torch.complex64).pin_memory() for _ in xs]
    hrt = [torch.empty(shape, dtype=torch.complex64).pin_memory() for _ in xs]
    with croft_lib.Plan(*shape) as p:
        croft_lib.croft_exec_host_pipeline(p.handle, hin, hout, croft_lib.CROFT_OP_FORWARD)
        croft_lib.croft_exec_host_pipeline(p.handle, hin, hrt, croft_lib.CROFT_OP_FORWARD | croft_lib.CROFT_OP_BACKWARD)
        torch.cuda.synchronize()
        assert croft_lib.croft_plan_workspace_bytes(p.handle) == 3 * int(np.prod(shape)) * 8
    for x, y, r in zip(xs, hout, hrt):
        assert oracle.rel_l2(y.numpy(), oracle.forward(x)) <= tol(shape)
        assert oracle.rel_l2(r.numpy(), x.size * x.astype(np.complex128)) <= tol(shape)


def test_pipeline_in_place_host_buffers_and_stream_order(croft_lib):
    shape = (16, 16, 16)
    xs = [S.white_noise(shape, 60 + i) for i in range(5)]
    bufs = [_pinned(x.copy()) for x in xs]
    s = torch.cuda.Stream()
    marker = torch.zeros(1, device="cuda")
    with croft_lib.Plan(*shape) as p:
        with torch.cuda.stream(s):
            marker.fill_(1.0)  # queued before the pipeline on the same stream
            croft_lib.croft_exec_host_pipeline(p.handle, bufs, bufs, croft_lib.CROFT_OP_BACKWARD, s)
            marker.fill_(2.0)  # after it
        s.synchronize()
    assert float(marker.item()) == 2.0
    for x, b in zip(xs, bufs):
        assert oracle.rel_l2(b.numpy(), oracle.backward(x)) <= tol(shape)


def test_pipeline_argument_errors_and_oom(croft_lib):
    shape = (8, 8, 8)
    x = _pinned(S.white_noise(shape, 1))
    with croft_lib.Plan(*shape) as p:
        assert croft_lib.croft_exec_host_pipeline_status(p.handle, [x], [x], 0) == croft_lib.CROFT_ERR_INVALID_ARG
        assert croft_lib.croft_exec_host_pipeline_status(p.handle, [x], [x], 4) == croft_lib.CROFT_ERR_INVALID_ARG
        assert croft_lib.croft_exec_host_pipeline_status(p.handle, [], [], 1) == croft_lib.CROFT_OK
        base = croft_lib.croft_debug_live_allocations()
        croft_lib.croft_debug_fail_allocation(2)  # the second slot buffer
        try:
            st = croft_lib.croft_exec_host_pipeline_status(p.handle, [x], [x], 1)
        finally:
            croft_lib.croft_debug_fail_allocation(0)
        assert st == croft_lib.CROFT_ERR_OOM
        assert croft_lib.croft_debug_live_allocations() == base
        assert croft_lib.croft_exec_host_pipeline_status(p.handle, [x], [x], 1) == croft_lib.CROFT_OK
        torch.cuda.synchronize()
    with croft_lib.BatchPlan([shape], mode=croft_lib.CROFT_BATCH_PER_GRID) as bp:
        assert croft_lib.croft_exec_host_pipeline_status(bp.handle, [x], [x], 1) == croft_lib.CROFT_ERR_INVALID_ARG
