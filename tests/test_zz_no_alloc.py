"""The allocation-free batched entry point (collected last on purpose).

For callers that cannot allocate device memory (a framework pool owns it, or
the request path forbids cudaMalloc), croft_exec_batched_noalloc runs the
batched transform with its working memory in a static device array inside the
library.  It must give the same results as the plan-based batched entry point
(same kernel, same tiles), call after call, whatever ran before it.
"""

import math

import numpy as np
import pytest

import oracle
import synthetic_inputs as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

DIMS = [(48, 60, 64), (8, 6, 4), (1, 1, 1), (128, 2, 3), (30, 1, 25), (72, 80, 96), (64, 64, 64), (2, 3, 5)]


def _tol(shape):
    return 2e-6 * max(1.0, math.log2(int(np.prod(shape))))


def _same_bits(a, b):
    return torch.equal(a.view(torch.float32).view(torch.int32), b.view(torch.float32).view(torch.int32))


def _rel(a, b):
    a = a.cpu().numpy().astype(np.complex128)
    b = b.cpu().numpy().astype(np.complex128)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / den) if den > 0 else float(np.linalg.norm(a - b))


def test_noalloc_matches_plan_based_batched_exec_twice(croft_lib):
    from paper_2002_04896_gb300 import croft
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(5)
    xs = [torch.from_numpy((rng.uniform(-1, 1, d) + 1j * rng.uniform(-1, 1, d)).astype(np.complex64)).cuda()
          for d in DIMS]
    with croft.BatchPlan(DIMS, mode=croft.CROFT_BATCH_ONE_LAUNCH) as bp:
        ref_f = bp.forward(xs)
        ref_b = bp.backward(xs)
    torch.cuda.synchronize()
    for call in range(2):  # two calls in a row: the static array is reused
        outs_f = [torch.full_like(x, float("nan")) for x in xs]
        outs_b = [torch.full_like(x, float("nan")) for x in xs]
        croft.croft_exec_batched_noalloc(DIMS, xs, outs_f, -1)
        croft.croft_exec_batched_noalloc(DIMS, xs, outs_b, +1)
        torch.cuda.synchronize()
        for d, a, b, c, e in zip(DIMS, outs_f, ref_f, outs_b, ref_b):
            # same kernel, same tiles, same arithmetic: the same bits as the plan-based call
            assert _same_bits(a, b), (call, d, "forward", _rel(a, b))
            assert _same_bits(c, e), (call, d, "backward", _rel(c, e))
    # and against the FP64 oracle directly
    for d, x, a, c in zip(DIMS, xs, outs_f, outs_b):
        xh = x.cpu().numpy()
        assert oracle.rel_l2(a.cpu().numpy(), oracle.forward(xh)) <= _tol(d), (d, "forward vs oracle")
        assert oracle.rel_l2(c.cpu().numpy(), oracle.backward(xh)) <= _tol(d), (d, "backward vs oracle")


def test_noalloc_pme_grids_and_limits(croft_lib):
    from paper_2002_04896_gb300 import croft
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dims, grids = S.pme_batch(count=12, seed=3)
    xs = [torch.from_numpy(g).cuda() for g in grids]
    with croft.BatchPlan(dims, mode=croft.CROFT_BATCH_ONE_LAUNCH) as bp:
        ref = bp.forward(xs)
    outs = [torch.empty_like(x) for x in xs]
    croft.croft_exec_batched_noalloc(dims, xs, outs, -1)
    torch.cuda.synchronize()
    for d, a, b in zip(dims, outs, ref):
        assert _same_bits(a, b), (d, _rel(a, b))
    # beyond the static capacity: rejected by the library before any device work (raw addresses,
    # which the binding passes through unchecked, reach the C-side checks)
    p0 = xs[0].data_ptr()
    too_many = [(2, 2, 2)] * (croft.CROFT_NOALLOC_MAX_GRIDS + 1)
    st = croft.croft_exec_batched_noalloc_status(too_many, [p0] * len(too_many), [p0] * len(too_many), -1)
    assert st == croft.CROFT_ERR_UNSUPPORTED_SIZE
    st = croft.croft_exec_batched_noalloc_status([(256, 4, 4)], [p0], [p0], -1)
    assert st == croft.CROFT_ERR_UNSUPPORTED_SIZE
    st = croft.croft_exec_batched_noalloc_status([(4, 4, 4)], [p0], [p0], 0)
    assert st == croft.CROFT_ERR_INVALID_ARG


def test_noalloc_refuses_a_capturing_stream(croft_lib):
    """Its host tables live only for the call, so a copy recorded into a graph would read freed
    memory on replay: the call returns CROFT_ERR_INVALID_ARG while the stream captures, before
    any device work."""
    from paper_2002_04896_gb300 import croft
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dims = [(8, 6, 4)]
    x = torch.zeros(dims[0], dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    croft.croft_exec_batched_noalloc(dims, [x], [y], -1)  # first call on the device: set-up outside capture
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    statuses = []
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            statuses.append(croft.croft_exec_batched_noalloc_status(dims, [x], [y], -1, s))
            y.add_(0)  # one captured op, so the graph is not empty
    assert statuses == [croft.CROFT_ERR_INVALID_ARG]
