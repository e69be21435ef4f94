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

import synthetic_inputs as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

DIMS = [(48, 60, 64), (8, 6, 4), (1, 1, 1), (128, 2, 3), (30, 1, 25), (72, 80, 96), (64, 64, 64), (2, 3, 5)]


def _tol(shape):
    return 2e-6 * max(1.0, math.log2(int(np.prod(shape))))


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
            assert _rel(a, b) <= _tol(d), (call, d, "forward")
            assert _rel(c, e) <= _tol(d), (call, d, "backward")


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
        assert _rel(a, b) <= _tol(d)
    # beyond the static capacity: rejected before any device work
    too_many = [(2, 2, 2)] * (croft.CROFT_NOALLOC_MAX_GRIDS + 1)
    st = croft.croft_exec_batched_noalloc_status(too_many, [xs[0]] * len(too_many), [xs[0]] * len(too_many), -1)
    assert st == croft.CROFT_ERR_UNSUPPORTED_SIZE
    st = croft.croft_exec_batched_noalloc_status([(256, 4, 4)], [xs[0]], [xs[0]], -1)
    assert st == croft.CROFT_ERR_UNSUPPORTED_SIZE
    st = croft.croft_exec_batched_noalloc_status([(4, 4, 4)], [xs[0]], [xs[0]], 0)
    assert st == croft.CROFT_ERR_INVALID_ARG
