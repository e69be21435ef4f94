"""Failure paths exercised without any GPU fault (needs a GPU for plan creation).

Allocation failure is injected on the host (the k-th library allocation fails);
every plan constructor must return CROFT_ERR_OOM and release everything it had
allocated.  Device-side waits are covered by the batched timeout test.
"""

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _sweep(croft, create):
    base = croft.croft_debug_live_allocations()
    failures = 0
    try:
        for k in range(1, 64):
            croft.croft_debug_fail_allocation(k)
            st, h = create()
            if st == croft.CROFT_OK:
                croft.croft_debug_fail_allocation(0)
                croft.croft_plan_destroy(h)
                break
            assert st == croft.CROFT_ERR_OOM, (k, croft.croft_status_string(st))
            assert h is None
            assert croft.croft_debug_live_allocations() == base, f"leak after failing allocation {k}"
            failures += 1
        else:
            pytest.fail("plan creation never succeeded")
    finally:
        croft.croft_debug_fail_allocation(0)
    assert croft.croft_debug_live_allocations() == base
    return failures


def test_single_grid_plan_oom_at_every_allocation(croft_lib):
    assert _sweep(croft_lib, lambda: croft_lib.croft_plan_create_status(64, 48, 40)) == 3  # one table per axis


def test_tensor_core_plan_oom_at_every_allocation(croft_lib):
    n = _sweep(croft_lib, lambda: croft_lib.croft_plan_create_status(4, 256, 512, croft_lib.CROFT_C2C_F32_TC_BF16X3))
    assert n == 5  # DFT-16 operand, status word, three twiddle tables


def test_batched_plan_oom_at_every_allocation(croft_lib):
    dims = [(48, 60, 64), (8, 6, 4), (4, 144, 10)]
    n = _sweep(croft_lib, lambda: croft_lib.croft_plan_create_batched_status(dims, 0, croft_lib.CROFT_BATCH_ONE_LAUNCH))
    assert n >= 5


def test_grouped_batched_plan_oom_at_every_allocation(croft_lib):
    dims = [(48, 60, 64), (8, 6, 4), (4, 144, 10)]
    n = _sweep(croft_lib, lambda: croft_lib.croft_plan_create_batched_status(dims, 0, croft_lib.CROFT_BATCH_GROUPED))
    assert n >= 4  # pinned segment table, segments, CTA map, twiddle pool (+ the single-grid plan of the 144 grid)


def test_destroy_releases_everything(croft_lib):
    base = croft_lib.croft_debug_live_allocations()
    with croft_lib.Plan(32, 32, 32):
        assert croft_lib.croft_debug_live_allocations() > base
    with croft_lib.BatchPlan([(8, 8, 8), (16, 12, 10)], mode=croft_lib.CROFT_BATCH_PER_GRID):
        pass
    assert croft_lib.croft_debug_live_allocations() == base
