"""Batched form: many uneven grids per launch, through the C ABI (needs a GPU)."""

import math

import numpy as np
import pytest

import oracle
import synthetic_inputs as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def tol(shape):
    return 2e-6 * max(1.0, math.log2(int(np.prod(shape))))


MIXED = [(48, 60, 64), (8, 6, 4), (1, 1, 1), (1, 48, 1), (128, 2, 3), (4, 144, 10), (30, 1, 25), (2, 3, 5),
         (72, 80, 96)]


@pytest.fixture(scope="module")
def mixed_inputs():
    rng = np.random.default_rng(11)
    return [(rng.uniform(-1, 1, d) + 1j * rng.uniform(-1, 1, d)).astype(np.complex64) for d in MIXED]


@pytest.mark.parametrize("mode", [1, 2, 3, 4])
def test_mixed_batch_every_mode_matches_oracle(croft_lib, mixed_inputs, mode):
    ins = [torch.from_numpy(x).cuda() for x in mixed_inputs]
    with croft_lib.BatchPlan(MIXED, mode=mode) as bp:
        yf = bp.forward(ins)
        yb = bp.backward(ins)
        torch.cuda.synchronize()
        assert croft_lib.croft_plan_last_device_status(bp.handle) == croft_lib.CROFT_OK
    for x, a, b in zip(mixed_inputs, yf, yb):
        ef = oracle.rel_l2(a.cpu().numpy(), oracle.forward(x))
        eb = oracle.rel_l2(b.cpu().numpy(), oracle.backward(x))
        assert ef <= tol(x.shape) and eb <= tol(x.shape), (x.shape, mode, ef, eb)


def test_mixed_batch_in_place_and_deterministic(croft_lib, mixed_inputs):
    with croft_lib.BatchPlan(MIXED, mode=croft_lib.CROFT_BATCH_ONE_LAUNCH) as bp:
        ins = [torch.from_numpy(x).cuda() for x in mixed_inputs]
        a = bp.forward(ins)
        b = bp.forward(ins)
        c = [t.clone() for t in ins]
        bp.forward(c, c)
        torch.cuda.synchronize()
    for u, v, w in zip(a, b, c):
        assert torch.equal(u.view(torch.int32), v.view(torch.int32))
        assert torch.equal(u.view(torch.int32), w.view(torch.int32))


@pytest.fixture(scope="module")
def pme_batch():
    dims, grids = S.pme_batch(count=96, seed=3)
    return dims, grids


def test_pme_batch_96_one_launch_vs_oracle_and_per_grid(croft_lib, pme_batch):
    """The 96-grid PME batch: every grid against the oracle and against its own single-grid plan."""
    dims, grids = pme_batch
    ins = [torch.from_numpy(g).cuda() for g in grids]
    with croft_lib.BatchPlan(dims, mode=croft_lib.CROFT_BATCH_ONE_LAUNCH) as bp, \
            croft_lib.BatchPlan(dims, mode=croft_lib.CROFT_BATCH_PER_GRID) as pg:
        a = bp.forward(ins)
        b = pg.forward(ins)
        r = bp.backward(a)
        torch.cuda.synchronize()
        assert croft_lib.croft_plan_last_device_status(bp.handle) == croft_lib.CROFT_OK
        assert croft_lib.croft_plan_num_launches(bp.handle) == 1
    worst = 0.0
    for g, x in enumerate(grids):
        t = tol(x.shape)
        ya = a[g].cpu().numpy()
        ef = oracle.rel_l2(ya, oracle.forward(x))
        ep = oracle.rel_l2(ya, b[g].cpu().numpy())
        er = oracle.rel_l2(r[g].cpu().numpy(), x.size * x.astype(np.complex128))
        worst = max(worst, ef / t, er / t)
        assert ef <= t and ep <= t and er <= t, (g, dims[g], ef, ep, er)
    print(f"pme batch of 96: worst error / tolerance = {worst:.3e}")


def test_pme_batch_96_grouped_matches_single_grid_plans_bitwise(croft_lib, pme_batch):
    """The grouped schedule runs the single-grid pass kernels' arithmetic: the same bits as per-grid plans."""
    dims, grids = pme_batch
    ins = [torch.from_numpy(g).cuda() for g in grids]
    with croft_lib.BatchPlan(dims, mode=croft_lib.CROFT_BATCH_GROUPED) as gp, \
            croft_lib.BatchPlan(dims, mode=croft_lib.CROFT_BATCH_PER_GRID) as pg:
        a = gp.forward(ins)
        b = pg.forward(ins)
        ra = gp.backward(a)
        rb = pg.backward(b)
        c = [t.clone() for t in ins]
        gp.forward(c, c)  # in place
        torch.cuda.synchronize()
        n_len = len({d[a] for d in dims for a in range(3)})
        assert 3 <= croft_lib.croft_plan_num_launches(gp.handle) <= 3 * n_len
        assert "grouped" in gp.describe()
    for g in range(len(grids)):
        assert torch.equal(a[g].view(torch.int32), b[g].view(torch.int32)), (g, dims[g])
        assert torch.equal(ra[g].view(torch.int32), rb[g].view(torch.int32)), (g, dims[g])
        assert torch.equal(a[g].view(torch.int32), c[g].view(torch.int32)), (g, dims[g])
    # and against the oracle on a sample of the grids
    for g in range(0, len(grids), 12):
        x = grids[g]
        assert oracle.rel_l2(a[g].cpu().numpy(), oracle.forward(x)) <= tol(x.shape)


def test_autotune_chooses_and_caches(croft_lib, pme_batch, tmp_path, monkeypatch):
    dims, _ = pme_batch
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("CROFT_TUNE_CACHE", str(cache))
    monkeypatch.delenv("CROFT_TUNE", raising=False)
    sub = dims[:24]
    with croft_lib.BatchPlan(sub) as bp:
        desc = bp.describe()
    assert cache.exists()
    line = cache.read_text().strip().splitlines()[-1]
    assert line.startswith("batch-v2:24:") and "one_launch_us=" in line and "grouped_us=" in line
    mode = int(line.split()[1])
    assert mode in (1, 2, 3, 4)
    assert ["one_launch", "per_pass", "per_grid", "grouped"][mode - 1] in desc
    print(desc)
    # a second plan reads the cache (no new line appended)
    with croft_lib.BatchPlan(sub):
        pass
    assert len(cache.read_text().strip().splitlines()) == 1


def test_bounded_wait_times_out_with_status_and_context_survives(croft_lib, mixed_inputs):
    """A dependency count nothing reaches: the waits give up after the limit, status TIMEOUT, no hang."""
    ins = [torch.from_numpy(x).cuda() for x in mixed_inputs]
    with croft_lib.BatchPlan(MIXED, mode=croft_lib.CROFT_BATCH_ONE_LAUNCH) as bp:
        croft_lib.croft_plan_set_wait_limit(bp.handle, 2_000_000)  # ~1 ms of SM clock
        croft_lib.croft_plan_set_test_unsatisfiable_wait(bp.handle, True)
        bp.forward(ins)
        torch.cuda.synchronize()
        assert croft_lib.croft_plan_last_device_status(bp.handle) == croft_lib.CROFT_ERR_TIMEOUT
        croft_lib.croft_plan_set_test_unsatisfiable_wait(bp.handle, False)
        y = bp.forward(ins)
        torch.cuda.synchronize()
        assert croft_lib.croft_plan_last_device_status(bp.handle) == croft_lib.CROFT_OK
    for x, a in zip(mixed_inputs, y):
        assert oracle.rel_l2(a.cpu().numpy(), oracle.forward(x)) <= tol(x.shape)


def test_batched_argument_errors(croft_lib):
    st, h = croft_lib.croft_plan_create_batched_status([(4, 4, 4)], 0, 7)
    assert st == croft_lib.CROFT_ERR_INVALID_ARG and h is None
    st, h = croft_lib.croft_plan_create_batched_status([(4, 7, 4)], 0, 1)
    assert st == croft_lib.CROFT_ERR_UNSUPPORTED_SIZE
    st, h = croft_lib.croft_plan_create_batched_status([], 0, 1)
    assert st == croft_lib.CROFT_ERR_INVALID_ARG
    x = torch.zeros((4, 4, 4), dtype=torch.complex64, device="cuda")
    with croft_lib.BatchPlan([(4, 4, 4)], mode=1) as bp:
        base = x.data_ptr()
        assert croft_lib.croft_exec_batched_forward_status(bp.handle, [base + 8], [base + 8]) == \
            croft_lib.CROFT_ERR_INVALID_ARG
        assert croft_lib.croft_exec_batched_forward_status(bp.handle, [base], [base + 16]) == \
            croft_lib.CROFT_ERR_INVALID_ARG
        # a single-grid exec on a batched plan is an argument error
        assert croft_lib.croft_exec_forward_status(bp.handle, base, base) == croft_lib.CROFT_ERR_INVALID_ARG
