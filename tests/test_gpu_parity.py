"""CUDA path vs the FP64 oracle, through the C ABI (needs a GPU).

Tolerance (FP32 path): relative L2 error <= 2e-6 * log2(N), N = nx*ny*nz,
measured against the oracle run on the same complex64 input.
"""

import math

import numpy as np
import pytest

import oracle
import synthetic_inputs as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def tol(shape):
    n = int(np.prod(shape))
    return 2e-6 * max(1.0, math.log2(n))


@pytest.fixture(scope="module")
def dev(croft_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def run(croft, x_np, direction="forward", inplace=False, dtype=0, schedule=None):
    x = torch.from_numpy(np.ascontiguousarray(x_np)).cuda()
    with croft.Plan(*x_np.shape, dtype=dtype, schedule=schedule) as p:
        out = x if inplace else torch.empty_like(x)
        getattr(p, direction)(x, out)
        torch.cuda.synchronize()
        return out.cpu().numpy()


def _supported_sizes(limit):
    out = []
    for n in range(2, limit + 1):
        m = n
        for p in (2, 3, 5):
            while m % p == 0:
                m //= p
        if m == 1:
            out.append(n)
    return out


@pytest.mark.parametrize("n", _supported_sizes(4096))
def test_every_axis_length_on_every_axis(croft_lib, dev, n):
    """Each supported length as the z (contiguous), y and x (strided) axis, ragged batch sizes."""
    rng = np.random.default_rng(n)
    for shape in [(2, 3, n), (3, n, 5), (n, 2, 3)]:
        x = (rng.uniform(-1, 1, shape) + 1j * rng.uniform(-1, 1, shape)).astype(np.complex64)
        y = run(croft_lib, x)
        ref = oracle.forward(x)
        e = oracle.rel_l2(y, ref)
        assert e <= tol(shape), (shape, e)


LONG_PENCIL_SIZES = [n for n in _supported_sizes(512) if n > 256]  # 32 threads per pencil


def _pass_desc(desc, axis):
    part = desc[desc.index(axis + ":"):]
    return part.split(" | ")[0]


@pytest.mark.parametrize("n", LONG_PENCIL_SIZES)
def test_long_pencil_x_pass_over_wide_stride(croft_lib, dev, n):
    """A length of 32-thread pencils as the x axis with its elements 18 KB apart takes the
    16-column tile (the y pass of the length-n axis above, 40 bytes apart, the 8-column one);
    2250 columns leave a ragged last tile."""
    rng = np.random.default_rng(1000 + n)
    shape = (n, 45, 50)
    x = (rng.uniform(-1, 1, shape) + 1j * rng.uniform(-1, 1, shape)).astype(np.complex64)
    with croft_lib.Plan(*shape) as p:
        assert " W=16 " in _pass_desc(p.describe(), "x"), p.describe()
    y = run(croft_lib, x)
    e = oracle.rel_l2(y, oracle.forward(x))
    assert e <= tol(shape), (shape, e)


@pytest.mark.parametrize("n", [270, 320, 324, 360, 384, 405, 432, 480])
def test_24_thread_pencils_where_the_rule_takes_them(croft_lib, dev, n):
    """The column passes of these lengths run 24 threads per pencil where the rule says so
    (8-column y tiles of 192 threads, 16-column x tiles of 384), 32 elsewhere, against the oracle
    with ragged tiles."""
    rng = np.random.default_rng(2400 + n)
    for shape, axis, narrow in (((3, n, 5), "y", True), ((n, 45, 50), "x", False)):
        x = (rng.uniform(-1, 1, shape) + 1j * rng.uniform(-1, 1, shape)).astype(np.complex64)
        with croft_lib.Plan(*shape) as p:
            d = _pass_desc(p.describe(), axis)
        t24 = n in ((324, 360, 405) if narrow else (324, 360, 384, 405))
        want = (" T=24 W=8 block=192 " if narrow else " T=24 W=16 block=384 ") if t24 else " T=32 "
        assert want in d, (shape, d)
        y = run(croft_lib, x)
        e = oracle.rel_l2(y, oracle.forward(x))
        assert e <= tol(shape), (shape, e)


def test_16_thread_pencils_by_default_for_432_and_480_across_long_strides(croft_lib, dev):
    """432- and 480-point x passes across 256 KB or more take 16 threads per pencil (16-column,
    256-thread tiles); shorter strides keep 32 (their parity: the tuned-plan tests)."""
    for n in (432, 480):
        with croft_lib.Plan(n, 128, 256) as p:
            assert " T=16 W=16 block=256 " in _pass_desc(p.describe(), "x"), p.describe()
        with croft_lib.Plan(n, 64, 64) as p:
            assert " T=32 " in _pass_desc(p.describe(), "x"), p.describe()


def test_column_width_follows_the_stride(croft_lib, dev):
    """512^3: the y pass (4 KB stride) runs 8-column tiles, the x pass (2 MB stride) 16-column
    tiles split over a cluster pair of 256-thread CTAs; below 256 KB strides the plain
    16-column, 512-thread tile."""
    with croft_lib.Plan(512, 512, 512) as p:
        d = p.describe()
    assert " W=8 block=256 " in _pass_desc(d, "y"), d
    assert "+pair" in _pass_desc(d, "x") and " W=16 block=256 " in _pass_desc(d, "x"), d
    with croft_lib.Plan(512, 128, 128) as p:
        d = p.describe()
    assert "+pair" not in d and " W=16 block=512 " in _pass_desc(d, "x"), d


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 1, 8), (1, 16, 1), (32, 1, 1), (2, 2, 2), (6, 10, 15),
                                   (64, 48, 40), (5, 3, 1), (1, 60, 128)])
def test_small_and_degenerate_shapes(croft_lib, dev, shape):
    rng = np.random.default_rng(1)
    x = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)
    for direction, ref in (("forward", oracle.forward(x)), ("backward", oracle.backward(x))):
        y = run(croft_lib, x, direction)
        assert oracle.rel_l2(y, ref) <= tol(shape), (shape, direction)


def test_noise32_forward_backward_roundtrip(croft_lib, dev):
    """32^3 white noise (seed 0): forward, backward and backward(forward(x)) = N x."""
    x = S.white_noise((32, 32, 32), 0)
    t = tol(x.shape)
    yf = run(croft_lib, x, "forward")
    ref_f = oracle.forward(x)
    ef = oracle.rel_l2(yf, ref_f)
    ref_f32 = np.ascontiguousarray(ref_f, dtype=np.complex64)
    yb = run(croft_lib, ref_f32, "backward")
    eb = oracle.rel_l2(yb, oracle.backward(ref_f32))
    yr = run(croft_lib, yf, "backward")
    er = oracle.rel_l2(yr, x.size * x.astype(np.complex128))
    print(f"noise32 rel_l2 fwd {ef:.3e} bwd {eb:.3e} roundtrip {er:.3e} (tol {t:.2e})")
    assert ef <= t and eb <= t and er <= t


def test_in_place_equals_out_of_place_bitwise(croft_lib, dev):
    x = S.white_noise((48, 40, 30), 5)
    a = run(croft_lib, x, "forward", inplace=False)
    b = run(croft_lib, x, "forward", inplace=True)
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_deterministic_bitwise(croft_lib, dev):
    x = torch.from_numpy(S.white_noise((64, 60, 72), 6)).cuda()
    with croft_lib.Plan(64, 60, 72) as p:
        a = p.forward(x)
        b = p.forward(x)
        torch.cuda.synchronize()
        assert torch.equal(a.view(torch.int32), b.view(torch.int32))


def test_input_untouched_out_of_place(croft_lib, dev):
    xn = S.white_noise((16, 24, 20), 7)
    x = torch.from_numpy(xn).cuda()
    with croft_lib.Plan(16, 24, 20) as p:
        p.forward(x)
        p.backward(x)
        torch.cuda.synchronize()
    assert np.array_equal(x.cpu().numpy(), xn)


def test_side_stream_and_timing_hook(croft_lib, dev):
    x = torch.from_numpy(S.white_noise((64, 64, 64), 8)).cuda()
    out = torch.empty_like(x)
    s = torch.cuda.Stream()
    with croft_lib.Plan(64, 64, 64) as p:
        croft_lib.croft_plan_set_timing(p.handle, True)
        with torch.cuda.stream(s):
            croft_lib.croft_exec_forward(p.handle, x, out, s)
        times = croft_lib.croft_plan_pass_times(p.handle)
        s.synchronize()
        assert len(times) == croft_lib.croft_plan_num_launches(p.handle) in (2, 3)
        assert all(t > 0 for t in times)
    assert oracle.rel_l2(out.cpu().numpy(), oracle.forward(x.cpu().numpy())) <= tol((64, 64, 64))


def test_invalid_pointers_rejected(croft_lib, dev):
    x = torch.zeros(8 * 8 * 8 + 4, dtype=torch.complex64, device="cuda")
    with croft_lib.Plan(8, 8, 8) as p:
        h = p.handle
        base = x.data_ptr()
        # partial overlap
        assert croft_lib.croft_exec_forward_status(h, base, base + 16 * 8, 0) == croft_lib.CROFT_ERR_INVALID_ARG
        # misaligned (8-byte, not 16-byte)
        assert croft_lib.croft_exec_forward_status(h, base + 8, base + 8, 0) == croft_lib.CROFT_ERR_INVALID_ARG
        # null
        assert croft_lib.croft_exec_forward_status(h, 0, base, 0) == croft_lib.CROFT_ERR_INVALID_ARG
        # exact in-place is fine
        assert croft_lib.croft_exec_forward_status(h, base, base, 0) == croft_lib.CROFT_OK
    torch.cuda.synchronize()


def test_binding_rejects_non_contiguous_and_wrong_dtype(croft_lib, dev):
    x = torch.zeros((8, 6, 4), dtype=torch.complex64, device="cuda")
    with croft_lib.Plan(8, 6, 4) as p:
        with pytest.raises(ValueError):
            p.forward(x.permute(2, 1, 0).contiguous().permute(2, 1, 0))  # right shape, permuted strides
        with pytest.raises(ValueError):
            p.forward(x.to(torch.complex128))
        with pytest.raises(ValueError):
            p.forward(torch.zeros((8, 6, 5), dtype=torch.complex64, device="cuda"))


PLANE_SHAPES = [(32, 32), (64, 64), (128, 128), (256, 256), (384, 384)]


@pytest.mark.parametrize("ny,nz", PLANE_SHAPES)
def test_fused_plane_schedule_matches_oracle(croft_lib, dev, ny, nz):
    """The fused yz-plane pass (cluster / DSMEM all-to-all) + x pass, forward and backward."""
    shape = (3, ny, nz)
    x = S.white_noise(shape, ny + nz)
    d = torch.from_numpy(x).cuda()
    with croft_lib.Plan(*shape, schedule=croft_lib.CROFT_SCHEDULE_PLANE_FUSED) as p:
        desc = p.describe()
        assert "yz:plane" in desc, desc
        assert croft_lib.croft_plan_num_launches(p.handle) == 2
        yf = p.forward(d)
        yb = p.backward(d)
        torch.cuda.synchronize()
    ef = oracle.rel_l2(yf.cpu().numpy(), oracle.forward(x))
    eb = oracle.rel_l2(yb.cpu().numpy(), oracle.backward(x))
    print(f"fused {shape}: fwd {ef:.3e} bwd {eb:.3e}")
    assert ef <= tol(shape) and eb <= tol(shape)


@pytest.mark.parametrize("ny,nz", PLANE_SHAPES[:4])
def test_fused_plane_only_no_x_axis(croft_lib, dev, ny, nz):
    x = S.white_noise((1, ny, nz), 3)
    y = run(croft_lib, x, schedule=croft_lib.CROFT_SCHEDULE_PLANE_FUSED)
    assert oracle.rel_l2(y, oracle.forward(x)) <= tol(x.shape)


def test_schedules_agree(croft_lib, dev):
    x = torch.from_numpy(S.white_noise((16, 256, 256), 9)).cuda()
    with croft_lib.Plan(16, 256, 256, schedule=croft_lib.CROFT_SCHEDULE_PLANE_FUSED) as pa, \
            croft_lib.Plan(16, 256, 256, schedule=croft_lib.CROFT_SCHEDULE_THREE_PASS) as p3:
        assert "yz:plane" in pa.describe()
        assert croft_lib.croft_plan_num_launches(p3.handle) == 3
        a = pa.forward(x)
        b = p3.forward(x)
        torch.cuda.synchronize()
    assert oracle.rel_l2(a.cpu().numpy(), b.cpu().numpy()) <= tol((16, 256, 256))


def test_fused_schedule_unavailable_shape(croft_lib, dev):
    st, h = croft_lib.croft_plan_create_status(4, 48, 80, 0, croft_lib.CROFT_SCHEDULE_PLANE_FUSED)
    assert st == croft_lib.CROFT_ERR_UNSUPPORTED_SIZE and h is None
    st, h = croft_lib.croft_plan_create_status(4, 48, 80, 0, 9)
    assert st == croft_lib.CROFT_ERR_INVALID_ARG and h is None


@pytest.mark.parametrize("shape,slab_mb", [((48, 40, 30), "0.05"), ((9, 64, 64), "0.1"), ((16, 1, 32), "0.01"),
                                           ((12, 20, 1), "0.005"), ((10, 1, 1), "1"), ((64, 48, 40), "16")])
def test_slab_schedule_matches_oracle(croft_lib, dev, shape, slab_mb, monkeypatch):
    """Slab-by-slab z then y (L2-resident), then x: every slab boundary and degenerate axis."""
    monkeypatch.setenv("CROFT_SLAB_MB", slab_mb)
    x = S.white_noise(shape, 31)
    d = torch.from_numpy(x).cuda()
    with croft_lib.Plan(*shape, schedule=croft_lib.CROFT_SCHEDULE_SLAB_L2) as p:
        croft_lib.croft_plan_set_timing(p.handle, True)
        yf = p.forward(d)
        t = croft_lib.croft_plan_pass_times(p.handle)
        yb = p.backward(d)
        zb = yf.clone()
        p.backward(zb, zb)  # in place
        torch.cuda.synchronize()
    assert 1 <= len(t) <= 2 and all(v > 0 for v in t)
    assert oracle.rel_l2(yf.cpu().numpy(), oracle.forward(x)) <= tol(shape)
    assert oracle.rel_l2(yb.cpu().numpy(), oracle.backward(x)) <= tol(shape)
    assert oracle.rel_l2(zb.cpu().numpy(), x.size * x.astype(np.complex128)) <= tol(shape)


def test_exec_captured_in_a_cuda_graph(croft_lib, dev):
    """Forward, backward and a convolution captured into one CUDA graph (the passes' programmatic
    dependent launches become graph edges) replay to the same bits as direct calls."""
    shape = (64, 48, 40)
    rng = np.random.default_rng(5)
    x_np = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)
    x = torch.from_numpy(x_np).cuda()
    g = torch.rand(shape, dtype=torch.float32, device="cuda")
    with croft_lib.Plan(*shape) as p:
        y_ref = p.forward(x)
        z_ref = p.backward(y_ref)
        c_ref = p.convolve(x, g)
        y = torch.empty_like(x)
        z = torch.empty_like(x)
        c = torch.empty_like(x)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            p.forward(x, y)  # warm-up outside the capture
        torch.cuda.current_stream().wait_stream(s)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s):
            p.forward(x, y)
            p.backward(y, z)
            p.convolve(x, g, c)
        y.zero_()
        z.zero_()
        c.zero_()
        graph.replay()
        torch.cuda.synchronize()
    assert torch.equal(y.view(torch.int32), y_ref.view(torch.int32))
    assert torch.equal(z.view(torch.int32), z_ref.view(torch.int32))
    assert torch.equal(c.view(torch.int32), c_ref.view(torch.int32))
