"""PME reciprocal-space convolution B(G * F(x)) through croft_exec_convolve vs the FP64 oracle (needs a GPU).

Tolerance (complex64 plans): relative L2 error <= 4e-6 * log2(N): the bar of one
transform (2e-6 * log2 N) for each of the two transforms; the product with G
adds one rounding.  complex128 plans: 2e-14 * log2(N).  Tensor-core plans:
2 * 3e-5.  G is float32 (float64 for complex128) and the oracle receives the
same values upcast exactly.
"""

import math

import numpy as np
import pytest

import oracle
import synthetic_inputs as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def tol(shape, f64=False):
    n = int(np.prod(shape))
    return (2e-14 if f64 else 4e-6) * max(1.0, math.log2(n))


@pytest.fixture(scope="module")
def dev(croft_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _inputs(shape, seed, f64=False):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, shape) + 1j * rng.uniform(-1, 1, shape)
    g = rng.uniform(0.0, 1.0, shape)
    if f64:
        return x.astype(np.complex128), g.astype(np.float64)
    return x.astype(np.complex64), g.astype(np.float32)


def conv_gpu(croft, x_np, g_np, dtype=0, schedule=None, inplace=False):
    x = torch.from_numpy(np.ascontiguousarray(x_np)).cuda()
    g = torch.from_numpy(np.ascontiguousarray(g_np)).cuda()
    with croft.Plan(*x_np.shape, dtype=dtype, schedule=schedule) as p:
        out = x if inplace else torch.empty_like(x)
        p.convolve(x, g, out)
        torch.cuda.synchronize()
        return out.cpu().numpy(), p


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
def test_every_length_as_the_fused_axis(croft_lib, dev, n):
    """Every instantiated length as the x axis (the fused forward*G*backward pass), ragged column tile."""
    shape = (n, 2, 3)
    x, g = _inputs(shape, n)
    y, _ = conv_gpu(croft_lib, x, g)
    e = oracle.rel_l2(y, oracle.convolve(x, g))
    assert e <= tol(shape), (shape, e)


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 1, 8), (1, 16, 1), (32, 1, 1), (2, 2, 2), (6, 10, 15),
                                   (64, 48, 40), (5, 3, 1), (1, 60, 128), (32, 32, 32), (100, 36, 20),
                                   (48, 60, 64)])
def test_shapes(croft_lib, dev, shape):
    x, g = _inputs(shape, 7)
    y, _ = conv_gpu(croft_lib, x, g)
    e = oracle.rel_l2(y, oracle.convolve(x, g))
    assert e <= tol(shape), (shape, e)


def test_pme256_influence_function(croft_lib, dev):
    """The PME workload: the 256^3 charge grid and the smooth-PME influence function."""
    x = S.config_input("pme256")
    g = S.pme_influence(x.shape)
    y, _ = conv_gpu(croft_lib, x, g)
    ref = oracle.convolve(x, g)
    e = oracle.rel_l2(y, ref)
    assert e <= tol(x.shape), e
    # real input, real even G: the result is real and its mean is zero (G(0) = 0)
    scale = np.max(np.abs(ref.real))
    assert np.max(np.abs(y.imag)) <= 1e-4 * scale
    assert abs(np.sum(y.astype(np.complex128))) <= 1e-4 * np.sum(np.abs(ref))


def test_complex128(croft_lib, dev):
    for shape in [(64, 32, 16), (128, 128, 128), (5, 6, 4)]:
        x, g = _inputs(shape, 11, f64=True)
        y, _ = conv_gpu(croft_lib, x, g, dtype=croft_lib.CROFT_C2C_F64)
        e = oracle.rel_l2(y, oracle.convolve(x, g))
        assert e <= tol(shape, f64=True), (shape, e)


def test_unfused_paths(croft_lib, dev):
    """Plans whose last pass cannot take the fusion run F, multiply, B: same result."""
    c = croft_lib
    # tensor-core plan: the x pass is a tensor-core pass
    shape = (256, 64, 32)
    x, g = _inputs(shape, 12)
    y, p = conv_gpu(c, x, g, dtype=c.CROFT_C2C_F32_TC_BF16X3)
    e = oracle.rel_l2(y, oracle.convolve(x, g))
    assert e <= 2 * 3e-5, e
    # one yz-plane with the fused plane schedule: the only pass is the plane kernel
    shape = (1, 64, 64)
    x, g = _inputs(shape, 13)
    y, _ = conv_gpu(c, x, g, schedule=c.CROFT_SCHEDULE_PLANE_FUSED)
    assert oracle.rel_l2(y, oracle.convolve(x, g)) <= tol(shape)


def test_descriptions(croft_lib, dev):
    c = croft_lib
    with c.Plan(64, 64, 64) as p:
        assert "convolve: x fwd*G*bwd fused" in p.describe()
    with c.Plan(1, 64, 64, schedule=c.CROFT_SCHEDULE_PLANE_FUSED) as p:
        assert "convolve: forward, multiply, backward" in p.describe()


@pytest.mark.parametrize("schedule", ["three_pass", "plane_fused", "slab_l2"])
def test_schedules(croft_lib, dev, schedule):
    c = croft_lib
    sched = {"three_pass": c.CROFT_SCHEDULE_THREE_PASS, "plane_fused": c.CROFT_SCHEDULE_PLANE_FUSED,
             "slab_l2": c.CROFT_SCHEDULE_SLAB_L2}[schedule]
    shape = (48, 64, 64)
    x, g = _inputs(shape, 14)
    y, _ = conv_gpu(c, x, g, schedule=sched)
    assert oracle.rel_l2(y, oracle.convolve(x, g)) <= tol(shape)


def test_in_place_deterministic_inputs_untouched(croft_lib, dev):
    c = croft_lib
    shape = (64, 48, 40)
    x_np, g_np = _inputs(shape, 15)
    x = torch.from_numpy(x_np).cuda()
    g = torch.from_numpy(g_np).cuda()
    x0, g0 = x.clone(), g.clone()
    with c.Plan(*shape) as p:
        a = p.convolve(x, g)
        b = p.convolve(x, g)
        torch.cuda.synchronize()
        assert torch.equal(x, x0) and torch.equal(g, g0)
        assert torch.equal(a, b)
        y = x.clone()
        p.convolve(y, g, y)
        torch.cuda.synchronize()
        assert torch.equal(y, a)


def test_timing_groups(croft_lib, dev):
    c = croft_lib
    with c.Plan(64, 64, 64) as p:
        x = torch.randn(64, 64, 64, dtype=torch.complex64, device="cuda")
        g = torch.rand(64, 64, 64, dtype=torch.float32, device="cuda")
        c.croft_plan_set_timing(p.handle, True)
        p.convolve(x, g)
        t = c.croft_plan_pass_times(p.handle, 16)
        assert len(t) == 5 and all(v > 0 for v in t)
        p.forward(x)
        assert len(c.croft_plan_pass_times(p.handle, 16)) == 3


def test_argument_errors(croft_lib, dev):
    c = croft_lib
    shape = (16, 16, 16)
    x = torch.zeros(shape, dtype=torch.complex64, device="cuda")
    out = torch.empty_like(x)
    g = torch.ones(shape, dtype=torch.float32, device="cuda")
    with c.Plan(*shape) as p:
        h = p.handle
        st = c.croft_exec_convolve_status
        assert st(h, x, out, 0) == c.CROFT_ERR_INVALID_ARG                      # no G
        assert st(h, x, out, g.data_ptr() + 2) == c.CROFT_ERR_INVALID_ARG       # G misaligned
        assert st(h, x, out, out.data_ptr()) == c.CROFT_ERR_INVALID_ARG         # G overlaps out
        assert st(h, x.data_ptr() + 8, out, g) == c.CROFT_ERR_INVALID_ARG       # in misaligned
        assert st(h, x, out, g) == c.CROFT_OK
        with pytest.raises(ValueError):
            p.convolve(x, g.double())                                           # wrong G dtype
        with pytest.raises(ValueError):
            p.convolve(x, g[:8])                                                # wrong G size
    assert c.croft_exec_convolve_status(0, x, out, g) == c.CROFT_ERR_INVALID_ARG
    bp = c.croft_plan_create_batched([(16, 16, 16)])
    try:
        assert c.croft_exec_convolve_status(bp, x, out, g) == c.CROFT_ERR_INVALID_ARG
    finally:
        c.croft_plan_destroy(bp)
    torch.cuda.synchronize()


@pytest.mark.parametrize("name", ["pme480", "pme512"])
def test_full_size_properties(croft_lib, dev, name):
    """At the bench's full sizes (the oracle is too slow for the whole grid): the fused convolution
    equals forward, an elementwise multiply and backward run as separate calls, and with the real
    charge grid and the real even influence function the result is real with zero sum."""
    x_np = S.config_input(name)
    g_np = S.pme_influence(x_np.shape)
    x = torch.from_numpy(x_np).cuda()
    g = torch.from_numpy(g_np).cuda()
    with croft_lib.Plan(*x_np.shape) as p:
        c = p.convolve(x, g)
        y = p.forward(x)
        y.mul_(g)
        s = p.backward(y, y)
        torch.cuda.synchronize()
    n = x_np.size
    diff = float(torch.linalg.vector_norm((c - s).flatten()) / torch.linalg.vector_norm(s.flatten()))
    assert diff <= tol(x_np.shape), diff
    scale = float(c.real.abs().max())
    assert float(c.imag.abs().max()) <= 1e-4 * scale
    assert abs(complex(c.to(torch.complex128).sum())) <= 1e-4 * float(c.abs().to(torch.float64).sum())
    del x, g, c, y, s
    torch.cuda.empty_cache()
    assert n > 0


@pytest.mark.parametrize("n", [320, 512])
def test_fused_axis_on_the_radix16_first_split(croft_lib, dev, n):
    """Axes whose passes take the radix-16-first split by the rules (320; 512 at short strides)
    keep the fused convolution: it runs its own schedule on a twiddle table of its own."""
    shape = (n, 2, 3)
    with croft_lib.Plan(*shape) as p:
        d = p.describe()
    x_pass = d[d.index("x:"):].split(" | ")[0]
    assert ("radix=16x5x4" if n == 320 else "radix=16x8x4") in x_pass, d
    assert "fwd*G*bwd fused" in d, d
    x, g = _inputs(shape, 400 + n)
    y, _ = conv_gpu(croft_lib, x, g)
    e = oracle.rel_l2(y, oracle.convolve(x, g))
    assert e <= tol(shape), (shape, e)
