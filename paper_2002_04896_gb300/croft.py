"""Thin ctypes binding of libcroft.so (C ABI in include/croft.h).

Function names match the C entry points.  Arguments are marshalled only:
device pointers come from torch CUDA tensors (``tensor.data_ptr()``), streams
from ``torch.cuda.Stream.cuda_stream``; every step of the transform runs in the
library's CUDA kernels.  There is no fallback: if the shared library is missing
or fails to load, importing this module raises.
"""

from __future__ import annotations

import ctypes
import os

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libcroft.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"libcroft.so not built ({_LIB_PATH}); run paper_2002_04896_gb300.build.build()")
_lib = ctypes.CDLL(_LIB_PATH)

CROFT_C2C_F32 = 0
CROFT_C2C_F32_TC_BF16X3 = 1
CROFT_C2C_F64 = 2
CROFT_C2C_F32_TC_FP16X3 = 3

CROFT_SCHEDULE_AUTO = 0
CROFT_SCHEDULE_THREE_PASS = 1
CROFT_SCHEDULE_PLANE_FUSED = 2
CROFT_SCHEDULE_SLAB_L2 = 3
CROFT_SCHEDULE_TUNED = 4

CROFT_NOALLOC_MAX_GRIDS = 256
CROFT_NOALLOC_MAX_ITEMS = 65536

CROFT_OP_FORWARD = 1
CROFT_OP_BACKWARD = 2

CROFT_BATCH_AUTO = 0
CROFT_BATCH_ONE_LAUNCH = 1
CROFT_BATCH_PER_PASS = 2
CROFT_BATCH_PER_GRID = 3
CROFT_BATCH_GROUPED = 4

CROFT_OK = 0
CROFT_ERR_INVALID_ARG = 1
CROFT_ERR_UNSUPPORTED_SIZE = 2
CROFT_ERR_OOM = 3
CROFT_ERR_CUDA = 4
CROFT_ERR_TIMEOUT = 5

_P = ctypes.c_void_p
_I = ctypes.c_int


def _sig(name, res, args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = args
    return f


_status_string = _sig("croft_status_string", ctypes.c_char_p, [_I])
_plan_create = _sig("croft_plan_create", _I, [ctypes.POINTER(_P), _I, _I, _I, _I])
_plan_create_schedule = _sig("croft_plan_create_schedule", _I, [ctypes.POINTER(_P), _I, _I, _I, _I, _I])
_exec_forward = _sig("croft_exec_forward", _I, [_P, _P, _P, _P])
_exec_backward = _sig("croft_exec_backward", _I, [_P, _P, _P, _P])
_workspace_bytes = _sig("croft_plan_workspace_bytes", ctypes.c_size_t, [_P])
_num_launches = _sig("croft_plan_num_launches", _I, [_P])
_describe = _sig("croft_plan_describe", _I, [_P, ctypes.c_char_p, _I])
_set_timing = _sig("croft_plan_set_timing", _I, [_P, _I])
_pass_times = _sig("croft_plan_pass_times", _I, [_P, ctypes.POINTER(ctypes.c_float), _I])
_last_device_status = _sig("croft_plan_last_device_status", _I, [_P])
_plan_destroy = _sig("croft_plan_destroy", _I, [_P])
_factorize = _sig("croft_factorize", _I, [_I, ctypes.POINTER(_I), _I])
_plan_create_batched = _sig("croft_plan_create_batched", _I, [ctypes.POINTER(_P), _I, ctypes.POINTER(_I), _I])
_plan_create_batched_mode = _sig("croft_plan_create_batched_mode", _I,
                                 [ctypes.POINTER(_P), _I, ctypes.POINTER(_I), _I, _I])
_exec_batched_forward = _sig("croft_exec_batched_forward", _I, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), _P])
_exec_batched_backward = _sig("croft_exec_batched_backward", _I, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), _P])
_set_wait_limit = _sig("croft_plan_set_wait_limit", _I, [_P, ctypes.c_longlong])
_set_test_unsat = _sig("croft_plan_set_test_unsatisfiable_wait", _I, [_P, _I])
_exec_host_pipeline = _sig("croft_exec_host_pipeline", _I,
                           [_P, _I, ctypes.POINTER(_P), ctypes.POINTER(_P), _I, _P])
_debug_fail_allocation = _sig("croft_debug_fail_allocation", None, [_I])
_debug_live_allocations = _sig("croft_debug_live_allocations", ctypes.c_long, [])
_exec_batched_noalloc = _sig("croft_exec_batched_noalloc", _I,
                             [_I, ctypes.POINTER(_I), ctypes.POINTER(_P), ctypes.POINTER(_P), _I, _P])
_exec_convolve = _sig("croft_exec_convolve", _I, [_P, _P, _P, _P, _P])
_tc_axes = _sig("croft_plan_tc_axes", _I, [_P])
_exec_axes = _sig("croft_exec_axes", _I, [_P, _P, _P, _I, _I, _P])
_transpose_blocks = _sig("croft_transpose_blocks", _I,
                         [_P, _P, ctypes.c_longlong, ctypes.c_longlong, ctypes.c_longlong, _P])
_twiddle_table = _sig("croft_twiddle_table", _I, [_I, ctypes.POINTER(_I), _I, ctypes.POINTER(ctypes.c_float)])

LIBRARY_PATH = _LIB_PATH
EXPORTED = [
    "croft_status_string", "croft_plan_create", "croft_plan_create_schedule", "croft_exec_forward", "croft_exec_backward",
    "croft_plan_workspace_bytes", "croft_plan_num_launches", "croft_plan_describe", "croft_plan_set_timing",
    "croft_plan_pass_times", "croft_plan_last_device_status", "croft_plan_destroy", "croft_factorize",
    "croft_twiddle_table", "croft_plan_create_batched", "croft_plan_create_batched_mode",
    "croft_exec_batched_forward", "croft_exec_batched_backward", "croft_plan_set_wait_limit",
    "croft_plan_set_test_unsatisfiable_wait", "croft_exec_batched_noalloc", "croft_debug_fail_allocation",
    "croft_debug_live_allocations", "croft_exec_host_pipeline", "croft_exec_convolve", "croft_plan_tc_axes",
    "croft_exec_axes", "croft_transpose_blocks",
]


class CroftError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {croft_status_string(status)}")
        self.status = status


def _check(status: int, what: str) -> None:
    if status != CROFT_OK:
        raise CroftError(status, what)


def croft_status_string(status: int) -> str:
    return _status_string(int(status)).decode()


def _stream_ptr(stream) -> int:
    if stream is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:  # noqa: BLE001
            return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _check_layout(x, numel=None, complex128=None) -> None:
    """dtype, contiguity and element count of a tensor argument (no device check)."""
    import torch
    if not isinstance(x, torch.Tensor):
        raise TypeError("expected a torch CUDA tensor or an integer device address")
    allowed = ((torch.complex64, torch.complex128) if complex128 is None
               else ((torch.complex128,) if complex128 else (torch.complex64,)))
    if x.dtype not in allowed:
        raise ValueError(f"croft: expected {' or '.join(map(str, allowed))}, got {x.dtype}")
    if not x.is_contiguous():
        raise ValueError("croft: tensors must be C-contiguous in (nx, ny, nz) order")
    if numel is not None and x.numel() != numel:
        raise ValueError(f"croft: tensor has {x.numel()} elements, plan expects {numel}")


def _ptr(x, numel=None, complex128=None) -> int:
    """Device address of a raw pointer (int) or of a C-contiguous complex CUDA tensor.

    complex128: True / False require that dtype; None (the raw entry points) accepts
    complex64 and complex128 and leaves matching the plan's dtype to the caller.
    """
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    import torch
    _check_layout(x, numel, complex128)
    if not x.is_cuda:
        raise ValueError("croft: tensors must live on a CUDA device")
    return int(x.data_ptr())


# ---------------------------------------------------------------------------
# raw entry points (status codes returned, not raised)
# ---------------------------------------------------------------------------

def croft_plan_create_status(nx: int, ny: int, nz: int, dtype: int = CROFT_C2C_F32, schedule=None):
    h = _P()
    if schedule is None:
        st = _plan_create(ctypes.byref(h), int(nx), int(ny), int(nz), int(dtype))
    else:
        st = _plan_create_schedule(ctypes.byref(h), int(nx), int(ny), int(nz), int(dtype), int(schedule))
    return st, h.value


def croft_exec_forward_status(plan: int, inp, out, stream=None) -> int:
    return _exec_forward(plan, _ptr(inp), _ptr(out), _stream_ptr(stream))


def croft_exec_backward_status(plan: int, inp, out, stream=None) -> int:
    return _exec_backward(plan, _ptr(inp), _ptr(out), _stream_ptr(stream))


def _real_ptr(g, numel=None, f64=None) -> int:
    """Device address of a raw pointer (int) or of a C-contiguous real CUDA tensor (the influence function)."""
    if g is None:
        return 0
    if isinstance(g, int):
        return g
    import torch
    if not isinstance(g, torch.Tensor) or not g.is_cuda:
        raise ValueError("croft: the influence function must be a CUDA tensor")
    allowed = ((torch.float32, torch.float64) if f64 is None else ((torch.float64,) if f64 else (torch.float32,)))
    if g.dtype not in allowed:
        raise ValueError(f"croft: expected {' or '.join(map(str, allowed))} for the influence function, got {g.dtype}")
    if not g.is_contiguous():
        raise ValueError("croft: the influence function must be C-contiguous in (kx, ky, kz) order")
    if numel is not None and g.numel() != numel:
        raise ValueError(f"croft: influence function has {g.numel()} elements, plan expects {numel}")
    return int(g.data_ptr())


def croft_exec_convolve_status(plan: int, inp, out, g, stream=None) -> int:
    return _exec_convolve(plan, _ptr(inp), _ptr(out), _real_ptr(g), _stream_ptr(stream))


# ---------------------------------------------------------------------------
# raising wrappers with the C names
# ---------------------------------------------------------------------------

def croft_plan_create(nx: int, ny: int, nz: int, dtype: int = CROFT_C2C_F32) -> int:
    st, h = croft_plan_create_status(nx, ny, nz, dtype)
    _check(st, f"croft_plan_create({nx},{ny},{nz},{dtype})")
    return h


def croft_plan_create_schedule(nx: int, ny: int, nz: int, dtype: int, schedule: int) -> int:
    st, h = croft_plan_create_status(nx, ny, nz, dtype, schedule)
    _check(st, f"croft_plan_create_schedule({nx},{ny},{nz},{dtype},{schedule})")
    return h


def croft_exec_forward(plan: int, inp, out, stream=None) -> None:
    _check(croft_exec_forward_status(plan, inp, out, stream), "croft_exec_forward")


def croft_exec_backward(plan: int, inp, out, stream=None) -> None:
    _check(croft_exec_backward_status(plan, inp, out, stream), "croft_exec_backward")


def croft_exec_convolve(plan: int, inp, out, g, stream=None) -> None:
    """out = B(G * F(in)): the PME reciprocal-space convolution (see include/croft.h)."""
    _check(croft_exec_convolve_status(plan, inp, out, g, stream), "croft_exec_convolve")


def croft_exec_axes_status(plan: int, inp, out, axes: int, direction: int, stream=None) -> int:
    return _exec_axes(plan, _ptr(inp), _ptr(out), int(axes), int(direction), _stream_ptr(stream))


def croft_exec_axes(plan: int, inp, out, axes: int, direction: int, stream=None) -> None:
    """The 1D transforms of the axes in the bit mask `axes` (bit a: axis a; 0 = x): direction -1
    forward (Eq. 1), +1 backward (Eq. 2)."""
    _check(croft_exec_axes_status(plan, inp, out, axes, direction, stream), "croft_exec_axes")


def croft_transpose_blocks(inp, out, d0: int, d1: int, block_bytes: int, stream=None) -> None:
    """out[j][i] = in[i][j] over d0 x d1 blocks of block_bytes (device tensors or addresses)."""
    def addr(t):
        if isinstance(t, int):
            return t
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError("croft: contiguous CUDA tensors expected")
        if t.numel() * t.element_size() < d0 * d1 * block_bytes:
            raise ValueError("croft: tensor smaller than d0 * d1 * block_bytes")
        return int(t.data_ptr())
    _check(_transpose_blocks(addr(inp), addr(out), int(d0), int(d1), int(block_bytes), _stream_ptr(stream)),
           "croft_transpose_blocks")


def croft_plan_tc_axes(plan: int) -> int:
    """Bit a set when axis a (0 = x, 1 = y, 2 = z) runs a radix-16 stage on the tensor cores."""
    return int(_tc_axes(plan))


def croft_plan_workspace_bytes(plan: int) -> int:
    return int(_workspace_bytes(plan))


def croft_plan_num_launches(plan: int) -> int:
    return int(_num_launches(plan))


def croft_plan_describe(plan: int) -> str:
    need = _describe(plan, None, 0)
    buf = ctypes.create_string_buffer(max(1, need + 1))
    _describe(plan, buf, len(buf))
    return buf.value.decode()


def croft_plan_set_timing(plan: int, enable: bool) -> None:
    _check(_set_timing(plan, 1 if enable else 0), "croft_plan_set_timing")


def croft_plan_pass_times(plan: int, cap: int = 8):
    arr = (ctypes.c_float * cap)()
    n = _pass_times(plan, arr, cap)
    if n < 0:
        raise CroftError(CROFT_ERR_CUDA, "croft_plan_pass_times")
    return [float(arr[i]) for i in range(min(n, cap))]


def croft_plan_last_device_status(plan: int) -> int:
    return int(_last_device_status(plan))


def croft_plan_destroy(plan) -> None:
    _check(_plan_destroy(plan), "croft_plan_destroy")


def croft_factorize(n: int):
    arr = (_I * 16)()
    k = _factorize(int(n), arr, 16)
    return None if k < 0 else [int(arr[i]) for i in range(k)]


def croft_twiddle_table(n: int, radices):
    import numpy as np
    rad = (_I * max(1, len(radices)))(*radices)
    out = np.zeros(2 * max(1, n - 1), dtype=np.float32)
    k = _twiddle_table(int(n), rad, len(radices), out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    if k < 0:
        return None
    return out[: 2 * k].view(np.complex64)


# ---------------------------------------------------------------------------
# batched form
# ---------------------------------------------------------------------------

def croft_plan_create_batched_status(dims, dtype: int = CROFT_C2C_F32, mode=None):
    flat = [int(v) for d in dims for v in d]
    arr = (_I * max(1, len(flat)))(*flat)
    h = _P()
    if mode is None:
        st = _plan_create_batched(ctypes.byref(h), len(dims), arr, int(dtype))
    else:
        st = _plan_create_batched_mode(ctypes.byref(h), len(dims), arr, int(dtype), int(mode))
    return st, h.value


def croft_plan_create_batched(dims, dtype: int = CROFT_C2C_F32, mode=None) -> int:
    st, h = croft_plan_create_batched_status(dims, dtype, mode)
    _check(st, f"croft_plan_create_batched({len(dims)} grids, mode={mode})")
    return h


def _ptr_array(xs, sizes=None):
    vals = [_ptr(x, None if sizes is None else sizes[i]) for i, x in enumerate(xs)]
    return (_P * max(1, len(vals)))(*vals)


def croft_exec_batched_forward_status(plan: int, ins, outs, stream=None) -> int:
    return _exec_batched_forward(plan, _ptr_array(ins), _ptr_array(outs), _stream_ptr(stream))


def croft_exec_batched_backward_status(plan: int, ins, outs, stream=None) -> int:
    return _exec_batched_backward(plan, _ptr_array(ins), _ptr_array(outs), _stream_ptr(stream))


def croft_exec_batched_forward(plan: int, ins, outs, stream=None) -> None:
    _check(croft_exec_batched_forward_status(plan, ins, outs, stream), "croft_exec_batched_forward")


def croft_exec_batched_backward(plan: int, ins, outs, stream=None) -> None:
    _check(croft_exec_batched_backward_status(plan, ins, outs, stream), "croft_exec_batched_backward")


def croft_plan_set_wait_limit(plan: int, cycles: int) -> None:
    _check(_set_wait_limit(plan, int(cycles)), "croft_plan_set_wait_limit")


def croft_plan_set_test_unsatisfiable_wait(plan: int, enable: bool) -> None:
    _check(_set_test_unsat(plan, 1 if enable else 0), "croft_plan_set_test_unsatisfiable_wait")


def croft_exec_batched_noalloc_status(dims, ins, outs, direction: int, stream=None) -> int:
    """The allocation-free batched entry point: direction -1 forward (Eq. 1), +1 backward (Eq. 2).

    The C side trusts `dims` for every size, so the lists are checked here first: one
    complex64 tensor (or raw address) in and out per grid, each with the grid's element count.
    """
    dims = [tuple(int(v) for v in d) for d in dims]
    if any(len(d) != 3 for d in dims):
        raise ValueError("croft: each grid needs three axis lengths")
    if len(ins) != len(dims) or len(outs) != len(dims):
        raise ValueError(f"croft: {len(dims)} grids need as many inputs and outputs "
                         f"(got {len(ins)} and {len(outs)})")
    sizes = [d[0] * d[1] * d[2] for d in dims]
    for i, x in enumerate(list(ins) + list(outs)):
        if not isinstance(x, int):
            _check_layout(x, sizes[i % len(dims)], complex128=False)
    pin = [_ptr(x, sizes[i], complex128=False) for i, x in enumerate(ins)]
    pout = [_ptr(x, sizes[i], complex128=False) for i, x in enumerate(outs)]
    flat = [v for d in dims for v in d]
    arr = (_I * max(1, len(flat)))(*flat)
    return _exec_batched_noalloc(len(dims), arr, (_P * max(1, len(pin)))(*pin), (_P * max(1, len(pout)))(*pout),
                                 int(direction), _stream_ptr(stream))


def croft_exec_batched_noalloc(dims, ins, outs, direction: int, stream=None) -> None:
    _check(croft_exec_batched_noalloc_status(dims, ins, outs, direction, stream), "croft_exec_batched_noalloc")


def _host_ptr(x) -> int:
    if isinstance(x, int):
        return x
    import torch
    if isinstance(x, torch.Tensor):
        if x.is_cuda or x.dtype not in (torch.complex64, torch.complex128) or not x.is_contiguous():
            raise ValueError("host pipeline: expected contiguous complex CPU tensors (pinned for overlap)")
        return int(x.data_ptr())
    return int(x.ctypes.data)  # numpy array


def croft_exec_host_pipeline_status(plan: int, host_in, host_out, ops: int, stream=None) -> int:
    """Stream host grids through the GPU: upload, transform(s) in place, download, overlapped across grids."""
    n = len(host_in)
    a = (_P * max(1, n))(*[_host_ptr(x) for x in host_in])
    b = (_P * max(1, n))(*[_host_ptr(x) for x in host_out])
    return _exec_host_pipeline(plan, n, a, b, int(ops), _stream_ptr(stream))


def croft_exec_host_pipeline(plan: int, host_in, host_out, ops: int, stream=None) -> None:
    _check(croft_exec_host_pipeline_status(plan, host_in, host_out, ops, stream), "croft_exec_host_pipeline")


def croft_debug_fail_allocation(k: int) -> None:
    _debug_fail_allocation(int(k))


def croft_debug_live_allocations() -> int:
    return int(_debug_live_allocations())


class BatchPlan:
    """RAII helper around a batched plan: lists of torch tensors in and out."""

    def __init__(self, dims, dtype: int = CROFT_C2C_F32, mode=None):
        self.dims = [tuple(int(v) for v in d) for d in dims]
        self.handle = None
        self.handle = croft_plan_create_batched(self.dims, dtype, mode)

    def _check_lists(self, ins, outs):
        if len(ins) != len(self.dims) or len(outs) != len(self.dims):
            raise ValueError("one input and one output per grid")
        for d, a, b in zip(self.dims, ins, outs):
            n = d[0] * d[1] * d[2]
            _ptr(a, n)
            _ptr(b, n)

    def forward(self, ins, outs=None, stream=None):
        import torch
        if outs is None:
            outs = [torch.empty(d, dtype=torch.complex64, device=x.device) for d, x in zip(self.dims, ins)]
        self._check_lists(ins, outs)
        croft_exec_batched_forward(self.handle, ins, outs, stream)
        return outs

    def backward(self, ins, outs=None, stream=None):
        import torch
        if outs is None:
            outs = [torch.empty(d, dtype=torch.complex64, device=x.device) for d, x in zip(self.dims, ins)]
        self._check_lists(ins, outs)
        croft_exec_batched_backward(self.handle, ins, outs, stream)
        return outs

    def describe(self) -> str:
        return croft_plan_describe(self.handle)

    def close(self):
        if self.handle:
            croft_plan_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


class Plan:
    """RAII helper around a croft plan (torch tensors in, torch tensors out)."""

    def __init__(self, nx: int, ny: int, nz: int, dtype: int = CROFT_C2C_F32, schedule=None):
        self.shape = (int(nx), int(ny), int(nz))
        self.dtype = dtype
        self.handle = None
        if schedule is None:
            self.handle = croft_plan_create(nx, ny, nz, dtype)
        else:
            self.handle = croft_plan_create_schedule(nx, ny, nz, dtype, schedule)

    def _out(self, inp, out):
        f64 = self.dtype == CROFT_C2C_F64
        if out is None:
            import torch
            out = torch.empty(self.shape, dtype=torch.complex128 if f64 else torch.complex64, device=inp.device)
        n = self.shape[0] * self.shape[1] * self.shape[2]
        return _ptr(inp, n, f64), _ptr(out, n, f64), out

    def forward(self, inp, out=None, stream=None):
        pi, po, out = self._out(inp, out)
        croft_exec_forward(self.handle, pi, po, stream)
        return out

    def backward(self, inp, out=None, stream=None):
        pi, po, out = self._out(inp, out)
        croft_exec_backward(self.handle, pi, po, stream)
        return out

    def convolve(self, inp, g, out=None, stream=None):
        """B(G * F(inp)) with a real influence function g of the grid's shape (float32, or float64 for complex128)."""
        pi, po, out = self._out(inp, out)
        n = self.shape[0] * self.shape[1] * self.shape[2]
        croft_exec_convolve(self.handle, pi, po, _real_ptr(g, n, self.dtype == CROFT_C2C_F64), stream)
        return out

    def describe(self) -> str:
        return croft_plan_describe(self.handle)

    def close(self):
        if self.handle:
            croft_plan_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass
