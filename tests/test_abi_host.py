"""C-ABI library: loads, exports every declared symbol, host-side validation (no GPU needed)."""

import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(croft_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_symbol(croft_lib):
    lib = ctypes.CDLL(croft_lib.LIBRARY_PATH)
    declared = _declared_symbols()
    assert len(declared) >= 10
    for name in declared:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    assert set(croft_lib.EXPORTED) <= set(declared)


def test_status_strings(croft_lib):
    for code, name in [(0, "CROFT_OK"), (1, "CROFT_ERR_INVALID_ARG"), (2, "CROFT_ERR_UNSUPPORTED_SIZE"),
                       (3, "CROFT_ERR_OOM"), (4, "CROFT_ERR_CUDA"), (5, "CROFT_ERR_TIMEOUT")]:
        assert croft_lib.croft_status_string(code) == name
    assert croft_lib.croft_status_string(99) == "CROFT_ERR_UNKNOWN"


@pytest.mark.parametrize("dims", [(7, 8, 8), (8, 8, 0), (4097, 1, 1), (11, 2, 2), (8, 8, -4), (1, 14, 1)])
def test_unsupported_sizes_rejected_before_any_device_call(croft_lib, dims):
    st, h = croft_lib.croft_plan_create_status(*dims)
    assert st == croft_lib.CROFT_ERR_UNSUPPORTED_SIZE and h is None


def test_bad_dtype_and_null_out(croft_lib):
    st, h = croft_lib.croft_plan_create_status(8, 8, 8, 7)
    assert st == croft_lib.CROFT_ERR_INVALID_ARG and h is None
    lib = ctypes.CDLL(croft_lib.LIBRARY_PATH)
    lib.croft_plan_create.restype = ctypes.c_int
    assert lib.croft_plan_create(None, 8, 8, 8, 0) == croft_lib.CROFT_ERR_INVALID_ARG


def test_null_plan_calls(croft_lib):
    assert croft_lib.croft_exec_forward_status(None, 0, 0, 0) == croft_lib.CROFT_ERR_INVALID_ARG
    assert croft_lib.croft_exec_backward_status(None, 0, 0, 0) == croft_lib.CROFT_ERR_INVALID_ARG
    croft_lib.croft_plan_destroy(None)  # no-op
    assert croft_lib.croft_plan_last_device_status(None) == croft_lib.CROFT_ERR_INVALID_ARG
    assert croft_lib.croft_plan_num_launches(None) == -1


def test_no_cpu_fallback_without_a_gpu(croft_lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    st, h = croft_lib.croft_plan_create_status(8, 8, 8)
    assert st == croft_lib.CROFT_ERR_CUDA and h is None


def _supported(n):
    for p in (2, 3, 5):
        while n % p == 0:
            n //= p
    return n == 1


def test_factorize_all_sizes(croft_lib):
    for n in range(1, 4100):
        r = croft_lib.croft_factorize(n)
        if not _supported(n) or n > 4096:
            assert r is None, n
            continue
        assert r is not None
        assert int(np.prod(r)) == n if r else n == 1
        assert all(x in (2, 3, 4, 5, 8, 9, 15, 16) for x in r)
        assert len(r) <= 7


@pytest.mark.parametrize("n", [2, 3, 5, 16, 32, 60, 256, 360, 480, 512, 4096, 3888])
def test_twiddle_tables_match_float64_exponentials(croft_lib, n):
    """Entry p-1+(j-1)p+k of the table is exp(-2 pi i jk/(pR)) rounded to float32 (within one rounding)."""
    r = croft_lib.croft_factorize(n)
    tw = croft_lib.croft_twiddle_table(n, r)
    assert tw is not None and tw.shape == (n - 1,)
    ref = np.empty(n - 1, dtype=np.complex128)
    p = 1
    for R in r:
        j = np.arange(1, R)[:, None]
        k = np.arange(p)[None, :]
        ref[p - 1:p - 1 + (R - 1) * p] = np.exp(-2j * np.pi * ((j * k) % (p * R)) / (p * R)).ravel()
        p *= R
    err = np.abs(tw.astype(np.complex128) - ref)
    assert err.max() <= 2.0 ** -24 * 1.5, err.max()
    # quarter-turn multiples are exact
    p = 1
    for R in r:
        for j in range(1, R):
            for k in range(p):
                if (4 * j * k) % (p * R) == 0:
                    q = (4 * j * k) // (p * R)
                    assert tw[p - 1 + (j - 1) * p + k] == [1, -1j, -1, 1j][q % 4]
        p *= R


def test_row_layout_generator_models_the_library_schedule(croft_lib):
    """gen_row_layouts.py replays the kernels' stages: its schedule must be the library's, for every length."""
    import importlib.util
    import os
    path = os.path.join(os.path.dirname(croft_lib.LIBRARY_PATH), "csrc", "gen_row_layouts.py")
    spec = importlib.util.spec_from_file_location("gen_row_layouts", path)
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    for n in range(2, 4097):
        if gen.supported(n):
            assert gen.sched(n) == croft_lib.croft_factorize(n), n


def test_noalloc_binding_rejects_bad_lists_before_the_library(croft_lib):
    """The C side of croft_exec_batched_noalloc trusts dims for every size; the binding checks
    the lists first: counts, element counts and dtype (CPU tensors, so nothing reaches a device)."""
    import torch
    dims = [(4, 4, 4), (2, 3, 5)]
    good = [torch.zeros(d, dtype=torch.complex64) for d in dims]
    with pytest.raises(ValueError, match="inputs and outputs"):
        croft_lib.croft_exec_batched_noalloc_status(dims, good[:1], good, -1)
    with pytest.raises(ValueError, match="inputs and outputs"):
        croft_lib.croft_exec_batched_noalloc_status(dims, good, good[:1], -1)
    short = [torch.zeros((4, 4, 3), dtype=torch.complex64), good[1]]
    with pytest.raises(ValueError, match="elements"):
        croft_lib.croft_exec_batched_noalloc_status(dims, short, good, -1)
    wide = [torch.zeros(d, dtype=torch.complex128) for d in dims]
    with pytest.raises(ValueError, match="complex64"):
        croft_lib.croft_exec_batched_noalloc_status(dims, good, wide, -1)
    with pytest.raises(ValueError, match="three axis lengths"):
        croft_lib.croft_exec_batched_noalloc_status([(4, 4)], good[:1], good[:1], -1)
    # well-formed lists get as far as the device check
    with pytest.raises(ValueError, match="CUDA device"):
        croft_lib.croft_exec_batched_noalloc_status(dims, good, good, -1)
