"""Host checks of the tensor-core stage's B operand (``csrc/croft_tc_operand.h``), compiled
with the host C++ compiler (CPU only).

The radix-16 stage multiplies by the real 32 x 32 form [[C, S], [-S, C]] of the 16-point
DFT matrix, split into hi = rn(B) and lo = rn(B - hi) in bfloat16 or binary16.  Pinned here
against numpy's own rounding (float64 -> float16 directly; bfloat16 as the float32 value
rounded to 8 significant bits, ties to even), entry by entry, in the core-matrix layout, and
the two halves together against the exact DFT matrix.
"""

import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2002_04896_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <cstdlib>
#include "croft_tc_operand.h"
int main(int argc, char** argv) {
    if (argc > 1) {  // conversion sweep: read doubles, print both encodings
        double v;
        while (std::scanf("%lf", &v) == 1) std::printf("%u %u\n", f16_bits_rn(v), bf16_bits_rn(v));
        return 0;
    }
    for (int prec = 0; prec < 2; ++prec) {
        unsigned char buf[4096];
        tc_dft16_operand(buf, prec == 1);
        for (int n = 0; n < 32; ++n)
            for (int k = 0; k < 32; ++k) {
                unsigned short hi, lo;
                std::memcpy(&hi, buf + tc_cm_offset(n, k), 2);
                std::memcpy(&lo, buf + 2048 + tc_cm_offset(n, k), 2);
                std::printf("%d %d %d %u %u\n", prec, n, k, hi, lo);
            }
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def prog(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("tcop")
    src = d / "t.cpp"
    src.write_text(PROGRAM.replace("#include <cstdlib>", "#include <cstdlib>\n#include <cstring>"))
    exe = d / "t"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    return str(exe)


def _bf16_bits(v):
    """bfloat16 bits of float64 values: one rounding to 8 significant bits, ties to even."""
    v = np.asarray(v, dtype=np.float64)
    m, e = np.frexp(v)
    ex = np.maximum(e - 1, -126)
    ulp = np.ldexp(1.0, ex - 7)
    r = np.rint(v / ulp) * ulp
    return (r.astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)


def test_conversions_match_numpy(prog):
    rng = np.random.default_rng(0)
    vals = np.concatenate([
        rng.uniform(-1, 1, 4000), rng.uniform(-1e-4, 1e-4, 2000), rng.uniform(-1e-7, 1e-7, 500),
        np.ldexp(rng.integers(1, 2048, 500).astype(np.float64), -24) * rng.choice([-1, 1], 500),
        (np.arange(-1024, 1024) + 0.5) * 2.0 ** -11,  # exact ties of binary16 in [-0.5, 0.5)
        [0.0, 1.0, -1.0, 0.5, 2.0 ** -14, 2.0 ** -24, 3 * 2.0 ** -25, 65504.0]])
    text = "\n".join(repr(float(v)) for v in vals)
    out = subprocess.run([prog, "sweep"], input=text, capture_output=True, text=True, check=True).stdout.split()
    got = np.array(out, dtype=np.int64).reshape(-1, 2)
    np.testing.assert_array_equal(got[:, 0], vals.astype(np.float16).view(np.uint16))
    np.testing.assert_array_equal(got[:, 1], _bf16_bits(vals))


def test_dft16_operand_halves(prog):
    out = subprocess.run([prog], capture_output=True, text=True, check=True).stdout.split()
    rows = np.array(out, dtype=np.int64).reshape(-1, 5)
    j = np.arange(16)
    r = np.outer(j, j) % 16
    f = np.exp(-2j * np.pi * (r / 16.0))  # F[n][j]
    quarter = {0: 1.0, 4: -1j, 8: -1.0, 12: 1j}  # multiples of a quarter turn are exact
    for q, val in quarter.items():
        f[r == q] = val
    big = np.block([[f.real, -f.imag], [f.imag, f.real]])       # B[n][k]: re outputs, then im outputs
    for prec in (0, 1):
        r = rows[rows[:, 0] == prec]
        b = big[r[:, 1], r[:, 2]]
        if prec == 1:
            hi = r[:, 3].astype(np.uint16).view(np.float16).astype(np.float64)
            lo = r[:, 4].astype(np.uint16).view(np.float16).astype(np.float64)
            # compared as values: +0 and -0 are the same operand
            np.testing.assert_array_equal(hi, b.astype(np.float16).astype(np.float64))
            np.testing.assert_array_equal(lo, (b - hi).astype(np.float16).astype(np.float64))
            assert np.max(np.abs(hi + lo - b)) <= 2.0 ** -23
        else:
            hi = (r[:, 3].astype(np.uint32) << 16).astype(np.uint32).view(np.float32).astype(np.float64)
            lo = (r[:, 4].astype(np.uint32) << 16).astype(np.uint32).view(np.float32).astype(np.float64)
            def val(bits):
                return (bits.astype(np.uint32) << 16).astype(np.uint32).view(np.float32).astype(np.float64)
            np.testing.assert_array_equal(hi, val(_bf16_bits(b)))
            np.testing.assert_array_equal(lo, val(_bf16_bits(b - hi)))
            assert np.max(np.abs(hi + lo - b)) <= 2.0 ** -16
        # exact entries (0, +-1) have no lo part
        exact = np.isin(b, [0.0, 1.0, -1.0])
        assert np.all(lo[exact] == 0.0)
