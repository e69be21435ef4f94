"""Host check of the column split's invariant-divisor division (``csrc/croft_coldiv.h``),
compiled with the host C++ compiler (CPU only).

The column passes split a pencil index into (col / M, col % M) with a multiply-high and two
shifts (Granlund and Montgomery, 1994).  Checked here against Python's integer division for
every divisor up to 5000, every power of two and its neighbours, and random 32-bit divisors,
each on the dividends at the edges (0, d - 1, d, d + 1, 2^31, 2^32 - 1) and random ones.
"""

import os
import random
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2002_04896_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "croft_coldiv.h"
int main() {
    long long d, limit;
    unsigned long long n;
    while (std::scanf("%lld %lld %llu", &d, &limit, &n) == 3) {
        const CroftColDiv v = croft_coldiv_make(d, limit);
        if (!v.m) { std::printf("none\n"); continue; }
        std::printf("%u\n", croft_coldiv_q(v.m, v.s1, v.s2, (unsigned)n));
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def coldiv(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("coldiv")
    src, exe = d / "coldiv.cpp", d / "coldiv"
    src.write_text(PROGRAM)
    subprocess.run([cxx, "-O2", "-std=c++17", f"-I{CSRC}", str(src), "-o", str(exe)], check=True)
    return str(exe)


def _run(exe, cases):
    text = "".join(f"{d} {lim} {n}\n" for d, lim, n in cases)
    out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout.split()
    assert len(out) == len(cases)
    return out


def test_quotients_match_integer_division(coldiv):
    rng = random.Random(20021)
    divisors = list(range(1, 5001))
    divisors += [1 << k for k in range(32)] + [(1 << k) + 1 for k in range(32)] + [(1 << k) - 1 for k in range(2, 33)]
    divisors += [rng.randrange(1, 1 << 32) for _ in range(3000)]
    cases = []
    for d in divisors:
        ns = {0, 1, d - 1, d, d + 1, 2 * d - 1, (1 << 31) - 1, 1 << 31, (1 << 32) - 2, (1 << 32) - 1}
        ns |= {rng.randrange(0, 1 << 32) for _ in range(8)}
        cases += [(d, 1 << 32, n) for n in sorted(ns) if 0 <= n < (1 << 32)]
    out = _run(coldiv, cases)
    bad = [(d, n, q) for (d, _, n), q in zip(cases, out) if q == "none" or int(q) != n // d]
    assert not bad, bad[:10]


def test_out_of_range_divisors_are_refused(coldiv):
    # a divisor or a dividend range beyond 32 bits leaves the divider unset (the kernels divide)
    cases = [(0, 100, 5), (1 << 32, 1 << 32, 5), (7, (1 << 32) + 1, 5), (7, -1, 5)]
    assert _run(coldiv, cases) == ["none"] * 4
