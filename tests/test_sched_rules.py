"""Host checks of the compile-time schedule and tile rules of the pass kernels
(``csrc/croft_sched.h``), compiled with the host C++ compiler (CPU only).

The kernels, the planner and the twiddle-table builder all take their radix
schedules, threads per pencil, column-tile widths and launch bounds from this
one header; these tests pin the rules it states for every supported length:
the schedule is a factorisation into the butterfly set with the first-stage
rule, the tiles fit the launch and shared-memory limits, and the narrow
8-column tile is chosen exactly for short-stride complex64 passes of 32-thread
pencils.
"""

import math
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2002_04896_gb300", "csrc")
RADICES = {2, 3, 4, 5, 8, 9, 15, 16}
# 32-thread lengths whose short-stride column passes keep the 16-column tile (measured faster)
WIDE_SHORT_STRIDE = {270, 288, 300, 320, 375, 384, 400}

PROGRAM = r"""
#include <cstdio>
#include <initializer_list>
#include "croft_sched.h"
int main() {
    for (int n = 2; n <= 4096; ++n) {
        int m = n;
        for (int p : {2, 3, 5})
            while (m % p == 0) m /= p;
        if (m != 1) continue;
        for (int layout = 0; layout < 2; ++layout) {
            const CroftSched s = croft_pass_sched(n, layout, 8);
            std::printf("S %d %d", n, layout);
            for (int i = 0; i < s.count; ++i) std::printf(" %d", s.r[i]);
            std::printf("\n");
        }
        std::printf("T %d %d\n", n, croft_threads_per_pencil(n));
        for (int es : {8, 16})
            std::printf("W %d %d %d %d %d\n", n, es, croft_col_width(n, es), croft_col_width_at(n, es, 4096),
                        croft_col_width_at(n, es, 1 << 21));
        std::printf("B %d %d %d %d\n", n, croft_col_minb(n, 8), croft_pass_minb(n, 8), croft_col_narrow_minb(n));
        std::printf("X %d %d %d %d %d\n", n, croft_col_t24(n, true) ? 1 : 0, croft_col_t24(n, false) ? 1 : 0,
                    croft_col_sv_default(n, 8, 4096), croft_col_sv_default(n, 8, 1 << 21));
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def rules(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("sched")
    src, exe = d / "rules.cpp", d / "rules"
    src.write_text(PROGRAM)
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    r = {"S": {}, "T": {}, "W": {}, "B": {}, "X": {}}
    for line in out.splitlines():
        tag, *v = line.split()
        v = [int(a) for a in v]
        if tag == "S":
            r["S"][(v[0], v[1])] = v[2:]
        elif tag == "T":
            r["T"][v[0]] = v[1]
        elif tag == "W":
            r["W"][(v[0], v[1])] = v[2:]
        elif tag == "X":
            r["X"][v[0]] = v[1:]
        else:
            r["B"][v[0]] = v[1:]
    return r


def test_every_length_is_covered(rules):
    assert len(rules["T"]) == 136  # 2 <= n <= 4096 of the form 2^a 3^b 5^c


def test_schedules_factorise_into_the_butterfly_set(rules):
    for (n, layout), rs in rules["S"].items():
        assert math.prod(rs) == n, (n, layout, rs)
        assert set(rs) <= RADICES, (n, layout, rs)
        assert len(rs) <= 8


def test_first_stage_rule(rules):
    """The first stage (the one that loads from HBM) takes a radix whose butterflies give
    a thread at most emax elements whenever the schedule has one."""
    for (n, layout), rs in rules["S"].items():
        t = rules["T"][n]
        emax = 16 if n <= 1024 else 32
        per_thread = [-(-(n // r) // t) * r for r in rs]
        if any(e <= emax for e in per_thread):
            assert per_thread[0] <= emax, (n, layout, rs, t)


def test_power_of_two_split(rules):
    """Row passes split the power-of-two part greedily into radix-16 stages; column
    passes of complex64 32-thread pencils split it into near-equal stages."""
    for (n, layout), rs in rules["S"].items():
        pow2 = sorted((r for r in rs if r in (2, 4, 8, 16)), reverse=True)
        a = int(math.log2(math.prod(pow2))) if pow2 else 0
        if a == 0:
            continue
        even = layout == 1 and rules["T"][n] == 32
        if even:
            k = -(-a // 4)
            sizes = sorted((int(math.log2(r)) for r in pow2), reverse=True)
            assert len(sizes) == k and max(sizes) - min(sizes) <= 1, (n, rs)
        else:
            assert [int(math.log2(r)) for r in pow2][:-1] == [4] * (len(pow2) - 1), (n, rs)


def test_threads_per_pencil(rules):
    for n, t in rules["T"].items():
        assert t == 1 << (t.bit_length() - 1) and t <= 32 or t % 32 == 0, (n, t)
        emax = 16 if n <= 1024 else 32
        assert t * emax >= n, (n, t)


def test_column_tiles_fit_the_launch_and_shared_memory(rules):
    for (n, es), (w, w_short, w_long) in rules["W"].items():
        t = rules["T"][n]
        tw_pad = (n + 1) // 2 * 2
        for width in (w, w_short, w_long):
            assert width >= 1 and width * t <= 512, (n, es, width, t)
            fits = (tw_pad + n * width) * es <= 100 * 1024
            assert fits or width == 1, (n, es, width)  # narrowed down to one column at most
            assert fits or es == 16, (n, es, width)  # every complex64 length fits
        assert w_long == w, (n, es)  # megabyte strides keep the default width
        narrow = es == 8 and t == 32 and n not in WIDE_SHORT_STRIDE
        assert (w_short == 8 and w_short != w) == narrow, (n, es, w, w_short)
        if not narrow:
            assert w_short == w


def test_launch_bounds(rules):
    for n, (col_minb, pass_minb, narrow_minb) in rules["B"].items():
        t = rules["T"][n]
        assert col_minb == (3 if t == 32 else 1), n
        assert pass_minb == (5 if n in (256, 270, 288, 300, 324, 375, 400, 432, 480) else 0), n
        assert narrow_minb in (4, 5), n
        assert (narrow_minb == 4) == (n in (480, 486, 500)), n
        # registers a thread may keep under the bound: 48 for five 256-thread CTAs, 64 for four
        assert 65536 // (narrow_minb * 256) >= 48


def test_24_thread_pencils(rules):
    # the 24-thread column kernels exist only for 32-thread lengths; their CTAs (8 or 16 columns
    # x 24 threads) stay within the launch bound and the shared-memory budget of the tile
    chosen = {n for n, (nar, wide, _, _) in rules["X"].items() if nar or wide}
    assert chosen == {324, 360, 384, 405}
    for n in chosen:
        assert rules["T"][n] == 32, n
        nar, wide, _, _ = rules["X"][n]
        w, w_short, _ = rules["W"][(n, 8)]
        assert w == 16 and (w_short == 8 or not nar), n  # short-stride 24-thread lengths are narrow
        for width, on in ((w_short, nar), (w, wide)):
            if on:
                assert width * 24 <= 512 and 24 * 20 >= n, (n, width)  # at most 20 points a thread
                assert ((n + 1) // 2 * 2 + n * width) * 8 <= 100 * 1024, (n, width)
        # 24 lanes use the butterfly slots of every stage at least as well as 32
        s = rules["S"][(n, 1)]
        def util(t):
            return sum(n // r for r in s) / sum(-(-(n // r) // t) * t for r in s)
        assert util(24) >= util(32) - 0.05, (n, util(24), util(32))


def test_radix16_first_split_by_default(rules):
    # the rules' schedule variant: 320 points at every stride (16·5·4), 512 at short strides
    # (16·8·4); both are 32-thread lengths whose variant kernels exist (16-column at 320, the
    # narrow tile at 512)
    sv = {n: tuple(v[2:]) for n, v in rules["X"].items() if v[2] or v[3]}
    assert sv == {320: (1, 1), 512: (2, 0)}
    for n in sv:
        assert rules["T"][n] == 32
    assert rules["W"][(320, 8)][1] == 16 and rules["W"][(512, 8)][1] == 8


def test_mixed_split_of_512(tmp_path):
    import shutil, subprocess
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "m.cpp"
    src.write_text('#include <cstdio>\n#include "croft_sched.h"\nint main(){CroftSched s=croft_pass_sched_v(512,1,8,2);'
                   'for(int i=0;i<s.count;++i)std::printf("%d ",s.r[i]);return 0;}\n')
    exe = tmp_path / "m"
    subprocess.run([cxx, "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    assert [int(v) for v in out] == [16, 8, 4]


def _run_snippet(tmp_path, body):
    import shutil, subprocess
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "s.cpp"
    src.write_text('#include <cstdio>\n#include <initializer_list>\n#include "croft_sched.h"\nint main(){' + body + 'return 0;}\n')
    exe = tmp_path / "s"
    subprocess.run([cxx, "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    return subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout


def test_tensor_core_schedule_has_one_radix16_stage_first(tmp_path):
    # every length <= 1024 with a factor 16: one radix-16 stage (the tensor-core one) first, then
    # a factorisation of n / 16 into the butterfly set
    out = _run_snippet(tmp_path, 'for(int n=16;n<=1024;n+=16){CroftSched s=croft_make_sched_tc(n);'
                                 'std::printf("%d",n);for(int i=0;i<s.count;++i)std::printf(" %d",s.r[i]);std::printf("\\n");}')
    for line in out.strip().splitlines():
        n, *rs = (int(v) for v in line.split())
        m = n
        for p in (2, 3, 5):
            while m % p == 0:
                m //= p
        if m != 1:
            assert rs == [], (n, rs)  # not of the form 2^a 3^b 5^c: no schedule
            continue
        assert rs[0] == 16, (n, rs)
        assert math.prod(rs) == n and set(rs) <= RADICES, (n, rs)
    assert "512 16 8 4" in out and "256 16 16" in out and "1024 16 8 8" in out


def test_pair_and_16_thread_defaults(tmp_path):
    out = _run_snippet(tmp_path, 'for(int n : {480, 486, 500, 512, 432, 450}) for(long long sb : {4096LL, 1LL << 18, 1LL << 21})'
                                 'std::printf("%d %lld %d %d\\n", n, sb, croft_pair_default(n, 8, sb) ? 1 : 0, croft_col_t16(n, 8, sb) ? 1 : 0);')
    got = {(int(a), int(b)): (int(c), int(d)) for a, b, c, d in (line.split() for line in out.strip().splitlines())}
    for (n, sb), (pair, t16) in got.items():
        assert pair == int(n == 486 or (n in (500, 512) and sb >= 1 << 18)), (n, sb)
        assert t16 == int(n in (432, 480) and sb >= 1 << 18), (n, sb)
