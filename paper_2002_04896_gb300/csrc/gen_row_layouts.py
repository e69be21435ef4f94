#!/usr/bin/env python3
"""Generate croft_row_layouts.h: the shared-memory layout of the row (contiguous-axis) pencils.

For every supported length n the pass kernels keep W pencils of n complex64 in
shared memory, pencil c at c * ld, and the buffer written by Stockham stage s
stores element e at e + (e // L_s) * D_s.  This script replays the kernels'
exact shared-memory access pattern (threads-per-pencil T and pencils per CTA W
as the planner picks them, every stage's reads and writes, one warp instruction
at a time) on a model of the 32 four-byte banks (an 8-byte access by a warp
needs max(ceil(distinct/16), most distinct addresses on one bank pair)
wavefronts) and keeps, per n, the cheapest of: one pad slot per 16 elements for
every stage, the closed-form per-stage pad, and a greedy search over D_s and ld.

Run from this directory:  python3 gen_row_layouts.py > croft_row_layouts.h
"""

import math
from collections import Counter

MAXN = 4096
MAX_STAGES = 8


def supported(n):
    m = n
    for p in (2, 3, 5):
        while m % p == 0:
            m //= p
    return m == 1


def sched(n):
    m, a = n, 0
    while m % 2 == 0:
        m //= 2
        a += 1
    c3 = c5 = 0
    while m % 3 == 0:
        m //= 3
        c3 += 1
    while m % 5 == 0:
        m //= 5
        c5 += 1
    r = []
    aa = a
    while aa >= 4:
        r.append(16)
        aa -= 4
    if aa:
        r.append(1 << aa)
    n9, r3 = c3 // 2, c3 % 2  # must match croft_make_sched: 15, 9s, 5s, 3
    n15 = 1 if (r3 and c5 > 0) else 0
    if n15:
        r3, c5 = 0, c5 - 1
    r = sorted(r + [15] * n15 + [9] * n9 + [5] * c5 + [3] * r3, reverse=True)  # largest radix first ...
    t = threads_per_pencil(n)  # ... but the first stage: the largest radix with <= emax elements per thread
    for i, R in enumerate(r):
        if -(-(n // R) // t) * R <= emax(n):
            r = [R] + r[:i] + r[i + 1:]
            break
    return r


def emax(n):
    return 16 if n <= 1024 else 32


def threads_per_pencil(n):  # must match croft_threads_per_pencil
    t = (n + emax(n) - 1) // emax(n)
    if t <= 32:
        p = 1
        while p < t:
            p *= 2
        return p
    return (t + 31) // 32 * 32


def pencils_per_cta(n, ld):  # must match the planner's ROW shape
    t = threads_per_pencil(n)
    w = max(1, (256 + t - 1) // t)
    while w > 1 and (w * t > 512 or (n + 1 + w * ld) * 8 > 100 * 1024):
        w -= 1
    return w


def wavefronts(addrs):
    d = set(addrs)
    pairs = Counter(a % 16 for a in d)
    return max(math.ceil(len(d) / 16), max(pairs.values()))


def cost(n, lay, ld):
    r = sched(n)
    t = threads_per_pencil(n)
    w = pencils_per_cta(n, ld)
    nthreads = w * t
    total = 0

    def idx(s, a):
        L, D = lay[s]
        return a if D == 0 else a + (a // L) * D

    p = 1
    for s, R in enumerate(r):
        nb = n // R
        qm = (nb + t - 1) // t
        for q in range(qm):
            for w0 in range(0, nthreads, 32):
                act = [(tid // t, tid % t + q * t) for tid in range(w0, min(w0 + 32, nthreads))]
                act = [(c, b) for c, b in act if b < nb]
                if not act:
                    continue
                for j in range(R):
                    if s > 0:
                        total += wavefronts([c * ld + idx(s - 1, b + j * nb) for c, b in act])
                    if s < len(r) - 1:
                        total += wavefronts([c * ld + idx(s, (b - b % p) * R + b % p + j * p) for c, b in act])
        p *= R
    return total


def extent(n, lay):
    ld = n
    for L, D in lay:
        ld = max(ld, (n - 1) + ((n - 1) // L) * D + 1)
    return ld


def closed_form(r, s):
    p = 1
    for i in range(s):
        p *= r[i]
    L = p * r[s]
    if p >= 16:
        return (L, 0)
    runs = (32 + p - 1) // p
    for D in range(16):
        hits = Counter()
        lanes = 0
        for q in range(runs):
            for i in range(p):
                if lanes < 32:
                    e = q * L + i
                    hits[(e + (e // L) * D) % 16] += 1
                    lanes += 1
        if max(hits.values()) <= 2:
            return (L, D)
    return (L, 1)


def fits(n, ld):
    # padding may cost at most a quarter of the pencil (shared memory is occupancy)
    return ld <= n + n // 4 + 16


def best_layout(n):
    r = sched(n)
    ns = len(r) - 1
    if ns <= 0:
        return [], n
    cands = [[(16, 1)] * ns, [closed_form(r, s) for s in range(ns)]]
    scored = []
    for lay in cands:
        ld0 = extent(n, lay)
        for extra in range(0, 4):
            if fits(n, ld0 + extra) or lay is cands[0]:
                scored.append((cost(n, lay, ld0 + extra), lay, ld0 + extra))
    scored.sort(key=lambda x: x[0])
    _, cur, ld = scored[0]
    cur = list(cur)
    if n <= 1024:  # greedy refinement (larger sizes: too slow to model, keep the best candidate)
        for s in range(ns):
            best = None
            for D in range(0, 17):
                trial = list(cur)
                trial[s] = (cur[s][0], D)
                ldt = extent(n, trial)
                if not fits(n, ldt):
                    continue
                c = cost(n, trial, ldt)
                if best is None or c < best[0]:
                    best = (c, D)
            cur[s] = (cur[s][0], best[1])
        ld0 = extent(n, cur)
        best = None
        for extra in range(0, 17):
            if not fits(n, ld0 + extra) and extra > 0:
                continue
            c = cost(n, cur, ld0 + extra)
            if best is None or c < best[0]:
                best = (c, ld0 + extra)
        ld = best[1]
    return cur, ld


def main():
    print("// croft_row_layouts.h - GENERATED by gen_row_layouts.py; do not edit by hand.")
    print("// Shared-memory layout of the row pencils for every supported length n:")
    print("// pencil stride ld and, per stage s, the padding e -> e + (e / L[s]) * D[s] of")
    print("// the buffer stage s writes (chosen on a model of the 32 shared-memory banks).")
    print("#pragma once")
    print()
    print("struct CroftRowLayout {")
    print("    int ld;")
    print(f"    int L[{MAX_STAGES}];")
    print(f"    int D[{MAX_STAGES}];")
    print("};")
    print()
    print("CROFT_HD constexpr CroftRowLayout croft_row_layout(int n) {")
    print("    switch (n) {")
    for n in range(2, MAXN + 1):
        if not supported(n) or len(sched(n)) < 2:
            continue
        lay, ld = best_layout(n)
        Ls = [l for l, _ in lay] + [1] * (MAX_STAGES - len(lay))
        Ds = [d for _, d in lay] + [0] * (MAX_STAGES - len(lay))
        print(f"        case {n}: return CroftRowLayout{{{ld}, {{{', '.join(map(str, Ls))}}}, "
              f"{{{', '.join(map(str, Ds))}}}}};")
    print("        default: return CroftRowLayout{n, {1, 1, 1, 1, 1, 1, 1, 1}, {0, 0, 0, 0, 0, 0, 0, 0}};")
    print("    }")
    print("}")


if __name__ == "__main__":
    main()
