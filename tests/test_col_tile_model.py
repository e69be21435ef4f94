"""Host model of the first-stage shared-memory stores of a narrow (8-column, 64-byte
row) column tile (CPU only).

In a column pass the tile holds element a of column c at float2 index a * W + c; a
warp is 32 / W pencil-lanes times W columns, and in the first stage (p = 1) lane b
writes output j of its radix-R butterfly to row R * b + j.  Shared memory serves
8-byte accesses in 16 bank pairs per wavefront.  With W = 8 a row covers half of the
bank pairs, so when R is even the four rows one store instruction writes (consecutive
b, the same j) all fall on the same half.  The kernels then let odd butterflies store
each output pair (j, j+1) in swapped order (``SmemColFixed::kPairSwap`` in
``csrc/croft_fft_core.cuh``).  These checks replay both orders.
"""

import math
from collections import Counter

import pytest


def wavefronts(addrs):
    """Wavefronts for one warp's 8-byte accesses: distinct addresses, 16 bank pairs."""
    d = set(addrs)
    return max(math.ceil(len(d) / 16), max(Counter(a % 16 for a in d).values()))


def first_stage_stores(R, W, T, swap):
    """Per store instruction, the tile indices one warp writes; and every thread's row set."""
    nthreads = W * T
    nb = 512 // R if 512 % R == 0 else 480 // R  # butterflies per pencil (any multiple of T works)
    qm = -(-nb // T)
    per_instr = []
    rows_of = {}
    for w0 in range(0, nthreads, 32):
        for q in range(qm):
            for i in range(R):
                addrs = []
                for tid in range(w0, w0 + 32):
                    c, b = tid % W, tid // W + q * T
                    if b >= nb:
                        continue
                    odd = b & 1 if swap else 0
                    j = i ^ odd if (swap and R % 2 == 0) else i
                    row = R * b + j
                    addrs.append(row * W + c)
                    rows_of.setdefault((tid, q), []).append(row)
                if addrs:
                    per_instr.append(addrs)
    return per_instr, rows_of


@pytest.mark.parametrize("R", [2, 4, 8, 16])
def test_pair_swap_removes_first_stage_conflicts_on_64_byte_rows(R):
    plain, rows_plain = first_stage_stores(R, 8, 32, swap=False)
    swapped, rows_swapped = first_stage_stores(R, 8, 32, swap=True)
    ideal = sum(math.ceil(len(set(a)) / 16) for a in plain)
    assert sum(wavefronts(a) for a in plain) == 2 * ideal  # every instruction on one half
    assert sum(wavefronts(a) for a in swapped) == ideal
    # the same stores: each thread writes the same rows, only in another order
    assert {k: sorted(v) for k, v in rows_plain.items()} == {k: sorted(v) for k, v in rows_swapped.items()}


@pytest.mark.parametrize("R", [3, 5, 9, 15])
def test_odd_first_radix_needs_no_swap(R):
    plain, _ = first_stage_stores(R, 8, 32, swap=False)
    ideal = sum(math.ceil(len(set(a)) / 16) for a in plain)
    assert sum(wavefronts(a) for a in plain) == ideal


@pytest.mark.parametrize("R", [2, 4, 8, 16])
def test_128_byte_rows_have_no_first_stage_conflicts(R):
    """16-column tiles (the default width) cover every bank pair in one row."""
    plain, _ = first_stage_stores(R, 16, 32, swap=False)
    ideal = sum(math.ceil(len(set(a)) / 16) for a in plain)
    assert sum(wavefronts(a) for a in plain) == ideal
