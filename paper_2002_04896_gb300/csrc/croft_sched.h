// croft_sched.h - the radix schedule of a length-n axis, shared by the host
// planner (twiddle-table layout, launch shape) and the device kernels (which
// are specialised on n, so every loop bound, stride and twiddle offset is a
// compile-time constant).
#pragma once

#ifdef __CUDACC__
#define CROFT_HD __host__ __device__
#else
#define CROFT_HD
#endif

#define CROFT_MAX_STAGES 8  // 2^a 3^b 5^c <= 4096 needs at most 7 stages
#define CROFT_MAX_N 4096

struct CroftSched {
    int count;                  // number of stages (0 for n = 1, -1 if unsupported)
    int r[CROFT_MAX_STAGES];    // radix of each stage, in execution order
};

// Schedule: the power-of-two part of n as radix-16 stages and one stage with the
// rest (2, 4 or 8; measured against near-equal splits: 64 = 16·4 vs 8·8 45 vs 51
// us per pass at 64x64x4096, 512 = 16·16·2 vs 8·8·8 324 vs 332 us for the row
// pass, the others equal); then the odd part with the fewest
// stages of at most 16 points: pairs of factors 3 as radix 9, an unpaired 3 with a
// 5 as radix 15, then the remaining 5s and 3 (each stage is a shared-memory round
// trip and a barrier).  The first stage needs no twiddles, so the largest radix
// goes there.
//
// even_pow2: the power-of-two part in ceil(a/4) stages of near-equal size instead
// (croft_pass_sched picks it for the column passes of 32-thread pencils).
CROFT_HD constexpr CroftSched croft_make_sched(int n, bool even_pow2 = false) {
    CroftSched s{0, {0, 0, 0, 0, 0, 0, 0, 0}};
    if (n < 1 || n > CROFT_MAX_N) {
        s.count = -1;
        return s;
    }
    int m = n, a = 0, c3 = 0, c5 = 0;
    while (m % 2 == 0) { m /= 2; ++a; }
    while (m % 3 == 0) { m /= 3; ++c3; }
    while (m % 5 == 0) { m /= 5; ++c5; }
    if (m != 1) {
        s.count = -1;
        return s;
    }
    int k = 0;
    if (even_pow2 && a > 0) {
        const int st = (a + 3) / 4;
        const int base = a / st, extra = a % st;
        for (int i = 0; i < st; ++i) s.r[k++] = 1 << (base + (i < extra ? 1 : 0));
    } else {
        for (int aa = a; aa > 0; aa -= 4) s.r[k++] = 1 << (aa >= 4 ? 4 : aa);
    }
    const int n9 = c3 / 2;
    int r3 = c3 % 2;
    const int n15 = (r3 && c5 > 0) ? 1 : 0;
    if (n15) {
        r3 = 0;
        c5 -= 1;
    }
    for (int i = 0; i < n15; ++i) s.r[k++] = 15;
    for (int i = 0; i < n9; ++i) s.r[k++] = 9;
    for (int i = 0; i < c5; ++i) s.r[k++] = 5;
    for (int i = 0; i < r3; ++i) s.r[k++] = 3;
    s.count = k;
    // Largest radix first (insertion sort; at most 8 stages) ...
    for (int i = 1; i < k; ++i)
        for (int j = i; j > 0 && s.r[j] > s.r[j - 1]; --j) {
            const int t = s.r[j];
            s.r[j] = s.r[j - 1];
            s.r[j - 1] = t;
        }
    // ... except that the first stage - the one that loads from HBM - takes the largest radix
    // whose butterflies give a thread at most emax elements (croft_threads_per_pencil's
    // budget), when there is one: 480 = 15·8·4 (15 per thread) ran its passes 294-350 us, but
    // 360 = 9·8·5 (two 9-point butterflies, 18 per thread) 182 us against 162 for 8·9·5.
    const int emax = n <= 1024 ? 16 : 32;
    int tpp = (n + emax - 1) / emax;
    if (tpp > 32) {
        tpp = (tpp + 31) / 32 * 32;
    } else {
        int p2 = 1;
        while (p2 < tpp) p2 *= 2;
        tpp = p2;
    }
    for (int i = 0; i < k; ++i) {
        const int nb = n / s.r[i];
        if (((nb + tpp - 1) / tpp) * s.r[i] <= emax) {
            const int first = s.r[i];
            for (int j = i; j > 0; --j) s.r[j] = s.r[j - 1];
            s.r[0] = first;
            break;
        }
    }
    return s;
}

// Schedule of the tensor-core variant: one radix-16 stage first (it runs as a split-operand
// GEMM on the tensor cores), then the near-equal split of the rest on the CUDA cores.  One
// tensor-core stage instead of one per factor 16: each such stage costs a GEMM round trip and
// adds the split's rounding (512^3 forward+backward, bf16x3: 3.55 -> 3.31 ms, round trip
// 1.12e-5 -> 7.6e-6; fp16x3 3.78 -> 3.34 ms, 2.0e-6 -> 1.1e-6).
CROFT_HD constexpr CroftSched croft_make_sched_tc(int n) {
    CroftSched s{0, {0, 0, 0, 0, 0, 0, 0, 0}};
    int m = n, k = 0;
    if (m > 1 && m % 16 == 0) {
        s.r[k++] = 16;
        m /= 16;
    }
    const CroftSched rest = croft_make_sched(m, true);
    if (rest.count < 0 || k + rest.count > CROFT_MAX_STAGES) {
        s.count = -1;
        return s;
    }
    for (int i = 0; i < rest.count; ++i) s.r[k++] = rest.r[i];
    s.count = k;
    return s;
}

// Length of the sub-transforms that stage `stage` combines (product of the earlier radices).
CROFT_HD constexpr int croft_sched_p(const CroftSched& s, int stage) {
    int p = 1;
    for (int i = 0; i < stage; ++i) p *= s.r[i];
    return p;
}

// Padded shared-memory length of one pencil in the row layout: one pad slot per
// 16 elements keeps the stride-R writes of the early Stockham stages conflict-free.
CROFT_HD constexpr int croft_row_ld(int n) { return n + (n - 1) / 16 + 1; }

#include "croft_row_layouts.h"

// Pencil stride (float2 slots) of the row layout with per-stage padding (croft_row_layouts.h).
CROFT_HD constexpr int croft_row_ld_staged(int n) { return croft_make_sched(n).count > 1 ? croft_row_layout(n).ld : n; }

// Per-thread element budget and threads per pencil of the pass kernels.
CROFT_HD constexpr int croft_emax(int n) { return n <= 1024 ? 16 : 32; }
// Threads per pencil: at least n / emax, rounded up to a power of two (<= 32) or a
// multiple of 32, so that a warp never straddles pencils unevenly.
CROFT_HD constexpr int croft_threads_per_pencil(int n) {
    const int t = (n + croft_emax(n) - 1) / croft_emax(n);
    if (t > 32) return (t + 31) / 32 * 32;
    int p = 1;
    while (p < t) p *= 2;
    return p;
}

// The schedule of a pass over a length-n axis (layout 0 = ROW, 1 = COL; es = complex
// element size): the column passes of complex64 32-thread pencils (lengths 270..512,
// bounded to 40 registers) take the near-equal power-of-two split - at 480 the
// column passes ran 330 / 349 us with 15·8·4 against 340 / 362 with 16·15·2, while the
// row pass prefers 16·15·2 (285 vs 294 us) - every other pass the radix-16 one.
// Twiddle tables are built for the pass's schedule.
CROFT_HD constexpr bool croft_even_pow2_pass(int n, int layout, int es) {
    return layout == 1 && es == 8 && croft_threads_per_pencil(n) == 32;
}
CROFT_HD constexpr CroftSched croft_pass_sched(int n, int layout, int es) {
    return croft_make_sched(n, croft_even_pow2_pass(n, layout, es));
}
// Schedule variants a tuned plan may pick per pass (CROFT_SCHEDULE_TUNED): sv = 0 the rule
// above; sv = 1 the other power-of-two split for the passes that have one built (the column
// passes of complex64 32-thread pencils: the radix-16-first split instead of the near-equal
// one).  croft_sched_variants(n, layout, es) is 2 for those passes, else 1.
CROFT_HD constexpr int croft_sched_variants(int n, int layout, int es) { return croft_even_pow2_pass(n, layout, es) ? 2 : 1; }
// Schedule variant 2: one radix-16 stage first, then the near-equal split of the rest (512 =
// 16·8·4); a rule's choice only (croft_col_sv_default), not a tuner candidate.
CROFT_HD constexpr CroftSched croft_make_sched_mixed(int n) {
    CroftSched rest = croft_make_sched(n / 16, true);
    CroftSched s{0, {0, 0, 0, 0, 0, 0, 0, 0}};
    s.r[0] = 16;
    for (int i = 0; i < rest.count; ++i) s.r[1 + i] = rest.r[i];
    s.count = rest.count + 1;
    return s;
}
CROFT_HD constexpr CroftSched croft_pass_sched_v(int n, int layout, int es, int sv) {
    return sv == 2 ? croft_make_sched_mixed(n) : croft_make_sched(n, croft_even_pow2_pass(n, layout, es) && sv == 0);
}
// The schedule variant the rules give a column pass (where the sweep of every 32-thread length
// measured another split faster by more than 1.5 %): 320 points at every stride, variant 1
// (16·5·4 against 8·8·5, 16-column tiles: y of 512 x 320 x 512 231 / 260 us, x of 320 x 512 x
// 512 240 / 287); the 512-point short-stride pass, variant 2 (16·8·4; 8-column tiles: 512^3 y
// 387 us against 391 for 16·16·2 and 399 for 8·8·8).  Twiddle tables follow the pass's
// variant; a fused convolution on such an axis gets a table of its own.
CROFT_HD constexpr int croft_col_sv_default(int n, int es, long long stride_bytes) {
    return (es == 8 && n == 512 && stride_bytes <= 16 * 1024) ? 2 : ((es == 8 && n == 320) ? 1 : 0);
}

// Column-tile width (columns per CTA) of a COL pass - a compile-time constant of
// its kernel - for length n and complex element size es bytes: 16 columns
// (128-byte rows), widened while the CTA stays within 256 threads, narrowed while
// the CTA exceeds 512 threads or the data tile 100 KB.  (A strided-copy probe
// with the same tiles reaches 0.97 of the copy peak across the x pass's
// megabyte strides with 16 columns and 0.47 with 8.)
CROFT_HD constexpr int croft_col_width(int n, int es) {
    const int t = croft_threads_per_pencil(n);
    int w = 16;
    while (w * 2 * t <= 256) w *= 2;
    const long long tw_pad = ((n + 1) / 2) * 2;
    while (w > 1 && (w * t > 512 || (tw_pad + (long long)n * w) * es > 100 * 1024)) w /= 2;
    return w;
}

// CTAs per SM that a COL pass kernel's register allocation must allow (its launch
// bound).  Complex64 pencils of 32 threads (lengths 270..512) make 512-thread
// CTAs that take ~60 registers unconstrained - two per SM, and the compute phase
// of both can leave no loads in flight; bounding them to three per SM (40
// registers, 12-44 bytes of spills) measured 15-37 % faster on the y and x passes
// of 320^3 .. 512^3 grids.
CROFT_HD constexpr int croft_col_minb(int n, int es) { return (es == 8 && croft_threads_per_pencil(n) == 32) ? 3 : 1; }

// Short-stride column passes of complex64 32-thread pencils (the y pass: the axis's
// elements at most 16 KB apart) take 8-column, 256-thread tiles bounded to five CTAs
// per SM instead (48 registers, 0-52 bytes of spills; croft_col_narrow_minb): 512^3 y
// pass 455 -> 414 us, 320^3 121 -> 115 us, 360-point y pass of 384x360x320 162 -> 160
// us, 480^3 330 -> 332 us.  Across the x pass's megabyte strides the 64-byte row pieces
// lose (512^3 487 -> 649 us), so that pass keeps croft_col_width's 16 columns.
constexpr int kColNarrowWidth = 8;
// CTAs per SM the narrow kernel's registers must allow: five (48 registers), except where
// four (64) measured faster - the lengths whose five-CTA build spills most, and 480.  y pass
// of a 128 x n x 512 grid, five vs four: 480 100.3 / 98.3 us, 486 157.7 / 149.5, 500 143.4 /
// 139.3; the other 13 lengths 0-7 % slower at four (512 110.6 / 116.7, 400 81.9 / 88.0).
CROFT_HD constexpr int croft_col_narrow_minb(int n) { return (n == 480 || n == 486 || n == 500) ? 4 : 5; }
// Lengths whose short-stride passes keep the 16-column tile: per-pass events on 512 x n x 512
// (4 KB strides), 16 vs 8 columns, us: 270 206 / 219, 288 213 / 227, 300 225 / 235, 320 231 /
// 235 (radix-16-first split), 375 277 / 286, 384 268 / 280, 400 286 / 295 (the other lengths
// 3-15 % faster with 8).
CROFT_HD constexpr bool croft_col_narrow(int n, int es, long long stride_bytes) {
    return es == 8 && croft_threads_per_pencil(n) == 32 && stride_bytes <= 16 * 1024 && n != 270 && n != 288 &&
           n != 300 && n != 320 && n != 375 && n != 384 && n != 400;
}
// 24 threads per pencil instead of 32 for the complex64 column passes of some 270..512-point
// axes (short: strides of at most 16 KB, where these lengths take the 8-column tile; else the
// 16-column tile).  With 32 threads
// the butterflies of a stage often leave lanes idle (360 = 8·9·5: 45, 40 and 72 butterflies
// on 32 lanes use 70 % of the slots; on 24 lanes 93 %); the rule lists the lengths where 24
// measured faster and the kernel does not spill (56 registers: six 192-thread narrow CTAs or
// three 384-thread wide CTAs per SM).  Per-pass events, 24 vs 32 threads, y pass of
// 512 x n x 512 / x pass of n x 512 x 512: 270 0.97 / 1.00, 288 1.09 / 1.25, 300 0.99 / 1.00,
// 320 0.92 / 0.97, 324 0.95 / 0.93, 360 0.88 / 0.94, 384 1.05 / 0.94, 405 0.93 / 0.98 of the
// 32-thread time (the other lengths spill at 24).
CROFT_HD constexpr bool croft_col_t24(int n, bool short_stride) {
    if (short_stride) return n == 324 || n == 360 || n == 405;
    return n == 324 || n == 360 || n == 384 || n == 405;
}
// Column-tile width of a COL pass over a length-n axis whose elements lie stride_bytes apart.
CROFT_HD constexpr int croft_col_width_at(int n, int es, long long stride_bytes) {
    return croft_col_narrow(n, es, stride_bytes) ? kColNarrowWidth : croft_col_width(n, es);
}

// CTAs per SM that a 256-thread pass kernel's registers must allow (0: no bound).  The
// 256-point passes (16 threads per pencil, 16 pencils or columns per CTA) take ~50-52
// registers unbounded - four CTAs per SM by registers; bounded to five (48 registers,
// no spills) they keep more loads in flight.  So do the row passes (the z pass) of these
// mixed-radix lengths (48-63 registers unbounded, none spilling at 48): z pass of
// 512 x 512 x n, bounded / unbounded time: 270 0.85, 288 0.88, 300 0.87, 324 0.97, 375 0.94,
// 400 0.95, 432 0.94, 480 0.96 (320 and 384 unchanged; 360, 405, 450, 486, 500 spill at 48).
// The bound applies to both layouts' 256-thread kernels of these lengths; their column
// kernels take their own bounds (croft_col_minb, croft_col_narrow_minb).
CROFT_HD constexpr int croft_pass_minb(int n, int es) {
    return (es == 8 && (n == 256 || n == 270 || n == 288 || n == 300 || n == 324 || n == 375 || n == 400 || n == 432 || n == 480)) ? 5 : 0;
}

// Column-tile width of the fused convolution pass: the same as a COL pass (8 columns
// measured slower at every size from 384 to 512: 480^3 774 vs 690 us).
CROFT_HD constexpr int croft_conv_width(int n, int es) { return croft_col_width(n, es); }

// Whether a column pass of a length-n axis whose elements lie stride_bytes apart runs the
// tensor-copy ring kernel (croft_ring_kernel.cuh) by default: never so far.  Measured per pass
// against the plain kernels (CUDA events, L2 flushed): x pass 512^3 0.487 vs 0.488 ms, 480^3
// 0.435 vs 0.348, 384x360x320 0.250 vs 0.127, 320^3 0.119 vs 0.123; y pass 512^3 0.479 vs
// 0.399 (the narrow tile).  CROFT_RING=1 selects it for every column pass it can serve.
CROFT_HD constexpr bool croft_ring_default(int n, int es, long long stride_bytes) {
    return false && es == 8 && croft_threads_per_pencil(n) == 32 && stride_bytes > 16 * 1024;
}

// Whether a column pass runs the cluster-pair kernel (croft_pair_kernel.cuh) by default: the
// 512-point axes whose elements lie at least 256 KB apart (the x pass of grids well beyond the
// L2), where each half of the pair is a 256-point column transform (16 x 16, the best-tuned
// half).  Per-pass CUDA events, plain vs pair, ms: 512^3 x 0.488 / 0.425, 512x512x256 x 0.245 /
// 0.217, 512x256x256 x 0.125 / 0.112; it loses below that stride (512x128x128 x 0.029 / 0.032),
// on the 4 KB-stride y pass (512^3 y 0.400 / 0.407) and for the other even lengths (480^3 x
// 0.348 / 0.363, 384x360x320 x 0.127 / 0.168), where the tuner can still pick it.
// Also, from a sweep of every length (per-pass events, pair vs the rules' kernel, y pass of
// 512 x n x 512 / x pass of n x 512 x 512, us): 486 at any stride (483 / 553, 500 / 633; its
// plain kernel spills), 500 across 256 KB or more (549 / 629; y 532 / 516).
CROFT_HD constexpr bool croft_pair_default(int n, int es, long long stride_bytes) {
    return es == 8 && ((n == 512 && stride_bytes >= 256 * 1024) || n == 486 ||
                       (n == 500 && stride_bytes >= 256 * 1024));
}
// Whether a column pass takes 16 threads per pencil (32 points each, the 16-column tile in
// 256-thread CTAs) by default: 432 and 480 across 256 KB or more (x pass of n x 512 x 512:
// 354 / 371 and 389 / 395 us against 32 threads).
CROFT_HD constexpr bool croft_col_t16(int n, int es, long long stride_bytes) {
    return es == 8 && (n == 432 || n == 480) && stride_bytes >= 256 * 1024;
}
