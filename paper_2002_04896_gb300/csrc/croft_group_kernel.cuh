// croft_group_kernel.cuh - one pass over the pencils of many grids that share
// the axis length N (the grouped schedule of batched plans).
//
// A batch of uneven grids has few distinct axis lengths.  The grouped schedule
// launches, for each pass and each length N, one kernel over the tiles of every
// grid whose axis of that pass has length N; the launches of one pass are
// independent and run concurrently (sibling nodes of a CUDA graph).  Each kernel
// is the single-grid pass kernel specialised on N (compile-time radix schedule
// and tile width) with a per-CTA lookup of its grid: CTA b works on tile
// b - first_tile of segment cta_seg[b].
#pragma once
#include "croft_fft_core.cuh"
#include "croft_internal.h"

namespace croft {

struct GroupSeg {
    const float2* in;   // pass input of this grid (the exec's `in` for the grid's first pass)
    float2* out;
    long long M;        // element stride of the axis (1 for a ROW pass)
    long long ncols;    // pencils of this grid along the axis
    int first_tile;     // first CTA of this grid in the launch
    CroftColDiv cdiv;   // COL: col / M as a multiply-high (croft_coldiv.h; m = 0: divide)
};

struct GroupArgs {
    const GroupSeg* segs;           // this launch's segments (device table, pointers filled per exec)
    const unsigned short* cta_seg;  // segment of each CTA
    const float2* tw;               // twiddle table of N (N-1 entries)
    int W;                          // ROW: pencils per CTA
    float isign;                    // +1 forward, -1 backward
};

// ROW launches: W = 256 / T pencils per CTA; COL launches: the compile-time width
// croft_col_width(N).
template <int LAYOUT, int N>
__global__ void __launch_bounds__(256) croft_group_kernel(const __grid_constant__ GroupArgs A) {
    constexpr int T = croft_threads_per_pencil(N);
    constexpr int TW_PAD = ((N + 1) / 2) * 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* stw = reinterpret_cast<float2*>(smem_raw);
    float2* sbuf = stw + TW_PAD;
    pdl_allow_dependents();
    if (croft_make_sched(N).count > 1)
        for (int i = threadIdx.x; i < N - 1; i += blockDim.x) stw[i] = A.tw[i];
    // (the segment table is uploaded before the first pass starts; the grid is written by
    // the previous pass, whose launches reach this one over programmatic graph edges)
    const GroupSeg S = A.segs[A.cta_seg[blockIdx.x]];
    const long long tile = (long long)blockIdx.x - S.first_tile;
    pdl_wait();
    if constexpr (LAYOUT == LAYOUT_ROW) {
        const int c = threadIdx.x / T;
        const int lane = threadIdx.x - c * T;
        const long long col = tile * A.W + c;
        const bool ok = col < S.ncols;
        const long long base = col * N;
        fft_pencil_row<N, T>(GlobalInUnit{S.in + base, A.isign}, sbuf + c * croft_row_ld_staged(N),
                             GlobalOutUnit{S.out + base, A.isign}, stw, lane, ok);
    } else {
        constexpr int WC = croft_col_width(N, 8);
        const int c = threadIdx.x % WC;
        const int lane = threadIdx.x / WC;
        const long long col = tile * WC + c;
        const bool ok = col < S.ncols;
        long long b, m;
        if (S.cdiv.m) {
            const unsigned q = croft_coldiv_q(S.cdiv.m, S.cdiv.s1, S.cdiv.s2, (unsigned)col);
            b = q;
            m = (unsigned)col - q * (unsigned)S.M;
        } else {
            b = col / S.M;
            m = col - b * S.M;
        }
        const long long base = b * (long long)N * S.M + m;
        fft_pencil<N, T>(GlobalIn{S.in + base, S.M, A.isign}, SmemColFixed<float2, WC>{sbuf + c},
                         GlobalOut{S.out + base, S.M, A.isign}, stw, lane, ok);
    }
}

}  // namespace croft
