// croft_batched_kernel.cuh - many independent 3D grids of uneven sizes in one
// persistent launch.
//
// Paper mapping: the paper transforms one grid with a fixed plan; its "option 4"
// (Sec. 5.1) is a single plan that covers many 1D FFTs at once, and its chunk
// parameter K (Sec. 5.1) trades chunk size against the number of calls.  Here
// one launch covers every pencil of every pass of every grid of a batch (e.g.
// the per-system PME meshes of an MD ensemble): the work list holds one item per
// tile (W pencils of one axis of one grid), ordered pass by pass (all z tiles,
// then all y tiles, then all x tiles), and resident CTAs pull items from a
// single atomic counter, so uneven grids balance themselves.
//
// Dependencies: the y tiles of grid g need every z tile of g finished (and the
// x tiles every y tile).  The CTA that finishes a tile bumps done[g][pass]
// after a device-scope fence; a CTA holding a dependent item waits for the
// count with a bounded spin (clock64 budget, nanosleep back-off).  Items are
// dequeued in pass order, so whatever an item waits for was dequeued earlier by
// a running CTA that never waits on a later item: the wait always ends unless
// the budget runs out, in which case the CTA records CROFT_ERR_TIMEOUT in the
// status word, stops waiting (every later wait returns at once) and the host
// reads the status (croft_plan_last_device_status).  Data written by another
// CTA in the same launch is read through L2 only (ld.global.cg).
#pragma once
#include "croft_fft_core.cuh"
#include "croft_internal.h"

namespace croft {

#define CROFT_BATCH_THREADS 256
#define CROFT_BATCH_MAX_N 128

struct BatchGrid {
    const float2* in;
    float2* out;
    long long M[3];     // element stride of the pass's axis (pass 0 = z, 1 = y, 2 = x)
    long long ncols[3]; // pencils of the pass
    int n[3];           // FFT length of the pass (1 = pass skipped)
    int W[3];           // pencils per tile
    int ntiles[3];      // tiles of the pass (0 when skipped)
    int dep[3];         // pass this pass waits for (-1: none)
    int first_pass;     // first pass that runs (reads `in`; later passes read `out`)
    int tw_off[3];      // offset of the axis' twiddle table in the pool
    CroftColDiv cdiv[3];  // col / M[pass] as a multiply-high (croft_coldiv.h; m = 0: divide)
};

struct BatchItem {
    int grid;
    int pass;
    int tile;
    int pad;
};

struct BatchArgs {
    const BatchGrid* grids;
    const BatchItem* items;
    const float2* tw_pool;
    int* queue;           // work counter of this launch
    int* done;            // [count][3] finished tiles
    int* status;          // CROFT_OK / CROFT_ERR_TIMEOUT
    long long wait_cycles;
    int item_begin;       // this launch serves items [item_begin, item_end)
    int item_end;
    int extra_wait;       // test hook: grid 0's pass-1 items wait for one tile more than exists
    int direct;           // 1: one CTA per item (item = item_begin + blockIdx.x), no counters, no waits
    float isign;
};

typedef void (*batch_tile_fn)(const BatchGrid&, int pass, int tile, const float2* tw, float2* smem, float isign);

// One tile = W pencils of one pass of one grid, processed by the whole CTA.
template <int LAYOUT, int N>
__device__ __noinline__ void batch_tile(const BatchGrid& G, int pass, int tile, const float2* twg, float2* smem,
                                        float isign) {
    constexpr int T = croft_threads_per_pencil(N);
    float2* stw = smem;
    float2* sbuf = smem + ((CROFT_BATCH_MAX_N + 1) / 2) * 2;
    const int W = G.W[pass];
    if (croft_make_sched(N).count > 1)
        for (int i = threadIdx.x; i < N - 1; i += blockDim.x) stw[i] = __ldg(twg + i);
    const float2* in = (pass == G.first_pass) ? G.in : G.out;
    float2* out = G.out;
    if (LAYOUT == LAYOUT_ROW) {
        const int c = threadIdx.x / T;
        const int lane = threadIdx.x - c * T;
        const long long col = (long long)tile * W + c;
        const bool ok = c < W && col < G.ncols[pass];
        const long long base = (ok ? col : 0) * N;
        fft_pencil_row<N, T>(GlobalInCG{in + base, 1, isign}, sbuf + (ok ? c : 0) * croft_row_ld_staged(N),
                             GlobalOutUnit{out + base, isign}, stw, lane, ok);
    } else {
        const long long M = G.M[pass];
        const int c = threadIdx.x % W;
        const int lane = threadIdx.x / W;
        const long long col = (long long)tile * W + c;
        const bool ok = lane < T && col < G.ncols[pass];
        const long long cc = ok ? col : 0;
        const CroftColDiv dv = G.cdiv[pass];
        long long b, m;
        if (dv.m) {
            const unsigned q = croft_coldiv_q(dv.m, dv.s1, dv.s2, (unsigned)cc);
            b = q;
            m = (unsigned)cc - q * (unsigned)M;
        } else {
            b = cc / M;
            m = cc - b * M;
        }
        const long long base = b * (long long)N * M + m;
        fft_pencil<N, T>(GlobalInCG{in + base, M, isign}, SmemCol{sbuf + c, W},
                         GlobalOut{out + base, M, isign}, stw, lane, ok);
    }
}

}  // namespace croft
