// croft_pair_kernel.cuh - column pass of an even length N by a pair of CTAs (a 2-CTA
// thread-block cluster) sharing one 16-column tile.
//
// Paper mapping: the same batched 1D FFT pass of Sec. 4.1 (steps 5, 9) with the
// rearrangement fused into the gather; inside the pencil it is one radix-2
// decimation-in-time step over two half-length transforms (the split the paper's
// 1D FFTs, FFTW's, are built from):
//     X[k]       = E[k] + w_N^k O[k],   X[k + N/2] = E[k] - w_N^k O[k],   k < N/2,
// with E = DFT_{N/2} of the even-indexed points and O of the odd-indexed ones.
//
// Why a pair: a 16-column tile (128-byte rows, the smallest piece the strided x pass
// can fetch at full HBM rate) of a 270..512-point axis needs 512 threads at 32 threads
// per pencil, and three such CTAs per SM only fit in 40 registers.  Split over two
// CTAs, each holds half the rows (N/2 x 16, 16 threads per pencil, 256 threads) - the
// shape of the 256-point passes, which run five CTAs per SM without spills:
//  * CTA r (its rank in the cluster) loads rows r, r + 2, r + 4, ... (full 128-byte
//    lines; the pair together reads every row of the tile once) and transforms them
//    with the half-length schedule in shared memory;
//  * a cluster barrier; then CTA r combines the outputs k of its half of [0, N/2)
//    (E from CTA 0's shared memory, O from CTA 1's, one of them read through
//    distributed shared memory) and writes rows k and k + N/2 (full lines) to HBM;
//  * a second cluster barrier (a relaxed arrive: it orders no memory) keeps each CTA's
//    shared memory alive until its partner has read it.
// The waits are cluster barriers between two co-scheduled CTAs of one launch.
#pragma once
#include <cooperative_groups.h>

#include "croft_fft_core.cuh"
#include "croft_internal.h"

namespace croft {

constexpr int kPairWidth = kPairTileWidth;  // columns per tile

// Threads of one CTA of a pair: 16 columns x the half length's threads per pencil.
template <int N>
__host__ __device__ constexpr int pair_threads() {
    return kPairWidth * croft_threads_per_pencil(N / 2);
}

// Shared memory (dynamic): [half-length twiddles: tw_pad][combine twiddles: N/2, rounded up to
// even][tile: N/2 x 16].
// A.tw: the half-length table (N/2 - 1 entries, its column schedule); A.tw2: w_N^k, k < N/2.
template <int N>
__global__ void __launch_bounds__(pair_threads<N>(), 5)
    croft_pair_kernel(const float2* in, float2* out, const __grid_constant__ PassArgs A) {
    static_assert(N % 2 == 0, "the pair kernel splits an even length");
    constexpr int N2 = N / 2;
    constexpr int T = croft_threads_per_pencil(N2);
    constexpr int W = kPairWidth;
    using S = typename std::conditional<croft_even_pow2_pass(N2, LAYOUT_COL, 8), EvenPow2Sched<N2>,
                                        DefaultSched<N2>>::type;
    constexpr CroftSched sc = S::get();
    namespace cg = cooperative_groups;
    const cg::cluster_group cluster = cg::this_cluster();
    const int r = (int)cluster.block_rank();

    extern __shared__ __align__(16) float2 pair_smem[];
    float2* stw = pair_smem;
    float2* ctw = pair_smem + A.tw_pad;
    float2* tile = ctw + (N2 + (N2 & 1));  // (keeps the tile 16-byte aligned)
    const int tid = threadIdx.x;
    pdl_allow_dependents();
    if (sc.count > 1)
        for (int i = tid; i < N2 - 1; i += blockDim.x) stw[i] = A.tw[i];
    for (int i = tid; i < N2; i += blockDim.x) ctw[i] = A.tw2[i];
    pdl_wait();

    const int c = tid % W;
    const int lane = tid / W;
    const long long col = (long long)(blockIdx.x / 2) * W + c;
    const bool ok = col < A.ncols;
    long long b, m;
    col_split(col, A, b, m);
    const long long base = b * (long long)N * A.M + m;

    // the half-length transform of rows r, r + 2, ... into the tile, natural order
    const GlobalInT<float2> src{in + base + (long long)r * A.M, 2 * A.M, A.isign};
    const SmemColFixed<float2, W> work{tile + c};
    if constexpr (sc.count == 1) {
        fft_stage_s<S, 0, T>(src, NoBarrier{}, work, stw, lane, ok);
    } else {
        fft_stage_s<S, 0, T>(src, NoBarrier{}, work, stw, lane, ok);
        __syncthreads();
        smem_stages_s<S, 1, sc.count - 1, T>(work, stw, lane, ok);
        fft_stage_s<S, sc.count - 1, T>(work, CtaBarrier{}, work, stw, lane, ok);
    }
    cluster.sync();  // both halves transformed and visible across the pair

    // radix-2 combination of outputs k in this CTA's half of [0, N/2)
    const float2* mine = tile;
    const float2* peer = cluster.map_shared_rank(tile, r ^ 1);
    const float2* E = r == 0 ? mine : peer;
    const float2* O = r == 0 ? peer : mine;
    constexpr int KH = (N2 + 1) / 2;
    const int k0 = r * KH;
    const int k1 = (k0 + KH < N2) ? k0 + KH : N2;
    const GlobalOutT<float2> dst{out + base, A.M, A.isign};
    if (ok)
        for (int k = k0 + lane; k < k1; k += T) {
            const float2 e = E[k * W + c];
            const float2 t = cmul(O[k * W + c], ctw[k]);
            dst.store(k, cadd(e, t));
            dst.store(k + N2, csub(e, t));
        }
    // The partner has finished reading this CTA's tile: every value it read feeds a store it
    // issued before arriving, so a relaxed arrive suffices (a release would wait for this
    // CTA's global stores to be performed).
    asm volatile("barrier.cluster.arrive.relaxed.aligned;\n\tbarrier.cluster.wait.aligned;" ::: "memory");
}

}  // namespace croft
