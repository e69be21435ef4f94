// croft_pass_kernel.cuh - one pass = a batched 1D FFT over all pencils of one axis.
//
// Paper mapping (Sec. 4.1): steps 1, 5 and 9 are the per-axis batched 1D FFTs;
// steps 2-4 and 6-8 (pack, all-to-all, unpack) only exist to make the next
// axis local to a process.  On one GPU every axis is addressable, so the
// rearrangement is fused into the FFT pass itself: a CTA gathers W whole
// pencils of a strided axis straight from HBM (W consecutive columns, i.e.
// W*8-byte contiguous row segments), transforms them on chip and writes them
// back to the same place.  The grid therefore stays in its natural layout
// between passes and after the last one (the paper's closing transposes,
// Sec. 4.2, are not needed).
//
// Inside a CTA each pencil is transformed with the Stockham auto-sort
// formulation: stage s with radix R combines R sub-transforms of length p
// into one of length pR.  Butterfly b (0 <= b < n/R), k = b mod p, reads
// x[b + j*n/R] (j = 0..R-1), multiplies input j by w_{pR}^{jk}, applies the
// radix-R DFT and writes output j to y[(b-k)*R + k + j*p].  The first stage
// reads HBM straight into registers and the last stage writes HBM straight
// from registers (unit-stride lanes in both cases); the stages in between
// exchange through shared memory in place.  Kernels are specialised on n, so
// the radix schedule, strides and twiddle offsets are compile-time constants.
#pragma once
#include "croft_butterflies.cuh"
#include "croft_internal.h"
#include "croft_sched.h"

namespace croft {

template <int N>
struct RowLd {
    static constexpr int value = N + (N - 1) / 16 + 1;  // one pad slot per 16 elements
};

template <int LAYOUT, int N>
__device__ __forceinline__ int smem_idx(int c, int a, int W) {
    if (LAYOUT == LAYOUT_ROW) return c * RowLd<N>::value + a + (a >> 4);  // conflict-free strided writes
    return a * W + c;  // W pencils side by side; W is a multiple of 16 so a warp row spans all banks
}

template <int N, int LAYOUT, int S>
__device__ __forceinline__ void stage_ct(const float2* gin, float2* gout, float2* sbuf, const float2* stw,
                                         const PassArgs& A, int lane, int c, bool ok) {
    constexpr CroftSched sc = croft_make_sched(N);
    constexpr int R = sc.r[S];
    constexpr int P = croft_sched_p(sc, S);
    constexpr int NB = N / R;
    constexpr int T = croft_threads_per_pencil(N);
    constexpr int QM = (NB + T - 1) / T;
    constexpr bool kFromGlobal = (S == 0);
    constexpr bool kToGlobal = (S == sc.count - 1);

    float2 v[QM][R];
#pragma unroll
    for (int q = 0; q < QM; ++q) {
        const int b = lane + q * T;
        if (ok && (NB % T == 0 || b < NB)) {
            if (kFromGlobal) {
                if (LAYOUT == LAYOUT_ROW) {
#pragma unroll
                    for (int j = 0; j < R; ++j) {
                        float2 t = gin[b + j * NB];
                        t.y *= A.isign;
                        v[q][j] = t;
                    }
                } else {
                    const float2* src = gin + (long long)b * A.M;
                    const long long step = (long long)NB * A.M;
#pragma unroll
                    for (int j = 0; j < R; ++j) {
                        float2 t = src[j * step];
                        t.y *= A.isign;
                        v[q][j] = t;
                    }
                }
            } else {
#pragma unroll
                for (int j = 0; j < R; ++j) v[q][j] = sbuf[smem_idx<LAYOUT, N>(c, b + j * NB, A.W)];
            }
        }
    }
    if (!kFromGlobal) __syncthreads();  // every read of this stage precedes any in-place write
#pragma unroll
    for (int q = 0; q < QM; ++q) {
        const int b = lane + q * T;
        if (ok && (NB % T == 0 || b < NB)) {
            const int k = (P == 1) ? 0 : b % P;
            if (P > 1) {
                const float2* w = stw + (P - 1) + k;
#pragma unroll
                for (int j = 1; j < R; ++j) v[q][j] = cmul(v[q][j], w[(j - 1) * P]);
            }
            dft<R>(v[q]);
            const int o = (b - k) * R + k;
            if (kToGlobal) {
                if (LAYOUT == LAYOUT_ROW) {
#pragma unroll
                    for (int j = 0; j < R; ++j) {
                        float2 t = v[q][j];
                        t.y *= A.isign;
                        gout[o + j * P] = t;
                    }
                } else {
                    float2* dst = gout + (long long)o * A.M;
                    const long long step = (long long)P * A.M;
#pragma unroll
                    for (int j = 0; j < R; ++j) {
                        float2 t = v[q][j];
                        t.y *= A.isign;
                        dst[j * step] = t;
                    }
                }
            } else {
#pragma unroll
                for (int j = 0; j < R; ++j) sbuf[smem_idx<LAYOUT, N>(c, o + j * P, A.W)] = v[q][j];
            }
        }
    }
    if (!kToGlobal) __syncthreads();
    if constexpr (S + 1 < sc.count) stage_ct<N, LAYOUT, S + 1>(gin, gout, sbuf, stw, A, lane, c, ok);
}

// Shared memory: [twiddles: tw_pad float2][tile: W pencils].
template <int LAYOUT, int N>
__global__ void __launch_bounds__(512) croft_pass_kernel(const float2* in, float2* out,
                                                          const __grid_constant__ PassArgs A) {
    constexpr int T = croft_threads_per_pencil(N);
    extern __shared__ float2 smem[];
    float2* stw = smem;
    float2* sbuf = smem + A.tw_pad;
    if (croft_make_sched(N).count > 1)
        for (int i = threadIdx.x; i < N - 1; i += blockDim.x) stw[i] = A.tw[i];

    int lane, c;
    if (LAYOUT == LAYOUT_ROW) {
        c = threadIdx.x / T;
        lane = threadIdx.x - c * T;
    } else {
        c = threadIdx.x % A.W;
        lane = threadIdx.x / A.W;
    }
    const long long col = (long long)blockIdx.x * A.W + c;
    const bool ok = col < A.ncols;
    long long base;
    if (LAYOUT == LAYOUT_ROW) {
        base = col * N;
    } else {
        const long long b = col / A.M;
        const long long m = col - b * A.M;
        base = b * (long long)N * A.M + m;
    }
    stage_ct<N, LAYOUT, 0>(in + base, out + base, sbuf, stw, A, lane, c, ok);
}

}  // namespace croft
