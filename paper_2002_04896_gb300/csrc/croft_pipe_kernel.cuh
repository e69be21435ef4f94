// croft_pipe_kernel.cuh - persistent pass kernel with the HBM loads on the TMA engine.
//
// Same pass as croft_pass_kernel (one batched 1D FFT over every pencil of one
// axis, the rearrangement between axes fused into the gather), organised for
// Blackwell: each CTA is persistent and walks its share of the tiles; the tile
// after the current one is already being copied HBM -> shared memory by the
// tensor memory accelerator (a 1D bulk copy for the contiguous z axis, 3D
// tensor-map boxes of W adjacent columns for the strided y / x axes) while the
// threads transform the current tile.  Completion is tracked by an mbarrier
// per buffer (expected transaction bytes).  No thread holds load data in
// registers while waiting for HBM, so memory latency is hidden by the copy in
// flight rather than by occupancy.  The last Stockham stage writes the result
// straight from registers to HBM (coalesced rows), as in the plain kernel.
//
// Buffer reuse: after a tile's last stage has read its buffer, the CTA
// synchronises, orders its shared-memory accesses before the async proxy
// (fence.proxy.async) and only then issues the copy of tile i + 2 into that
// buffer.  Every wait on an mbarrier is bounded.
#pragma once
#include <cuda.h>

#include "croft_fft_core.cuh"
#include "croft_internal.h"

namespace croft {

// Dense pencil c of a ROW tile as written by the bulk copy; conj on read when isign = -1.
struct SmemDenseIn {
    using value_type = float2;
    const float2* s;
    float isign;
    __device__ __forceinline__ float2 load(int a) const {
        float2 t = s[a];
        t.y *= isign;
        return t;
    }
};
struct SmemColIn {
    using value_type = float2;
    const float2* s;
    int W;
    float isign;
    __device__ __forceinline__ float2 load(int a) const {
        float2 t = s[a * W];
        t.y *= isign;
        return t;
    }
};

__device__ __forceinline__ uint32_t pipe_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool pipe_wait(uint32_t mbar, uint32_t parity) {
    uint32_t done = 0;
    for (long it = 0; it < (1L << 28) && !done; ++it) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
    }
    return done != 0;
}

// Issue the copy of tile t into buffer `buf` (thread 0 only).
template <int LAYOUT, int N>
__device__ __forceinline__ void pipe_issue(const PipeArgs& A, const CUtensorMap* tmap, const float2* in, long long t,
                                           float2* buf, uint32_t mbar) {
    const uint32_t dst = pipe_smem(buf);
    if (LAYOUT == LAYOUT_ROW) {
        const long long first = t * A.W;
        const long long cnt = (A.ncols - first < A.W) ? (A.ncols - first) : A.W;
        const uint32_t bytes = (uint32_t)(cnt * N * sizeof(float2));
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
            "l"(in + first * N), "r"(bytes), "r"(mbar)
            : "memory");
    } else {
        const long long b = t / A.tiles_per_row;
        const int m0 = (int)((t - b * A.tiles_per_row) * A.W);
        const uint32_t bytes = (uint32_t)(N * A.W * sizeof(float2));
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
        for (int r0 = 0; r0 < N; r0 += A.box_rows) {
            asm volatile(
                "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
                "%4}], [%5];" ::"r"(dst + (uint32_t)(r0 * A.W * sizeof(float2))),
                "l"(tmap), "r"(m0), "r"(r0), "r"((int)b), "r"(mbar)
                : "memory");
        }
    }
}

// Transform the tile held in `buf` and store it (whole CTA).  Kept out of line:
// inlined into the tile loop, the stage code of the longer schedules overwhelmed
// the register allocator (32 registers and heavy spilling).
template <int LAYOUT, int N>
__device__ __noinline__ void pipe_tile(float2* buf, float2* out, const PipeArgs& A, long long t, int c, int lane,
                                       const float2* stw) {
    constexpr int T = croft_threads_per_pencil(N);
    constexpr CroftSched sc = croft_make_sched(N);
    if (LAYOUT == LAYOUT_ROW) {
        const long long col = t * A.W + c;
        const bool ok = (c < A.W) && col < A.ncols;
        const long long base = (ok ? col : 0) * N;
        const SmemDenseIn src{buf + c * N, A.isign};
        const SmemRow work{buf + c * row_ld(N)};
        const GlobalOutUnit dst{out + base, A.isign};
        if constexpr (sc.count == 1) {
            fft_stage<N, 0, T>(src, NoBarrier{}, dst, stw, lane, ok);
        } else {
            fft_stage<N, 0, T>(src, CtaBarrier{}, work, stw, lane, ok);
            __syncthreads();
            smem_stages<N, 1, sc.count - 1, T>(work, stw, lane, ok);
            fft_stage<N, sc.count - 1, T>(work, NoBarrier{}, dst, stw, lane, ok);
        }
    } else {
        const long long b = t / A.tiles_per_row;
        const long long m = (t - b * A.tiles_per_row) * A.W + c;
        const bool ok = (lane < T) && m < A.M;
        const long long base = b * (long long)N * A.M + (ok ? m : 0);
        const SmemColIn src{buf + c, A.W, A.isign};
        const SmemCol work{buf + c, A.W};
        const GlobalOut dst{out + base, A.M, A.isign};
        if constexpr (sc.count == 1) {
            fft_stage<N, 0, T>(src, NoBarrier{}, dst, stw, lane, ok);
        } else {
            fft_stage<N, 0, T>(src, CtaBarrier{}, work, stw, lane, ok);
            __syncthreads();
            smem_stages<N, 1, sc.count - 1, T>(work, stw, lane, ok);
            fft_stage<N, sc.count - 1, T>(work, NoBarrier{}, dst, stw, lane, ok);
        }
    }
}

// Shared memory: [twiddles: tw_pad float2][buffer 0][buffer 1].
template <int LAYOUT, int N>
__global__ void __launch_bounds__(512) croft_pipe_kernel(const float2* in, float2* out, const __grid_constant__ PipeArgs A,
                                                          const __grid_constant__ CUtensorMap tmap) {
    constexpr int T = croft_threads_per_pencil(N);
    extern __shared__ __align__(128) float2 smem[];
    __shared__ __align__(8) uint64_t full[2];
    float2* stw = smem;
    float2* bufs[2] = {smem + A.tw_pad, smem + A.tw_pad + A.buf_elems};
    const int tid = threadIdx.x;
    const long long G = gridDim.x;
    const long long my_tiles = (A.ntiles - blockIdx.x + G - 1) / G;

    for (int i = tid; i < N - 1; i += blockDim.x) stw[i] = A.tw[i];
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(pipe_smem(&full[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(pipe_smem(&full[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
        for (int k = 0; k < 2 && k < my_tiles; ++k)
            pipe_issue<LAYOUT, N>(A, &tmap, in, blockIdx.x + k * G, bufs[k], pipe_smem(&full[k]));
    }
    __syncthreads();

    int c, lane;
    if (LAYOUT == LAYOUT_ROW) {
        c = tid / T;
        lane = tid - c * T;
    } else {
        c = tid % A.W;
        lane = tid / A.W;
    }
    for (long long i = 0; i < my_tiles; ++i) {
        const long long t = blockIdx.x + i * G;
        const int bsel = (int)(i & 1);
        float2* buf = bufs[bsel];
        pipe_wait(pipe_smem(&full[bsel]), (uint32_t)((i >> 1) & 1));
        pipe_tile<LAYOUT, N>(buf, out, A, t, c, lane, stw);
        __syncthreads();  // every read of this buffer done
        if (tid == 0 && i + 2 < my_tiles) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            pipe_issue<LAYOUT, N>(A, &tmap, in, t + 2 * G, buf, pipe_smem(&full[bsel]));
        }
    }
}

}  // namespace croft
