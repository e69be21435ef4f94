// croft_batched.cu - the persistent batched kernel and its launch (see croft_batched_kernel.cuh).
#include <cuda/atomic>

#include "croft_batched_kernel.cuh"
#include "croft_sizes.h"

namespace croft {


bool batch_size_supported(int n) {
    switch (n) {
#define CROFT_B_CASE(N) case N:
        CROFT_BATCH_SIZES(CROFT_B_CASE)
#undef CROFT_B_CASE
        return true;
        default: return false;
    }
}

// One indirect call site into per-size tile functions: a switch over inlined
// bodies overwhelms the register allocator, and a switch over direct calls
// gives the kernel a stack frame per call site.
__device__ batch_tile_fn g_tile_fns[2][CROFT_BATCH_MAX_N + 1] = {
#define CROFT_B_ROW(N) [N] = batch_tile<LAYOUT_ROW, N>,
    {CROFT_BATCH_SIZES(CROFT_B_ROW)},
#undef CROFT_B_ROW
#define CROFT_B_COL(N) [N] = batch_tile<LAYOUT_COL, N>,
    {CROFT_BATCH_SIZES(CROFT_B_COL)},
#undef CROFT_B_COL
};

__device__ __forceinline__ void run_tile(const BatchGrid& G, int pass, int tile, const float2* tw, float2* smem,
                                         float isign) {
    const int n = G.n[pass];
    const int col = (pass == 0 || G.M[pass] == 1) ? 0 : 1;
    const batch_tile_fn f = (n >= 2 && n <= CROFT_BATCH_MAX_N) ? g_tile_fns[col][n] : nullptr;
    if (f) f(G, pass, tile, tw, smem, isign);
}

// Bounded wait until *counter >= target (thread 0 only).  Returns false on timeout
// (status set) or when another CTA already timed out.
__device__ bool wait_count(const int* counter, int target, int* status, long long budget) {
    cuda::atomic_ref<int, cuda::thread_scope_device> c(*const_cast<int*>(counter));
    cuda::atomic_ref<int, cuda::thread_scope_device> st(*status);
    if (c.load(cuda::memory_order_acquire) >= target) return true;
    const long long t0 = clock64();
    unsigned ns = 32;
    while (true) {
        if (c.load(cuda::memory_order_acquire) >= target) return true;
        if (st.load(cuda::memory_order_relaxed) != 0) return false;
        if (clock64() - t0 > budget) {
            st.store(5 /* CROFT_ERR_TIMEOUT */, cuda::memory_order_relaxed);
            return false;
        }
        __nanosleep(ns);
        if (ns < 1024) ns *= 2;
    }
}

__global__ void __launch_bounds__(CROFT_BATCH_THREADS, 3) croft_batched_kernel(const __grid_constant__ BatchArgs A) {
    extern __shared__ float2 smem[];
    __shared__ int s_item;
    __shared__ int s_ok;
    if (A.direct) {  // kernel boundaries order the passes: nothing to count or wait for
        const int it = A.item_begin + blockIdx.x;
        if (it >= A.item_end) return;
        const BatchItem w = A.items[it];
        const BatchGrid& G = A.grids[w.grid];
        run_tile(G, w.pass, w.tile, A.tw_pool + G.tw_off[w.pass], smem, A.isign);
        return;
    }
    for (;;) {
        if (threadIdx.x == 0) s_item = A.item_begin + atomicAdd(A.queue, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= A.item_end) break;
        const BatchItem w = A.items[it];
        const BatchGrid& G = A.grids[w.grid];
        if (threadIdx.x == 0) {
            int ok = 1;
            const int d = G.dep[w.pass];
            if (d >= 0) {
                const int target = G.ntiles[d] + ((A.extra_wait && w.grid == 0 && w.pass == 1) ? 1 : 0);
                ok = wait_count(A.done + 3 * w.grid + d, target, A.status, A.wait_cycles) ? 1 : 0;
            }
            s_ok = ok;
        }
        __syncthreads();
        if (s_ok) run_tile(G, w.pass, w.tile, A.tw_pool + G.tw_off[w.pass], smem, A.isign);
        __syncthreads();  // every store of the tile issued; s_item / s_ok free for the next item
        if (threadIdx.x == 0) {
            __threadfence();
            cuda::atomic_ref<int, cuda::thread_scope_device> c(A.done[3 * w.grid + w.pass]);
            c.fetch_add(1, cuda::memory_order_release);
        }
    }
}

// COL tiles: as many adjacent columns as the CTA's threads allow, a multiple of 16.
int batch_col_width(int n) {
    const int T = croft_threads_per_pencil(n);
    int W = CROFT_BATCH_THREADS / T;
    if (W >= 16) W -= W % 16;
    return W;
}

int batch_smem_bytes() {
    int best = 0;
    const int tw = ((CROFT_BATCH_MAX_N + 1) / 2) * 2;
#define CROFT_B_SMEM(N)                                                                            \
    {                                                                                              \
        const int T = croft_threads_per_pencil(N);                                                 \
        const int Wr = CROFT_BATCH_THREADS / T;                                                    \
        const int Wc = batch_col_width(N);                                                         \
        int a = Wr * croft_row_ld_staged(N), b = N * Wc;                                           \
        int m = (a > b ? a : b) + tw;                                                              \
        if (m > best) best = m;                                                                    \
    }
    CROFT_BATCH_SIZES(CROFT_B_SMEM)
#undef CROFT_B_SMEM
    return best * 8;
}

cudaError_t batched_prepare(int smem) {
    if (smem <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(croft_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

int batched_blocks_per_sm(int smem) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, croft_batched_kernel, CROFT_BATCH_THREADS, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

void* batched_kernel_ptr() { return (void*)croft_batched_kernel; }

cudaError_t launch_batched(const BatchArgs& A, int blocks, int smem, cudaStream_t s) {
    croft_batched_kernel<<<blocks, CROFT_BATCH_THREADS, smem, s>>>(A);
    return cudaGetLastError();
}

}  // namespace croft
