// croft_ring_kernel.cuh - column pass with the HBM loads on the tensor memory
// accelerator, fed through a ring of tile buffers to two independent consumer
// groups (the strided y / x passes of 32-thread pencils: lengths 270..512).
//
// Paper mapping: the pass is the same batched 1D FFT of Sec. 4.1 (steps 5 and 9)
// with the all-to-all of steps 2-4 / 6-8 fused into the gather of W adjacent
// columns.  The paper overlaps the exchange of one chunk with the computation on
// another (a communication thread and K chunks, Sec. 5.1); here the "exchange"
// is the strided HBM gather and the overlap is between TMA copies in flight and
// the butterflies of other tiles.
//
// Organisation (one persistent CTA per SM, 1024 threads):
//  * two consumer groups of 512 threads (16 columns x 32 threads per pencil),
//    each synchronising on its own named barrier; group g transforms the CTA's
//    tiles i = g, g + 2, g + 4, ...;
//  * a ring of three 64 KB tile buffers in shared memory; tile i lives in
//    buffer i mod 3 and is copied there by cp.async.bulk.tensor (a 3D tensor map
//    over {columns, axis, batch rows}; boxes of 16 columns = 128-byte rows),
//    completing on that buffer's mbarrier (expected transaction bytes);
//  * when a group's last stage has read buffer i mod 3 (the group barrier in the
//    middle of that stage), one of its threads orders the group's shared-memory
//    accesses before the async proxy and issues the copy of tile i + 3 into the
//    same buffer.  The copy therefore runs while both groups compute, and no
//    thread holds load data in registers while HBM answers.
//  * Every stage exchanges through the tile buffer in place (the first stage
//    reads the copied tile, the last one writes HBM straight from registers).
//
// Every mbarrier wait is bounded; the group agrees on a timeout with a barrier
// reduction (so its named barriers stay matched), records CROFT_ERR_TIMEOUT in
// the status word and leaves the tile loop; before the CTA exits it waits
// (bounded) for every copy it issued, so no copy lands in freed shared memory.
#pragma once
#include <cuda.h>

#include "croft_fft_core.cuh"
#include "croft_internal.h"

namespace croft {

constexpr int kRingBufs = 3;      // tile buffers per CTA
constexpr int kRingGroups = 2;    // consumer groups per CTA
constexpr int kRingWidth = kRingTileWidth;  // columns per tile (128-byte rows)

// Column c of a [n][16] tile written by the tensor copy; conj on read when isign = -1.
template <class C>
struct RingColIn {
    using value_type = C;
    const C* s;
    float isign;
    __device__ __forceinline__ C load(int a) const {
        C t = s[a * kRingWidth];
        t.y *= isign;
        return t;
    }
};

// Named barrier of one consumer group (ids 1 and 2; id 0 is __syncthreads).
template <int NT>
struct GroupBarrier {
    int id;
    __device__ __forceinline__ void operator()() const { asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(NT) : "memory"); }
};
// Barrier that also ORs a predicate over the group.
template <int NT>
__device__ __forceinline__ bool group_any(int id, bool p) {
    int r;
    asm volatile(
        "{\n .reg .pred q, o;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred o, %2, %3, q;\n selp.u32 %0, 1, 0, o;\n}\n"
        : "=r"(r)
        : "r"((unsigned)p), "r"(id), "n"(NT)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ uint32_t ring_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Bounded wait for phase `parity` of an mbarrier: false when it did not complete within
// about `cycles` SM clocks.
__device__ __forceinline__ bool ring_wait(uint32_t mbar, uint32_t parity, long long cycles) {
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > cycles) return false;
    }
}

// Copy tile t (16 columns x n rows of one batch row) into buffer `buf`, completing on `mbar`.
template <int N>
__device__ __forceinline__ void ring_issue(const RingArgs& A, const CUtensorMap* tmap, long long t, void* buf,
                                           uint32_t mbar) {
    const long long b = t / A.tiles_per_row;
    const int m0 = (int)((t - b * A.tiles_per_row) * kRingWidth);
    constexpr uint32_t bytes = (uint32_t)N * kRingWidth * sizeof(float2);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
    const uint32_t dst = ring_smem(buf);
#pragma unroll
    for (int r0 = 0; r0 < N; r0 += A.box_rows) {
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
            "[%5];" ::"r"(dst + (uint32_t)(r0 * kRingWidth * sizeof(float2))),
            "l"(tmap), "r"(m0), "r"(r0), "r"((int)b), "r"(mbar)
            : "memory");
    }
}

// Shared-memory layout of the ring kernel: [twiddles: tw_pad float2][pad to 128 B][tiles].
extern __shared__ __align__(128) float2 ring_smem_base[];
__device__ __forceinline__ float2* ring_bufs(int tw_pad) {
    const uint32_t sb = ring_smem(ring_smem_base + tw_pad);
    return (float2*)((char*)(ring_smem_base + tw_pad) + ((128u - (sb & 127u)) & 127u));
}

struct RingState {  // the CTA's mbarriers and copy counters (static shared memory)
    uint64_t full[kRingBufs];
    int issued[kRingBufs], consumed[kRingBufs];  // copies per buffer (timeout clean-up)
};

// Release of a tile buffer in the middle of the last stage (its Mid): every thread orders
// its own accesses to the buffer before the copy that overwrites it (async proxy), the
// group agrees the buffer is free, and one thread issues the copy of the tile three ahead.
// (Only two integers stay live through the stage; the rest is recomputed here.)
template <int N, int GT>
struct RingRelease {
    int slot_bar;  // slot * 8 + barrier id
    int next;      // tile to copy into the buffer (-1: none); negative for every thread but one
    const RingArgs* A;
    const CUtensorMap* tmap;
    RingState* st;
    __device__ __forceinline__ void operator()() const {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("bar.sync %0, %1;" ::"r"(slot_bar & 7), "n"(GT) : "memory");
        if (next >= 0) {
            const int slot = slot_bar >> 3;
            ring_issue<N>(*A, tmap, next, ring_bufs(A->tw_pad) + slot * (N * kRingWidth), ring_smem(&st->full[slot]));
            atomicAdd(&st->issued[slot], 1);
        }
    }
};

template <int N>
__global__ void __launch_bounds__(kRingGroups * kRingWidth * 32, 1)
    croft_ring_kernel(const float2* in, float2* out, const __grid_constant__ RingArgs A,
                      const __grid_constant__ CUtensorMap tmap) {
    static_assert(croft_threads_per_pencil(N) == 32, "the ring kernel serves 32-thread pencils");
    constexpr int T = 32;
    constexpr int GT = kRingWidth * T;  // threads per consumer group
    using SchedT = EvenPow2Sched<N>;
    constexpr CroftSched sc = SchedT::get();
    static_assert(sc.count >= 2 && sc.count <= 4, "two to four stages");
    __shared__ RingState st;
    float2* stw = ring_smem_base;
    constexpr int kBufElems = N * kRingWidth;

    const int tid = threadIdx.x;
    const int grp = tid / GT;          // consumer group
    const int gtid = tid - grp * GT;   // thread within the group
    const int bar_id = 1 + grp;
    const int G = gridDim.x;
    const int my_tiles = ((int)A.ntiles - (int)blockIdx.x + G - 1) / G;

    pdl_allow_dependents();
    for (int i = tid; i < N - 1; i += blockDim.x) stw[i] = A.tw[i];
    if (tid == 0) {
        for (int k = 0; k < kRingBufs; ++k) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(ring_smem(&st.full[k])));
            st.issued[k] = (k < my_tiles) ? 1 : 0;
            st.consumed[k] = 0;
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    pdl_wait();  // the previous pass's writes are visible from here on
    if (tid == 0)
        for (int k = 0; k < kRingBufs && k < my_tiles; ++k)
            ring_issue<N>(A, &tmap, blockIdx.x + k * G, ring_bufs(A.tw_pad) + k * kBufElems, ring_smem(&st.full[k]));

    const int c = gtid % kRingWidth;  // column within the tile
    const int lane = gtid / kRingWidth;
    const GroupBarrier<GT> gbar{bar_id};
    bool failed = false;
    for (int i = grp; i < my_tiles; i += kRingGroups) {
        const int slot = i % kRingBufs;
        float2* buf = ring_bufs(A.tw_pad) + slot * kBufElems;
        const bool ok_wait = ring_wait(ring_smem(&st.full[slot]), (uint32_t)((i / kRingBufs) & 1), A.wait_cycles);
        if (group_any<GT>(bar_id, !ok_wait)) {
            failed = true;
            break;
        }
        if (gtid == 0) atomicAdd(&st.consumed[slot], 1);
        const RingColIn<float2> src{buf + c, A.isign};
        const SmemColFixed<float2, kRingWidth> work{buf + c};
        // first stage: copied tile -> registers -> the same buffer (in place)
        fft_stage_s<SchedT, 0, T>(src, gbar, work, stw, lane, true);
        gbar();
        if constexpr (sc.count > 2) {
            fft_stage_s<SchedT, 1, T>(work, gbar, work, stw, lane, true);
            gbar();
        }
        if constexpr (sc.count > 3) {
            fft_stage_s<SchedT, 2, T>(work, gbar, work, stw, lane, true);
            gbar();
        }
        // last stage: its reads, the buffer release, its stores to HBM
        const int t = (int)blockIdx.x + i * G;
        const int b = t / (int)A.tiles_per_row;
        const int m = (t - b * (int)A.tiles_per_row) * kRingWidth + c;
        const bool ok = m < A.M;
        const long long base = (long long)b * N * A.M + (ok ? m : 0);
        const int inext = i + kRingBufs;
        const RingRelease<N, GT> rel{slot * 8 + bar_id, (gtid == 0 && inext < my_tiles) ? (int)blockIdx.x + inext * G : -1,
                                     &A, &tmap, &st};
        fft_stage_s<SchedT, sc.count - 1, T>(work, rel, GlobalOutT<float2>{out + base, A.M, A.isign}, stw, lane, ok);
    }
    if (failed && gtid == 0 && A.status) atomicExch(A.status, 5 /* CROFT_ERR_TIMEOUT */);
    // Before the CTA's shared memory goes away, every copy it issued has landed.  On the normal
    // path each one was waited for by its consumer.  A buffer holds at most one copy in flight
    // (the next copy into it is issued only after its previous tile was consumed), so after a
    // timeout the copy pending in buffer k, if any, is use number consumed[k]: wait for that
    // phase once more (bounded).
    __syncthreads();
    if (tid == 0)
        for (int k = 0; k < kRingBufs; ++k)
            if (st.issued[k] > st.consumed[k])
                ring_wait(ring_smem(&st.full[k]), (uint32_t)(st.consumed[k] & 1), A.wait_cycles);
}

}  // namespace croft
