// croft_plane_kernel.cuh - fused z + y pass: the 2D FFT of whole yz-planes, one
// plane per thread-block cluster, exchanged through the cluster's distributed
// shared memory by the bulk-copy engine.
//
// Paper mapping (Sec. 4.1): steps 1-5 (FFT along the aligned axis, pack,
// all-to-all in the column communicator, unpack, FFT along the next axis) for
// one x-slab.  The C CTAs of a cluster play the paper's processes: CTA r owns
// rows y in [r*RY, (r+1)*RY) for the z transform (step 1) and columns
// z in [r*CZ, (r+1)*CZ) for the y transform (step 5), RY = NY/C, CZ = NZ/C.
//   step 2 (pack):   the last z stage writes its results grouped by the CTA
//                    that owns their column: block d = rows of this CTA x
//                    columns of CTA d, contiguous;
//   step 3 (all-to-all): one thread issues C bulk copies shared -> shared::cluster
//                    (cp.async.bulk), block d into CTA d's column tile at the rows
//                    of this CTA; each copy completes on the receiver's mbarrier;
//   step 4 (unpack): nothing to do - the blocks land in the receiver's [NY][CZ]
//                    layout;
//   step 5:          the y stages run locally and write HBM.
// The grid crosses HBM twice per transform (this pass + the x pass) instead of
// three times.
//
// Synchronisation.  Each CTA initialises its receive mbarrier with the bytes it
// expects (NY*CZ*8) and arrives on a cluster barrier; it waits on that barrier
// only right before its first bulk copy (so every peer's mbarrier is ready).
// After its receive mbarrier completes it arrives on a second cluster barrier
// and waits on it only at the very end: when that barrier completes, every
// copy of the cluster has landed, so no CTA exits while its shared memory is
// still read or written by a copy.  The mbarrier wait is bounded.
#pragma once
#include <type_traits>

#include "croft_fft_core.cuh"
#include "croft_internal.h"

namespace croft {

__device__ __forceinline__ uint32_t plane_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

template <int NY, int NZ, int C>
struct PlaneShape {
    static constexpr int RY = NY / C;                         // rows per CTA (z phase)
    static constexpr int CZ = NZ / C;                         // columns per CTA (y phase)
    static constexpr int TZ = croft_threads_per_pencil(NZ);
    static constexpr int TY = croft_threads_per_pencil(NY);
    static constexpr int LDZ = croft_row_ld_staged(NZ);
    static constexpr int THREADS = (RY * TZ > CZ * TY) ? RY * TZ : CZ * TY;
    static constexpr int TWZ = ((NZ + 1) / 2) * 2;            // twiddle slots (keep the tiles 16-byte aligned)
    static constexpr int TWY = (NY == NZ) ? 0 : ((NY + 1) / 2) * 2;
    static constexpr int ZTILE = ((RY * LDZ + 1) / 2) * 2;    // z phase: RY padded rows, then the packed blocks
    static constexpr int YTILE = NY * CZ;                     // y phase: [NY][CZ]
    static constexpr int SMEM_BYTES = (TWZ + TWY + ZTILE + YTILE) * 8;
    static constexpr uint32_t BLOCK_BYTES = RY * CZ * 8;      // one CTA -> one CTA
    static_assert(NY % C == 0 && NZ % C == 0, "cluster size must divide both plane axes");
    static_assert(THREADS <= 1024, "too many threads per CTA");
    static_assert(C == 1 || (BLOCK_BYTES % 16) == 0, "bulk copies move multiples of 16 bytes");
};

// Packed output of the last z stage: element z of row r goes to block z / CZ, row r, column z % CZ.
template <int RY, int CZ>
struct PackedBlocks {
    float2* base;  // the z tile, reused
    int r;         // local row
    __device__ __forceinline__ void store(int z, float2 v) const {
        base[(z / CZ) * (RY * CZ) + r * CZ + (z % CZ)] = v;
    }
};

__device__ __forceinline__ bool plane_wait(uint32_t mbar, uint32_t parity) {
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

// Grid: nplanes * C CTAs in clusters of C along x.  Plane p = blockIdx.x / C.
template <int NY, int NZ, int C>
__global__ void __launch_bounds__(PlaneShape<NY, NZ, C>::THREADS) croft_plane_kernel(
    const float2* in, float2* out, const __grid_constant__ PlaneArgs A) {
    using Sh = PlaneShape<NY, NZ, C>;
    constexpr CroftSched scz = croft_make_sched(NZ);
    // the y phase runs the y axis's column-pass schedule (its twiddle table follows it)
    using YS = typename std::conditional<croft_even_pow2_pass(NY, LAYOUT_COL, 8), EvenPow2Sched<NY>, DefaultSched<NY>>::type;
    constexpr CroftSched scy = YS::get();
    extern __shared__ __align__(16) float2 smem[];
    __shared__ __align__(8) uint64_t ybar;
    float2* twz = smem;
    float2* twy = (NY == NZ) ? smem : smem + Sh::TWZ;
    float2* ztile = smem + Sh::TWZ + Sh::TWY;
    float2* ytile = ztile + Sh::ZTILE;
    const int tid = threadIdx.x;
    for (int i = tid; i < NZ - 1; i += blockDim.x) twz[i] = A.tw_z[i];
    if (NY != NZ)
        for (int i = tid; i < NY - 1; i += blockDim.x) twy[i] = A.tw_y[i];

    unsigned rank = 0;
    if constexpr (C > 1) {
        rank = cooperative_groups::this_cluster().block_rank();
        if (tid == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(plane_smem(&ybar)));
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(plane_smem(&ybar)),
                         "r"((uint32_t)(NY * Sh::CZ * 8))
                         : "memory");
        }
        asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");  // (1) my mbarrier is ready
    }
    const long long plane = blockIdx.x / C;
    const long long off = plane * (long long)NY * NZ;
    pdl_allow_dependents();
    pdl_wait();

    // ---- z phase: rows rank*RY + r, one pencil per TZ threads --------------------
    {
        const int r = tid / Sh::TZ;
        const int lane = tid - r * Sh::TZ;
        const bool ok = r < Sh::RY;
        const int rr = ok ? r : 0;
        const int y = rank * Sh::RY + rr;
        const GlobalInUnit src{in + off + (long long)y * NZ, A.isign};
        float2* row = ztile + rr * Sh::LDZ;
        if constexpr (C > 1) {
            // every stage but the last in the padded rows; the last packs the blocks (in place)
            const PackedBlocks<Sh::RY, Sh::CZ> dst{ztile, rr};
            if constexpr (scz.count == 1) {
                fft_stage<NZ, 0, Sh::TZ>(src, NoBarrier{}, dst, twz, lane, ok);
            } else {
                const typename RowPadOf<NZ, 0>::type w0{row};
                fft_stage<NZ, 0, Sh::TZ>(src, NoBarrier{}, w0, twz, lane, ok);
                __syncthreads();
                row_stages<NZ, 1, scz.count - 1, Sh::TZ>(row, twz, lane, ok);
                const typename RowPadOf<NZ, scz.count - 2>::type wl{row};
                fft_stage<NZ, scz.count - 1, Sh::TZ>(wl, CtaBarrier{}, dst, twz, lane, ok);
            }
        } else {
            const SmemCol dst{ytile + y * Sh::CZ, 1};  // row y of the local [NY][NZ] tile
            fft_pencil_row<NZ, Sh::TZ>(src, row, dst, twz, lane, ok);
        }
    }

    // ---- exchange (steps 2-4) ----------------------------------------------------
    if constexpr (C > 1) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // packed blocks -> bulk-copy engine
        __syncthreads();
        asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");  // (1): every peer's mbarrier is ready
        if (tid == 0) {
            const uint32_t src0 = plane_smem(ztile);
            const uint32_t dst_local = plane_smem(ytile) + rank * Sh::BLOCK_BYTES;  // my rows in the receiver's tile
            const uint32_t bar_local = plane_smem(&ybar);
            for (unsigned d = 0; d < (unsigned)C; ++d) {
                uint32_t dst, bar;
                asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(dst) : "r"(dst_local), "r"(d));
                asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(bar) : "r"(bar_local), "r"(d));
                asm volatile(
                    "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                    "r"(src0 + d * Sh::BLOCK_BYTES), "r"(Sh::BLOCK_BYTES), "r"(bar)
                    : "memory");
            }
        }
        if (!plane_wait(plane_smem(&ybar), 0) && A.status) atomicExch(A.status, 5 /* CROFT_ERR_TIMEOUT */);
        asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");  // (2) all my incoming blocks landed
    } else {
        __syncthreads();
    }

    // ---- y phase: column rank*CZ + c, one pencil per TY threads, local -----------
    {
        const int c = tid % Sh::CZ;
        const int lane = tid / Sh::CZ;
        const bool ok = lane < Sh::TY;
        const int z = rank * Sh::CZ + c;
        const SmemCol col{ytile + c, Sh::CZ};
        const GlobalOut dst{out + off + z, NZ, A.isign};
        if constexpr (scy.count == 1) {
            fft_stage_s<YS, 0, Sh::TY>(col, NoBarrier{}, dst, twy, lane, ok);
        } else {
            fft_stage_s<YS, 0, Sh::TY>(col, CtaBarrier{}, col, twy, lane, ok);
            __syncthreads();
            smem_stages_s<YS, 1, scy.count - 1, Sh::TY>(col, twy, lane, ok);
            fft_stage_s<YS, scy.count - 1, Sh::TY>(col, NoBarrier{}, dst, twy, lane, ok);
        }
    }
    if constexpr (C > 1) asm volatile("barrier.cluster.wait.aligned;" ::: "memory");  // (2): no copy in flight
}

}  // namespace croft
