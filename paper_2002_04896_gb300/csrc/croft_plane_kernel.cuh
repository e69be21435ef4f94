// croft_plane_kernel.cuh - fused z + y pass: the 2D FFT of whole yz-planes, one
// plane per thread-block cluster, exchanged through the cluster's distributed
// shared memory.
//
// Paper mapping (Sec. 4.1): steps 1-5 (FFT along the aligned axis, pack,
// all-to-all in the column communicator, unpack, FFT along the next axis) for
// one x-slab.  The paper moves the slab between processes with MPI_Alltoall;
// here the C CTAs of a cluster play the processes: CTA r owns rows
// y in [r*NY/C, (r+1)*NY/C) for the z transform (step 1) and columns
// z in [r*NZ/C, (r+1)*NZ/C) for the y transform (step 5).  The pack +
// all-to-all + unpack of steps 2-4 is the last z stage storing each result
// straight into the shared memory of the CTA that owns its column (DSMEM
// stores, which do not stall the issuing thread); no byte of it touches HBM.
// The grid therefore crosses HBM twice per transform (this pass + the x pass)
// instead of three times.
//
// Each CTA has two tiles: its rows (z phase, padded rows) and its columns
// (y phase, [NY][CZ]).  Synchronisation is one cluster barrier between the
// phases (every remote store is done and visible); after it a CTA only
// touches its own shared memory, so no CTA can exit while another still
// accesses it.  All waits are hardware barriers.
#pragma once
#include "croft_fft_core.cuh"
#include "croft_internal.h"

namespace croft {

struct ClusterBarrier {
    __device__ __forceinline__ void operator()() const { cooperative_groups::this_cluster().sync(); }
};

// Element z of row y of the plane, stored into the y-phase tile of the CTA
// that owns column z (any CTA of the cluster, possibly this one).
template <int CZ>
struct DsmemColumnsOut {
    float2* ytile;  // y-phase tile: same offset in every CTA of the cluster
    int y;          // row
    __device__ __forceinline__ void store(int z, float2 v) const {
        float2* base = cooperative_groups::this_cluster().map_shared_rank(ytile, (unsigned)(z / CZ));
        base[y * CZ + (z % CZ)] = v;
    }
};

template <int NY, int NZ, int C>
struct PlaneShape {
    static constexpr int RY = NY / C;                         // rows per CTA (z phase)
    static constexpr int CZ = NZ / C;                         // columns per CTA (y phase)
    static constexpr int TZ = croft_threads_per_pencil(NZ);
    static constexpr int TY = croft_threads_per_pencil(NY);
    static constexpr int LDZ = row_ld(NZ);
    static constexpr int THREADS = (RY * TZ > CZ * TY) ? RY * TZ : CZ * TY;
    static constexpr int TWZ = ((NZ + 1) / 2) * 2;            // twiddle slots (16-byte aligned tile)
    static constexpr int TWY = (NY == NZ) ? 0 : ((NY + 1) / 2) * 2;
    static constexpr int ZTILE = RY * LDZ;   // z phase: RY padded rows
    static constexpr int YTILE = NY * CZ;    // y phase: [NY][CZ]
    static constexpr int SMEM_BYTES = (TWZ + TWY + ZTILE + YTILE) * 8;
    static_assert(NY % C == 0 && NZ % C == 0, "cluster size must divide both plane axes");
    static_assert(THREADS <= 1024, "too many threads per CTA");
};

// Grid: nplanes * C CTAs in clusters of C along x.  Plane p = blockIdx.x / C.
template <int NY, int NZ, int C>
__global__ void __launch_bounds__(PlaneShape<NY, NZ, C>::THREADS) croft_plane_kernel(
    const float2* in, float2* out, const __grid_constant__ PlaneArgs A) {
    using Sh = PlaneShape<NY, NZ, C>;
    constexpr CroftSched scy = croft_make_sched(NY);
    extern __shared__ float2 smem[];
    float2* twz = smem;
    float2* twy = (NY == NZ) ? smem : smem + Sh::TWZ;
    float2* ztile = smem + Sh::TWZ + Sh::TWY;
    float2* ytile = ztile + Sh::ZTILE;
    const int tid = threadIdx.x;
    for (int i = tid; i < NZ - 1; i += blockDim.x) twz[i] = A.tw_z[i];
    if (NY != NZ)
        for (int i = tid; i < NY - 1; i += blockDim.x) twy[i] = A.tw_y[i];

    const unsigned rank = (C == 1) ? 0u : cooperative_groups::this_cluster().block_rank();
    const long long plane = blockIdx.x / C;
    const long long off = plane * (long long)NY * NZ;

    // ---- z phase: row y = rank*RY + r, one pencil per TZ threads; the last stage
    //      stores into the owners' y tiles ---------------------------------------
    {
        const int r = tid / Sh::TZ;
        const int lane = tid - r * Sh::TZ;
        const bool ok = r < Sh::RY;
        const int rr = ok ? r : 0;
        const int y = rank * Sh::RY + rr;
        const GlobalInUnit src{in + off + (long long)y * NZ, A.isign};
        const SmemRow row{ztile + rr * Sh::LDZ};
        if constexpr (C > 1) {
            const DsmemColumnsOut<Sh::CZ> dst{ytile, y};
            fft_pencil<NZ, Sh::TZ>(src, row, dst, twz, lane, ok);
        } else {
            const SmemCol dst{ytile + y * Sh::CZ, 1};  // row y of the local [NY][NZ] tile
            fft_pencil<NZ, Sh::TZ>(src, row, dst, twz, lane, ok);
        }
    }
    if constexpr (C > 1) {
        ClusterBarrier{}();  // every row stored and visible cluster-wide
    } else {
        __syncthreads();
    }

    // ---- y phase: column z = rank*CZ + c, one pencil per TY threads, local -------
    {
        const int c = tid % Sh::CZ;
        const int lane = tid / Sh::CZ;
        const bool ok = lane < Sh::TY;
        const int z = rank * Sh::CZ + c;
        const SmemCol col{ytile + c, Sh::CZ};
        const GlobalOut dst{out + off + z, NZ, A.isign};
        if constexpr (scy.count == 1) {
            fft_stage<NY, 0, Sh::TY>(col, NoBarrier{}, dst, twy, lane, ok);
        } else {
            fft_stage<NY, 0, Sh::TY>(col, CtaBarrier{}, col, twy, lane, ok);
            __syncthreads();
            smem_stages<NY, 1, scy.count - 1, Sh::TY>(col, twy, lane, ok);
            fft_stage<NY, scy.count - 1, Sh::TY>(col, NoBarrier{}, dst, twy, lane, ok);
        }
    }
}

}  // namespace croft
