// croft_plane_kernel.cuh - fused z + y pass: the 2D FFT of whole yz-planes, one
// plane per thread-block cluster, held in the cluster's distributed shared memory.
//
// Paper mapping (Sec. 4.1): steps 1-5 (FFT along the aligned axis, pack,
// all-to-all in the column communicator, unpack, FFT along the next axis) for
// one x-slab.  The paper moves the slab between processes with MPI_Alltoall;
// here the C CTAs of a cluster play the processes: CTA r first owns rows
// y in [r*NY/C, (r+1)*NY/C) and transforms them along z (step 1), then owns
// columns z in [r*NZ/C, (r+1)*NZ/C) and transforms them along y (step 5).  The
// all-to-all of steps 2-4 is the first y stage reading its inputs straight
// from the other CTAs' shared memory (DSMEM); no byte of it touches HBM.  The
// grid therefore crosses HBM twice per transform (this pass + the x pass)
// instead of three times.
//
// Synchronisation (all waits are hardware barriers, none can spin forever):
//   z stages (CTA barriers) -> cluster barrier (every row done, visible to the
//   cluster) -> first y stage reads remote rows into registers -> cluster
//   barrier (every remote read done before any CTA overwrites its tile) ->
//   first y stage writes its outputs into the own tile -> y stages -> HBM.
#pragma once
#include "croft_fft_core.cuh"
#include "croft_internal.h"

namespace croft {

struct ClusterBarrier {
    __device__ __forceinline__ void operator()() const { cooperative_groups::this_cluster().sync(); }
};

// Row y, column z of the z-transformed plane, wherever in the cluster it lives:
// rows are split across the C CTAs in blocks of RY, each CTA's tile is RY
// padded rows of length LDZ.
template <int RY, int LDZ>
struct DsmemRows {
    float2* tile;  // this CTA's tile (same offset in every CTA of the cluster)
    int z;         // column
    __device__ __forceinline__ float2 load(int y) const {
        float2* base = cooperative_groups::this_cluster().map_shared_rank(tile, (unsigned)(y / RY));
        return base[(y % RY) * LDZ + z + (z >> 4)];
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
    static constexpr int TILE = (RY * LDZ > NY * CZ) ? RY * LDZ : NY * CZ;
    static constexpr int SMEM_BYTES = (TWZ + TWY + TILE) * 8;
    static_assert(NY % C == 0 && NZ % C == 0, "cluster size must divide both plane axes");
    static_assert(THREADS <= 1024, "too many threads per CTA");
};

// Grid: nplanes * C CTAs in clusters of C along x.  Plane p = blockIdx.x / C.
template <int NY, int NZ, int C>
__global__ void __launch_bounds__(PlaneShape<NY, NZ, C>::THREADS) croft_plane_kernel(
    const float2* in, float2* out, const __grid_constant__ PlaneArgs A) {
    using Sh = PlaneShape<NY, NZ, C>;
    constexpr CroftSched scz = croft_make_sched(NZ);
    constexpr CroftSched scy = croft_make_sched(NY);
    extern __shared__ float2 smem[];
    float2* twz = smem;
    float2* twy = (NY == NZ) ? smem : smem + Sh::TWZ;
    float2* tile = smem + Sh::TWZ + Sh::TWY;
    const int tid = threadIdx.x;
    for (int i = tid; i < NZ - 1; i += blockDim.x) twz[i] = A.tw_z[i];
    if (NY != NZ)
        for (int i = tid; i < NY - 1; i += blockDim.x) twy[i] = A.tw_y[i];

    const unsigned rank = (C == 1) ? 0u : cooperative_groups::this_cluster().block_rank();
    const long long plane = blockIdx.x / C;
    const long long off = plane * (long long)NY * NZ;

    // ---- z phase: row y = rank*RY + r, one pencil per TZ threads ----------------
    {
        const int r = tid / Sh::TZ;
        const int lane = tid - r * Sh::TZ;
        const bool ok = r < Sh::RY;
        const int rr = ok ? r : 0;
        const GlobalInUnit src{in + off + (long long)(rank * Sh::RY + rr) * NZ, A.isign};
        const SmemRow row{tile + rr * Sh::LDZ};
        fft_stage<NZ, 0, Sh::TZ>(src, NoBarrier{}, row, twz, lane, ok);
        __syncthreads();
        smem_stages<NZ, 1, scz.count, Sh::TZ>(row, twz, lane, ok);
    }
    if (C > 1) ClusterBarrier{}();

    // ---- y phase: column z = rank*CZ + c, one pencil per TY threads -------------
    {
        const int c = tid % Sh::CZ;
        const int lane = tid / Sh::CZ;
        const bool ok = lane < Sh::TY;
        const int z = rank * Sh::CZ + c;
        const SmemCol col{tile + c, Sh::CZ};
        const GlobalOut dst{out + off + z, NZ, A.isign};
        if constexpr (C > 1) {
            const DsmemRows<Sh::RY, Sh::LDZ> src{tile, z};
            if constexpr (scy.count == 1) {
                fft_stage<NY, 0, Sh::TY>(src, ClusterBarrier{}, dst, twy, lane, ok);
            } else {
                fft_stage<NY, 0, Sh::TY>(src, ClusterBarrier{}, col, twy, lane, ok);
                __syncthreads();
                smem_stages<NY, 1, scy.count - 1, Sh::TY>(col, twy, lane, ok);
                fft_stage<NY, scy.count - 1, Sh::TY>(col, NoBarrier{}, dst, twy, lane, ok);
            }
        } else {
            // single CTA: the rows are local; read them in place (padded row layout)
            struct LocalRows {
                const float2* tile;
                int z;
                __device__ __forceinline__ float2 load(int y) const { return tile[y * Sh::LDZ + z + (z >> 4)]; }
            };
            const LocalRows src{tile, z};
            if constexpr (scy.count == 1) {
                fft_stage<NY, 0, Sh::TY>(src, NoBarrier{}, dst, twy, lane, ok);
            } else {
                fft_stage<NY, 0, Sh::TY>(src, CtaBarrier{}, col, twy, lane, ok);
                __syncthreads();
                smem_stages<NY, 1, scy.count - 1, Sh::TY>(col, twy, lane, ok);
                fft_stage<NY, scy.count - 1, Sh::TY>(col, NoBarrier{}, dst, twy, lane, ok);
            }
        }
    }
}

}  // namespace croft
