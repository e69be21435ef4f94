// croft_planes.cu - instantiations of the fused z+y plane kernel and their registry.
//
// Per (ny, nz) plane shape, cluster sizes C for which a CTA's two tiles (NY/C
// padded rows for the z phase, NZ/C columns for the y phase) fit in shared
// memory with at most 1024 threads.  Other plane shapes run the other schedules.
#include "croft_plane_kernel.cuh"

namespace croft {

#define CROFT_PLANE(NY, NZ, C)                                                                       \
    {croft_plane_kernel<NY, NZ, C>, NY, NZ, C, PlaneShape<NY, NZ, C>::THREADS,                          \
     PlaneShape<NY, NZ, C>::SMEM_BYTES}

// Several cluster sizes per shape where they fit; the first entry is the default.
static const PlaneKernel kPlaneKernels[] = {
    CROFT_PLANE(32, 32, 1),     CROFT_PLANE(64, 64, 2),     CROFT_PLANE(64, 64, 1),
    CROFT_PLANE(128, 128, 4),   CROFT_PLANE(128, 128, 2),   CROFT_PLANE(256, 256, 16),
    CROFT_PLANE(256, 256, 8),   CROFT_PLANE(384, 384, 16),
};

const PlaneKernel* find_plane_kernel(int ny, int nz, int cluster) {
    for (const PlaneKernel& k : kPlaneKernels)
        if (k.ny == ny && k.nz == nz && (cluster <= 0 || k.cluster == cluster)) return &k;
    return nullptr;
}

}  // namespace croft
