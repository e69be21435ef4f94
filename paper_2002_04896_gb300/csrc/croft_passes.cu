// croft_passes.cu - finds the specialised kernel of a pass and launches it.
#include "croft_internal.h"

namespace croft {

pass_fn pass_kernel_for(int layout, int n) {
    pass_fn f = lookup_pass_kernel_group_0(layout, n);
    if (!f) f = lookup_pass_kernel_group_1(layout, n);
    if (!f) f = lookup_pass_kernel_group_2(layout, n);
    if (!f) f = lookup_pass_kernel_group_3(layout, n);
    return f;
}

static cudaLaunchConfig_t plane_config(const PassLaunch& L, cudaStream_t s, cudaLaunchAttribute* attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)L.grid, 1, 1);
    cfg.blockDim = dim3((unsigned)L.block, 1, 1);
    cfg.dynamicSmemBytes = (size_t)L.smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)L.pk.cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

cudaError_t prepare_pass(const PassLaunch& L) {
    if (L.kind == PASS_PLANE) {
        cudaError_t e = cudaFuncSetAttribute(L.pk.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, L.smem);
        if (e != cudaSuccess) return e;
        if (L.pk.cluster > 8) {
            e = cudaFuncSetAttribute(L.pk.fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (e != cudaSuccess) return e;
        }
        // the cluster must fit on the device at all
        cudaLaunchAttribute attr[1];
        cudaLaunchConfig_t cfg = plane_config(L, 0, attr);
        int nclusters = 0;
        e = cudaOccupancyMaxActiveClusters(&nclusters, L.pk.fn, &cfg);
        if (e != cudaSuccess) return e;
        return nclusters > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
    }
    pass_fn f = L.tc ? tc_pass_kernel_for(L.layout, L.args.n) : pass_kernel_for(L.layout, L.args.n);
    if (!f) return cudaErrorInvalidValue;
    if (L.smem <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, L.smem);
}

cudaError_t launch_pass(const PassLaunch& L, const float2* in, float2* out, cudaStream_t s) {
    if (L.kind == PASS_PLANE) {
        cudaLaunchAttribute attr[1];
        cudaLaunchConfig_t cfg = plane_config(L, s, attr);
        return cudaLaunchKernelEx(&cfg, L.pk.fn, in, out, L.pargs);
    }
    pass_fn f = L.tc ? tc_pass_kernel_for(L.layout, L.args.n) : pass_kernel_for(L.layout, L.args.n);
    if (!f) return cudaErrorInvalidValue;
    f<<<L.grid, L.block, L.smem, s>>>(in, out, L.args);
    return cudaGetLastError();
}

int active_clusters(const PassLaunch& L) {
    if (L.kind != PASS_PLANE) return 0;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = plane_config(L, 0, attr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, L.pk.fn, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

}  // namespace croft
