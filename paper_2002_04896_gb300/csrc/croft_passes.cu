// croft_passes.cu - finds the specialised pass kernel for an axis length and launches it.
#include "croft_internal.h"

namespace croft {

pass_fn pass_kernel_for(int layout, int n) {
    pass_fn f = lookup_pass_kernel_group_0(layout, n);
    if (!f) f = lookup_pass_kernel_group_1(layout, n);
    if (!f) f = lookup_pass_kernel_group_2(layout, n);
    if (!f) f = lookup_pass_kernel_group_3(layout, n);
    return f;
}

cudaError_t prepare_pass(const PassLaunch& L) {
    pass_fn f = pass_kernel_for(L.layout, L.args.n);
    if (!f) return cudaErrorInvalidValue;
    if (L.smem <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, L.smem);
}

cudaError_t launch_pass(const PassLaunch& L, const float2* in, float2* out, cudaStream_t s) {
    pass_fn f = pass_kernel_for(L.layout, L.args.n);
    if (!f) return cudaErrorInvalidValue;
    f<<<L.grid, L.block, L.smem, s>>>(in, out, L.args);
    return cudaGetLastError();
}

}  // namespace croft
