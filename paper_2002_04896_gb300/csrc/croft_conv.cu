// croft_conv.cu - instantiates the fused convolution pass (croft_conv_kernel.cuh).
// Compiled five times: -DCROFT_CONV_GROUP=0..3 take the four complex64 size groups
// of croft_sizes.h; 4 takes the complex128 lengths and the multiply-only kernels.
#include "croft_conv_kernel.cuh"
#include "croft_sizes.h"

#ifndef CROFT_CONV_GROUP
#error "compile with -DCROFT_CONV_GROUP=<0..4>"
#endif

namespace croft {

#define CROFT_CONV_CASE(N) \
    case N: return conv_kernel_of<N, float2>();

#define CROFT_CAT_(a, b) a##b
#define CROFT_CAT(a, b) CROFT_CAT_(a, b)

#if CROFT_CONV_GROUP < 4
conv_fn CROFT_CAT(lookup_conv_kernel_group_, CROFT_CONV_GROUP)(int n) {
    switch (n) {
        CROFT_CAT(CROFT_SIZES_, CROFT_CONV_GROUP)(CROFT_CONV_CASE)
        default: return nullptr;
    }
}
#else
// complex128: the lengths of the complex128 pass kernels
conv64_fn conv64_kernel_for(int n) {
#define CROFT_CONV64_CASE(N) \
    case N: return conv_kernel_of<N, double2>();
    switch (n) {
        CROFT_SIZES64(CROFT_CONV64_CASE)
        default: return nullptr;
    }
#undef CROFT_CONV64_CASE
}

cudaError_t launch_scale(const void* in, void* out, const void* g, long long n, bool f64, cudaStream_t s, bool pdl) {
    if (n <= 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > 152LL * 8) blocks = 152LL * 8;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks, 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    if (pdl) {
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    if (f64)
        return cudaLaunchKernelEx(&cfg, croft_scale_kernel<double2>, (const double2*)in, (double2*)out, (const double*)g, n);
    return cudaLaunchKernelEx(&cfg, croft_scale_kernel<float2>, (const float2*)in, (float2*)out, (const float*)g, n);
}
#endif

}  // namespace croft
