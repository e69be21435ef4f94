// croft_passes.cu - finds the specialised kernel of a pass and launches it.
#include <cudaTypedefs.h>

#include <string.h>

#include <mutex>

#include "croft_internal.h"

namespace croft {

int g_max_smem = 0;


// Launch shape of one pass (layouts: croft_internal.h; kernel: croft_pass_kernel.cuh).
// ROW: W pencils of length n per CTA, each padded to n + n/16 + 1 slots.
// COL: W adjacent columns per CTA, W a multiple of 16 (128-byte rows).
// Aim for ~256 threads per CTA and <= 100 KB of shared memory so that at
// least two CTAs share an SM.
bool shape_pass(PassLaunch& L, int layout, int n, long long M, long long ncols, int tc, bool f64, int want_w, int sv,
                int th) {
    memset(&L, 0, sizeof(L));
    L.layout = layout;
    L.tc = tc;
    L.sv = sv;
    L.th = (layout == LAYOUT_COL && !tc && !f64) ? th : 0;
    L.f64 = f64 ? 1 : 0;
    const long long es = f64 ? 16 : 8;  // bytes per element
    if (M < 1) return false;
    PassArgs& A = L.args;
    A.n = n;
    A.M = M;
    A.ncols = ncols;
    const int T = L.th > 0 ? L.th : croft_threads_per_pencil(n);
    L.T = T;
    A.tw_pad = ((n + 1) / 2) * 2;  // keeps the tile 16-byte aligned
    const long long smem_cap = 100 * 1024;
    const int max_threads = 512;   // the kernels' launch bound
    if (layout == LAYOUT_ROW) {
        const int ld = tc ? croft_row_ld(n) : croft_row_ld_staged(n);
        int W = (256 + T - 1) / T;
        if (W < 1) W = 1;
        while (W > 1 && (W * T > max_threads || (A.tw_pad + (long long)W * ld) * es > smem_cap)) --W;
        if ((long long)W > ncols && !tc) W = (int)ncols;  // (tensor-core tiles keep whole 128-row groups)
        A.W = W;
        L.smem = (int)((A.tw_pad + (long long)W * ld) * es);
    } else {
        int W = 16;
        if (tc) {
            while (W * 2 * T <= 256) W *= 2;
            if (croft_col_narrow(n, (int)es, M * es)) W = kColNarrowWidth;  // (two 128-butterfly groups)
        } else {
            W = croft_col_width_at(n, (int)es, M * es);  // a width the kernels are built for
        }
        if (want_w >= 1 && !tc) W = want_w;
        while (W > 1 && (W * T > max_threads || (A.tw_pad + (long long)n * W) * es > smem_cap)) W /= 2;
        A.W = W;
        L.smem = (int)((A.tw_pad + (long long)n * W) * es);
    }
    L.block = A.W * T;
    if (layout == LAYOUT_COL) A.cdiv = croft_coldiv_make(M, ncols + A.W);
    if (croft_make_sched(n).count <= 1 && !tc) L.smem = 0;  // single-stage kernels touch no shared memory
    if (tc) {
        // the A operands (128 bytes per thread) reuse the pass tile, which may be smaller
        const long long tile = L.smem - (long long)A.tw_pad * es, ops = 128LL * L.block;
        L.smem = (int)((long long)A.tw_pad * es + 4096 + (tile > ops ? tile : ops));  // + the DFT-16 operand
    }
    if (tc && (L.block % 128) != 0) return false;           // 128-butterfly GEMM groups
    if (L.block > max_threads) return false;
    long long grid = (ncols + A.W - 1) / A.W;
    if (grid > 0x7fffffffLL) return false;
    L.grid = (int)grid;
    if (L.smem > g_max_smem) return false;
    return true;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to libcuda).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        else
            cudaGetLastError();
    });
    return fn;
}

// 3D map over the source of a ring column pass: dims {M, n, B} (innermost first), box
// {16 columns, box_rows, 1}; 8-byte elements (one complex64 each), no swizzle.
static bool encode_ring_map(const PassLaunch& L, const float2* src, CUtensorMap* map) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)L.ra.M, (cuuint64_t)L.args.n, (cuuint64_t)L.B};
    const cuuint64_t strides[2] = {(cuuint64_t)L.ra.M * sizeof(float2), (cuuint64_t)L.ra.M * L.args.n * sizeof(float2)};
    const cuuint32_t box[3] = {(cuuint32_t)kRingTileWidth, (cuuint32_t)L.ra.box_rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, (void*)src, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static cudaLaunchConfig_t pair_config(const PassLaunch& L, cudaStream_t s, cudaLaunchAttribute* attr, bool pdl) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)L.grid, 1, 1);
    cfg.blockDim = dim3((unsigned)L.block, 1, 1);
    cfg.dynamicSmemBytes = (size_t)L.smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (pdl) {
        attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[1].val.programmaticStreamSerializationAllowed = 1;
        cfg.numAttrs = 2;
    }
    return cfg;
}

bool shape_pair(PassLaunch& L, int n, long long M, long long ncols) {
    memset(&L, 0, sizeof(L));
    pass_fn f = pair_kernel_for(n);
    if (!f || n % 2 || M < 1 || ncols % M != 0) return false;
    const int n2 = n / 2;
    L.kind = PASS_AXIS;
    L.layout = LAYOUT_COL;
    L.pair = 1;
    L.T = croft_threads_per_pencil(n2);
    PassArgs& A = L.args;
    A.n = n;
    A.M = M;
    A.ncols = ncols;
    A.W = kPairTileWidth;
    A.cdiv = croft_coldiv_make(M, ncols + kPairTileWidth);
    A.tw_pad = ((n2 + 1) / 2) * 2;
    L.block = kPairTileWidth * L.T;
    L.smem = (A.tw_pad + (n2 + (n2 & 1)) + n2 * kPairTileWidth) * (int)sizeof(float2);
    const long long grid = 2 * ((ncols + kPairTileWidth - 1) / kPairTileWidth);
    if (grid > 0x7fffffffLL || L.smem > g_max_smem) return false;
    L.grid = (int)grid;
    if (L.smem > 48 * 1024 && cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, L.smem) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchAttribute attr[2];
    cudaLaunchConfig_t cfg = pair_config(L, 0, attr, false);
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, f, &cfg) != cudaSuccess || clusters < 1) {
        cudaGetLastError();
        return false;
    }
    return true;
}

bool shape_ring(PassLaunch& L, int n, long long M, long long ncols) {
    memset(&L, 0, sizeof(L));
    ring_fn f = ring_kernel_for(n);
    // tensor copies need 16-byte strides (M even) and 16-byte aligned column starts (tiles of 16)
    if (!f || croft_threads_per_pencil(n) != 32 || M < 2 || (M % 2) != 0 || ncols % M != 0) return false;
    L.kind = PASS_AXIS;
    L.layout = LAYOUT_COL;
    L.ring = 1;
    L.T = 32;
    L.args.n = n;
    L.args.M = M;
    L.args.ncols = ncols;
    L.args.W = kRingTileWidth;
    RingArgs& R = L.ra;
    R.M = M;
    R.tiles_per_row = (M + kRingTileWidth - 1) / kRingTileWidth;
    L.B = ncols / M;
    R.ntiles = L.B * R.tiles_per_row;
    if (R.ntiles > 0x7fffffffLL || L.B > 0x7fffffffLL) return false;
    int k = (n + 255) / 256;  // rows per box: the largest divisor of n that is <= 256
    while (n % k) ++k;
    R.box_rows = n / k;
    R.tw_pad = ((n + 15) / 16) * 16;
    R.wait_cycles = 4000000000LL;  // ~2 s at the maximum SM clock
    L.block = 1024;
    L.smem = (R.tw_pad + 3 * n * kRingTileWidth) * (int)sizeof(float2) + 128;  // + alignment of the tiles
    if (L.smem > g_max_smem) return false;
    if (L.smem > 48 * 1024 && cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, L.smem) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, L.block, L.smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return false;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    L.grid = (int)(R.ntiles < (long long)sms ? R.ntiles : (long long)sms);
    return L.grid > 0 && tensor_map_encoder() != nullptr;
}

pass_fn pass_kernel_for(int layout, int n, int w, int sv, int th) {
    pass_fn f = lookup_pass_kernel_group_0(layout, n, w, sv, th);
    if (!f) f = lookup_pass_kernel_group_1(layout, n, w, sv, th);
    if (!f) f = lookup_pass_kernel_group_2(layout, n, w, sv, th);
    if (!f) f = lookup_pass_kernel_group_3(layout, n, w, sv, th);
    return f;
}

conv_fn conv_kernel_for(int n) {
    conv_fn f = lookup_conv_kernel_group_0(n);
    if (!f) f = lookup_conv_kernel_group_1(n);
    if (!f) f = lookup_conv_kernel_group_2(n);
    if (!f) f = lookup_conv_kernel_group_3(n);
    return f;
}

// attr must have room for two entries: the cluster shape and, with pdl, programmatic serialisation.
static cudaLaunchConfig_t plane_config(const PassLaunch& L, cudaStream_t s, cudaLaunchAttribute* attr, bool pdl = false) {
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
    if (pdl) {
        attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[1].val.programmaticStreamSerializationAllowed = 1;
        cfg.numAttrs = 2;
    }
    return cfg;
}

// Plain launch of a pass-shaped kernel, with programmatic stream serialisation when pdl
// (the kernel must call pdl_wait() before reading what the previous launch wrote).
template <class... P, class... A>
static cudaError_t launch_ex(void (*f)(P...), const PassLaunch& L, cudaStream_t s, bool pdl, A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)L.grid, 1, 1);
    cfg.blockDim = dim3((unsigned)L.block, 1, 1);
    cfg.dynamicSmemBytes = (size_t)L.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    if (pdl) {
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    return cudaLaunchKernelEx(&cfg, f, args...);
}

bool pass_supports_pdl(const PassLaunch& L) { return !L.tc; }

cudaError_t prepare_pass(const PassLaunch& L) {
    if (L.kind == PASS_PLANE) {
        cudaError_t e = cudaFuncSetAttribute(L.pk.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, L.smem);
        if (e != cudaSuccess) return e;
        if (L.pk.cluster > 8) {
            e = cudaFuncSetAttribute(L.pk.fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (e != cudaSuccess) return e;
        }
        // the cluster must fit on the device at all
        cudaLaunchAttribute attr[2];
        cudaLaunchConfig_t cfg = plane_config(L, 0, attr);
        int nclusters = 0;
        e = cudaOccupancyMaxActiveClusters(&nclusters, L.pk.fn, &cfg);
        if (e != cudaSuccess) return e;
        return nclusters > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
    }
    if (L.pair) return pair_kernel_for(L.args.n) ? cudaSuccess : cudaErrorInvalidValue;
    if (L.ring) {
        ring_fn f = ring_kernel_for(L.args.n);
        if (!f || !tensor_map_encoder()) return cudaErrorInvalidValue;
        if (L.smem <= 48 * 1024) return cudaSuccess;
        return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, L.smem);
    }
    if (L.f64) {
        pass64_fn f = pass64_kernel_for(L.layout, L.args.n, L.args.W);
        if (!f) return cudaErrorInvalidValue;
        if (L.smem <= 48 * 1024) return cudaSuccess;
        return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, L.smem);
    }
    pass_fn f = L.tc ? tc_pass_kernel_for(L.layout, L.args.n, L.tc - 1) : pass_kernel_for(L.layout, L.args.n, L.args.W, L.sv, L.th);
    if (!f) return cudaErrorInvalidValue;
    if (L.smem <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, L.smem);
}

cudaError_t launch_pass(const PassLaunch& L, const void* vin, void* vout, cudaStream_t s, bool pdl) {
    pdl = pdl && pass_supports_pdl(L);
    if (L.f64) {
        pass64_fn f = pass64_kernel_for(L.layout, L.args.n, L.args.W);
        if (!f) return cudaErrorInvalidValue;
        return launch_ex(f, L, s, pdl, (const double2*)vin, (double2*)vout, L.args);
    }
    const float2* in = (const float2*)vin;
    float2* out = (float2*)vout;
    if (L.kind == PASS_PLANE) {
        cudaLaunchAttribute attr[2];
        cudaLaunchConfig_t cfg = plane_config(L, s, attr, pdl);
        return cudaLaunchKernelEx(&cfg, L.pk.fn, in, out, L.pargs);
    }
    if (L.pair) {
        pass_fn f = pair_kernel_for(L.args.n);
        if (!f) return cudaErrorInvalidValue;
        cudaLaunchAttribute attr[2];
        cudaLaunchConfig_t cfg = pair_config(L, s, attr, pdl);
        return cudaLaunchKernelEx(&cfg, f, in, out, L.args);
    }
    if (L.ring) {
        ring_fn f = ring_kernel_for(L.args.n);
        if (!f) return cudaErrorInvalidValue;
        CUtensorMap map;
        memset(&map, 0, sizeof(map));
        if (!encode_ring_map(L, in, &map)) return cudaErrorInvalidValue;
        RingArgs ra = L.ra;
        ra.isign = L.args.isign;
        ra.tw = L.args.tw;
        ra.status = L.args.status;
        return launch_ex(f, L, s, pdl, in, out, ra, map);
    }
    if (L.tc) {
        pass_fn f = tc_pass_kernel_for(L.layout, L.args.n, L.tc - 1);
        if (!f) return cudaErrorInvalidValue;
        f<<<L.grid, L.block, L.smem, s>>>(in, out, L.args);
        return cudaGetLastError();
    }
    pass_fn f = pass_kernel_for(L.layout, L.args.n, L.args.W, L.sv, L.th);
    if (!f) return cudaErrorInvalidValue;
    return launch_ex(f, L, s, pdl, in, out, L.args);
}

cudaError_t launch_conv(const PassLaunch& L, const void* in, void* out, const void* g, cudaStream_t s, bool pdl) {
    if (L.f64) {
        conv64_fn f = conv64_kernel_for(L.args.n);
        if (!f) return cudaErrorInvalidValue;
        return launch_ex(f, L, s, pdl, (const double2*)in, (double2*)out, (const double*)g, L.args);
    }
    conv_fn f = conv_kernel_for(L.args.n);
    if (!f) return cudaErrorInvalidValue;
    return launch_ex(f, L, s, pdl, (const float2*)in, (float2*)out, (const float*)g, L.args);
}

int active_clusters(const PassLaunch& L) {
    if (L.kind != PASS_PLANE) return 0;
    cudaLaunchAttribute attr[2];
    cudaLaunchConfig_t cfg = plane_config(L, 0, attr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, L.pk.fn, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

}  // namespace croft
