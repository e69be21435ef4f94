// croft_tc_kernel.cuh - pass kernel whose first (radix-16) stage runs on the tensor cores.
//
// A radix-16 Stockham stage applies, to every butterfly b, the 16-point DFT
// matrix F (F[k][j] = exp(-2 pi i jk/16)) after the twiddles: y = F u.  Over a
// batch of butterflies this is a dense product.  In real arithmetic, with
// u = ur + i ui and F = C + i S,
//     [yr | yi] = [ur | ui] * [[C, S], [-S, C]]      (1 x 32 times 32 x 32),
// so 128 butterflies form a 128 x 32 x 32 GEMM: M = 128 rows (butterflies),
// N = 32 (re/im of the 16 outputs), K = 32 (re/im of the 16 inputs).
//
// Precision (split operands), two variants:
//  * bf16x3: each operand x is stored as hi = bf16(x) and lo = bf16(x - hi);
//    the products hi*hi + hi*lo + lo*hi are accumulated in FP32 (the lo*lo
//    term, ~2^-16 relative, is dropped).  bf16 keeps FP32's exponent range, so
//    no pre-scaling is needed; hi + lo carries ~16 significant bits.
//  * fp16x3: the same three products with fp16 halves (11-bit significands,
//    so hi + lo carries ~22 bits and the dropped lo*lo term is ~2^-22).  fp16's
//    range is narrow, so each butterfly's 16 inputs are first scaled by a power
//    of two that puts their largest real or imaginary part in [2^14, 2^15)
//    (exact), and the 16 outputs are scaled back after the product (exact: the
//    radix-16 DFT is linear, one butterfly per GEMM row).  This is the
//    per-pencil power-of-two scaling of the split-fp16 scheme, applied per
//    butterfly, the finest granularity one GEMM row allows.
//
// Hardware path (sm_103a): operands in shared memory in the K-major,
// no-swizzle core-matrix layout (8 rows x 16 bytes per core matrix; core
// matrices adjacent in K are 128 B apart, row groups 512 B apart); one thread
// issues tcgen05.mma.cta_group::1.kind::f16 (bf16 or fp16 in, f32 accumulate)
// for every 128-row group into its own 32 TMEM columns and commits to an
// mbarrier; one warp waits for it while the others wait at the CTA barrier, and
// every warp then reads its 32 rows back with tcgen05.ld.32x32b.x32: thread t
// receives the 32 accumulators of butterfly t.  The twiddles, the hi/lo split
// and the other radices stay on the CUDA cores.
//
// The operand buffers (A hi + A lo, 128 bytes per butterfly) reuse the pass's
// shared-memory tile, sized to at least 128 bytes per thread: every input of
// the stage is in registers before the tile is overwritten, and every MMA has
// completed (mbarrier) before the outputs are written back into it.
#pragma once
#include <type_traits>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "croft_fft_core.cuh"
#include "croft_internal.h"
#include "croft_tc_operand.h"

namespace croft {

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }


__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)(128 >> 4) << 16;  // leading (K) byte offset between core matrices
    d |= (uint64_t)(512 >> 4) << 32;  // stride (M/N) byte offset between 8-row groups
    d |= (uint64_t)1 << 46;           // descriptor version for sm_100-family
    return d;                         // base offset 0, no swizzle
}

// Operand precision of the tensor-core stage (PassLaunch::tc - 1).
enum TcPrec { TC_BF16X3 = 0, TC_FP16X3 = 1 };

// kind::f16 instruction descriptor: D f32, A and B of one type (bf16: bits 7-9 and 10-12 = 1;
// fp16: 0), both K-major, N = 32, M = 128.
template <int PREC>
__host__ __device__ constexpr uint32_t tc_idesc() {
    return (1u << 4) | (PREC == TC_BF16X3 ? (1u << 7) | (1u << 10) : 0u) | ((32u >> 3) << 17) | ((128u >> 4) << 24);
}

template <int PREC>
__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(tc_idesc<PREC>()), "r"(accumulate));
}

// Split a pair of floats into hi = rn(x) and lo = rn(x - hi) halves of the precision (packed
// two per 32-bit word, the first value in the low half).
template <int PREC>
__device__ __forceinline__ void tc_split2(float a, float b, uint32_t& hi, uint32_t& lo) {
    if constexpr (PREC == TC_BF16X3) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
        hi = *reinterpret_cast<const uint32_t*>(&h);
        lo = *reinterpret_cast<const uint32_t*>(&l);
    } else {
        const __half2 h = __floats2half2_rn(a, b);
        const float2 hf = __half22float2(h);
        const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
        hi = *reinterpret_cast<const uint32_t*>(&h);
        lo = *reinterpret_cast<const uint32_t*>(&l);
    }
}

// Bounded wait for the mbarrier phase with the given parity; false if it never completed.
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity) {
    uint32_t done = 0;
    for (long it = 0; it < (1L << 26) && !done; ++it) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity));
    }
    return done != 0;
}

__device__ __forceinline__ void tc_ld32(uint32_t taddr, float* out) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int i = 0; i < 32; ++i) out[i] = __uint_as_float(r[i]);
}

// Per-CTA tensor-core context.
struct TcCtx {
    unsigned char* abuf;  // A hi (G*8 KB) then A lo (G*8 KB), aliases the pass tile
    uint32_t b_hi;        // shared address of B hi (2 KB) and B lo (+2 KB)
    uint32_t mbar;        // the (first) mbarrier; per-group scope: group g's at mbar + 8 g
    uint32_t tmem;        // TMEM base (lane 0, first column); group g uses columns 32g..32g+31
    int groups;           // blockDim / 128
    int* status;          // device status word (timeout), may be null
    int gstride;          // per-group scope: bytes between the groups' operand buffers in the tile
};

// Synchronisation scope of a tensor-core pass.  GS = false: the CTA (__syncthreads; one thread
// issues every group's MMAs).  GS = true: each 128-thread GEMM group on its own (named barrier
// 1 + g, its own mbarrier, issuer and A operands): row passes whose groups own whole pencils,
// so that one group's MMA round trip overlaps another group's operand preparation.
template <bool GS>
__device__ __forceinline__ void tc_sync(int g) {
    if constexpr (GS) asm volatile("bar.sync %0, 128;" ::"r"(1 + g) : "memory");
    else __syncthreads();
}
template <bool GS>
struct TcBarrier {
    int g;
    __device__ __forceinline__ void operator()() const { tc_sync<GS>(g); }
};

// Radix-16 stage S of the (Tc16Sched) schedule on the tensor cores; at most one butterfly per
// thread (threads past the N/16 butterflies of a pencil contribute zero GEMM rows).
template <class SchedT, int S, int T, int PREC, bool GS, class Src, class Dst>
__device__ __forceinline__ void fft_stage_tc16(const Src& src, const Dst& dst, const float2* stw, int lane, bool ok_pencil,
                                               const TcCtx& tc, uint32_t parity) {
    constexpr int N = SchedT::N;
    constexpr CroftSched sc = SchedT::get();
    static_assert(sc.r[S] == 16, "tensor-core stage must be radix 16");
    constexpr int P = croft_sched_p(sc, S);
    constexpr int NB = N / 16;
    static_assert(NB <= T, "at most one butterfly per thread");
    const int b = lane;
    const bool ok = ok_pencil && (NB == T || b < NB);
    float2 u[16];
    if (ok) {
#pragma unroll
        for (int j = 0; j < 16; ++j) u[j] = src.load(b + j * NB);
        if (P > 1) {
            const int k = b % P;
            const float2* w = stw + (P - 1) + k;
#pragma unroll
            for (int j = 1; j < 16; ++j) u[j] = cmul(u[j], w[(j - 1) * P]);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) u[j] = make_float2(0.f, 0.f);
    }
    const int tid = threadIdx.x;
    const int g = tid >> 7, r = tid & 127;
    // every input of the stage read before the tile becomes the operand buffer (the first stage
    // reads HBM, not the tile: no barrier)
    if constexpr (S != 0) tc_sync<GS>(g);

    // fp16 operands: scale the butterfly by 2^sh so that its largest component lies in
    // [2^14, 2^15) (exact; undone on the outputs below)
    float scale = 1.f, unscale = 1.f;
    if constexpr (PREC == TC_FP16X3) {
        float m = 0.f;
#pragma unroll
        for (int j = 0; j < 16; ++j) m = fmaxf(m, fmaxf(fabsf(u[j].x), fabsf(u[j].y)));
        const int eb = (int)((__float_as_uint(m) >> 23) & 0xff);  // biased exponent of the largest part
        const int sh = min(141 - eb, 126);                         // 14 - (eb - 127), kept representable
        scale = __uint_as_float((uint32_t)(sh + 127) << 23);
        unscale = __uint_as_float((uint32_t)(127 - sh) << 23);
    }
    // A row for this butterfly: k < 16 real parts, k >= 16 imaginary parts; hi and lo halves
    // (per-group operands lie in the group's own part of the tile: tc.gstride bytes apart)
    unsigned char* ahi = GS ? tc.abuf + g * tc.gstride : tc.abuf + g * 8192;
    unsigned char* alo = GS ? ahi + 8192 : tc.abuf + tc.groups * 8192 + g * 8192;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        uint32_t h[4], l[4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            const int k = kk * 8 + e;
            const float x0 = ((k < 16) ? u[k].x : u[k - 16].y) * scale;
            const float x1 = ((k + 1 < 16) ? u[k + 1].x : u[k + 1 - 16].y) * scale;
            tc_split2<PREC>(x0, x1, h[e / 2], l[e / 2]);
        }
        *(uint4*)(ahi + tc_cm_offset(r, kk * 8)) = make_uint4(h[0], h[1], h[2], h[3]);
        *(uint4*)(alo + tc_cm_offset(r, kk * 8)) = make_uint4(l[0], l[1], l[2], l[3]);
    }
    asm volatile("fence.proxy.async.shared::cta;");  // generic-proxy smem writes -> tensor core
    asm volatile("tcgen05.fence::before_thread_sync;");
    tc_sync<GS>(g);
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t mbar = GS ? tc.mbar + 8 * g : tc.mbar;  // (per-group mbarriers 8 bytes apart)
    if (GS ? r == 0 : tid == 0) {
        const uint32_t a_hi = smem_addr(tc.abuf);
        for (int gg = GS ? g : 0; gg < (GS ? g + 1 : tc.groups); ++gg) {
            const uint32_t d = tc.tmem + 32 * gg;
            const uint32_t ah = GS ? a_hi + gg * tc.gstride : a_hi + gg * 8192;
            const uint32_t al = GS ? ah + 8192 : a_hi + tc.groups * 8192 + gg * 8192;
            uint32_t acc = 0;
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {  // K = 32 as two K = 16 steps
                tc_mma<PREC>(d, tc_desc(ah + ks * 256), tc_desc(tc.b_hi + ks * 256), acc);
                acc = 1;
                tc_mma<PREC>(d, tc_desc(ah + ks * 256), tc_desc(tc.b_hi + 2048 + ks * 256), 1);
                tc_mma<PREC>(d, tc_desc(al + ks * 256), tc_desc(tc.b_hi + ks * 256), 1);
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar));
    }
    // one warp (of the group / of the CTA) waits for the MMAs' commit (bounded), the others at
    // the barrier (no polling); the barrier then orders every thread's TMEM reads after the MMAs
    if ((GS ? r : tid) < 32 && !tc_wait(mbar, parity) && tc.status && (GS ? r : tid) == 0)
        atomicExch(tc.status, 5 /* CROFT_ERR_TIMEOUT */);
    tc_sync<GS>(g);
    asm volatile("tcgen05.fence::after_thread_sync;");
    float d[32];
    const int warp = tid >> 5;
    tc_ld32(tc.tmem + 32 * (warp >> 2) + ((uint32_t)((warp & 3) * 32) << 16), d);
    asm volatile("tcgen05.fence::before_thread_sync;");
    if constexpr (PREC == TC_FP16X3) {
#pragma unroll
        for (int i = 0; i < 32; ++i) d[i] *= unscale;
    }
    if (ok) {
        const int k = (P == 1) ? 0 : b % P;
        const int o = (b - k) * 16 + k;
        bool swap = false;
        if constexpr (P == 1 && std::is_same<Dst, SmemCol>::value) swap = dst.W == 8;  // 64-byte rows
        if (swap) {
            // odd butterflies store each output pair (j, j+1) in swapped order, so the rows one
            // store instruction writes alternate between the two bank halves
            const int odd = b & 1;
#pragma unroll
            for (int j = 0; j < 16; j += 2) {
                const float2 v0 = make_float2(d[j], d[16 + j]), v1 = make_float2(d[j + 1], d[17 + j]);
                dst.store(o + odd + j, odd ? v1 : v0);
                dst.store(o + 1 - odd + j, odd ? v0 : v1);
            }
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) dst.store(o + j * P, make_float2(d[j], d[16 + j]));
        }
    }
}

}  // namespace croft

namespace croft {

template <class SchedT, int S>
struct TcStageInfo {
    static constexpr bool tc = S == 0 && SchedT::get().r[S] == 16;
    static constexpr bool first = (S == 0);
    static constexpr bool last = (S == SchedT::get().count - 1);
};

// One stage with the given operands: the first (radix-16) stage on the tensor cores, the others
// on CUDA cores.
template <class SchedT, int S, int T, int PREC, bool GS, class Src, class Dst>
__device__ __forceinline__ void tc_run_stage(const Src& src, const Dst& dst, const float2* stw, int lane, bool ok,
                                             const TcCtx& tc, int tc_index) {
    using I = TcStageInfo<SchedT, S>;
    if constexpr (I::tc) {
        fft_stage_tc16<SchedT, S, T, PREC, GS>(src, dst, stw, lane, ok, tc, (uint32_t)(tc_index & 1));
    } else if constexpr (I::first) {
        fft_stage_s<SchedT, S, T>(src, NoBarrier{}, dst, stw, lane, ok);
    } else {
        fft_stage_s<SchedT, S, T>(src, TcBarrier<GS>{(int)threadIdx.x >> 7}, dst, stw, lane, ok);
    }
}

template <class SchedT, int S, int LAYOUT, int T, int PREC, bool GS>
__device__ __forceinline__ void tc_stages(const float2* gin, float2* gout, float2* tile, const float2* stw,
                                          const PassArgs& A, int c, int lane, bool ok, long long M, const TcCtx& tc,
                                          int tc_index) {
    constexpr int N = SchedT::N;
    using I = TcStageInfo<SchedT, S>;
    if constexpr (LAYOUT == LAYOUT_ROW) {
        const SmemRow sm{tile + c * row_ld(N)};
        if constexpr (I::first && I::last)
            tc_run_stage<SchedT, S, T, PREC, GS>(GlobalInUnit{gin, A.isign}, GlobalOutUnit{gout, A.isign}, stw, lane, ok, tc, tc_index);
        else if constexpr (I::first)
            tc_run_stage<SchedT, S, T, PREC, GS>(GlobalInUnit{gin, A.isign}, sm, stw, lane, ok, tc, tc_index);
        else if constexpr (I::last)
            tc_run_stage<SchedT, S, T, PREC, GS>(sm, GlobalOutUnit{gout, A.isign}, stw, lane, ok, tc, tc_index);
        else
            tc_run_stage<SchedT, S, T, PREC, GS>(sm, sm, stw, lane, ok, tc, tc_index);
    } else {
        const SmemCol sm{tile + c, A.W};
        if constexpr (I::first && I::last)
            tc_run_stage<SchedT, S, T, PREC, GS>(GlobalIn{gin, M, A.isign}, GlobalOut{gout, M, A.isign}, stw, lane, ok, tc, tc_index);
        else if constexpr (I::first)
            tc_run_stage<SchedT, S, T, PREC, GS>(GlobalIn{gin, M, A.isign}, sm, stw, lane, ok, tc, tc_index);
        else if constexpr (I::last)
            tc_run_stage<SchedT, S, T, PREC, GS>(sm, GlobalOut{gout, M, A.isign}, stw, lane, ok, tc, tc_index);
        else
            tc_run_stage<SchedT, S, T, PREC, GS>(sm, sm, stw, lane, ok, tc, tc_index);
    }
    if constexpr (!I::last) {
        tc_sync<GS>((int)threadIdx.x >> 7);
        tc_stages<SchedT, S + 1, LAYOUT, T, PREC, GS>(gin, gout, tile, stw, A, c, lane, ok, M, tc,
                                                      tc_index + (I::tc ? 1 : 0));
    }
}

// Shared memory: [twiddles: tw_pad float2][B operand: 4 KB][tile: the larger of the pass tile
// and blockDim x 128 bytes (the A operands)].  blockDim % 128 == 0.
template <int LAYOUT, int N, int PREC>
__global__ void __launch_bounds__(512) croft_pass_kernel_tc(const float2* in, float2* out,
                                                             const __grid_constant__ PassArgs A) {
    using SchedT = Tc16Sched<N>;
    constexpr int T = croft_threads_per_pencil(N);
    // per-group scope for row passes whose 128-thread groups own whole pencils and whose pencils
    // of one group hold that group's 16 KB of operands (16-byte aligned)
    constexpr int kGroupBytes = (128 / T) * croft_row_ld(N) * (int)sizeof(float2);
    constexpr bool GS = LAYOUT == LAYOUT_ROW && T <= 128 && 128 % T == 0 && kGroupBytes >= 16384 && kGroupBytes % 16 == 0;
    extern __shared__ __align__(16) float2 smem[];
    __shared__ __align__(8) uint64_t mbar[4];
    __shared__ uint32_t tmem_slot;
    float2* stw = smem;
    unsigned char* bmat = (unsigned char*)(smem + A.tw_pad);
    float2* tile = (float2*)(bmat + 4096);
    const int tid = threadIdx.x;
    for (int i = tid; i < N - 1; i += blockDim.x) stw[i] = A.tw[i];
    for (int i = tid; i < 4096 / 16; i += blockDim.x) ((uint4*)bmat)[i] = ((const uint4*)A.tc_b)[i];
    const int groups = blockDim.x >> 7;
    int ncols = 32;
    while (ncols < 32 * groups) ncols <<= 1;
    if (tid == 0) {
        for (int k = 0; k < 4; ++k) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar[k])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (tid < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const TcCtx tc{(unsigned char*)tile, smem_addr(bmat), smem_addr(&mbar[0]), tmem_slot, groups, A.status, kGroupBytes};

    int lane, c;
    long long base, M = 1;
    bool ok;
    if (LAYOUT == LAYOUT_ROW) {
        c = tid / T;
        lane = tid - c * T;
        const long long col = (long long)blockIdx.x * A.W + c;
        ok = col < A.ncols;
        base = (ok ? col : 0) * N;
    } else {
        c = tid % A.W;
        lane = tid / A.W;
        const long long col = (long long)blockIdx.x * A.W + c;
        ok = col < A.ncols;
        M = A.M;
        long long b, m;
        col_split(ok ? col : 0, A, b, m);
        base = b * (long long)N * M + m;
    }
    tc_stages<SchedT, 0, LAYOUT, T, PREC, GS>(in + base, out + base, tile, stw, A, c, lane, ok, M, tc, 0);

    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tc.tmem), "r"(ncols));
}

}  // namespace croft
