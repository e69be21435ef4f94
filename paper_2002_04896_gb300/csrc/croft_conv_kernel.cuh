// croft_conv_kernel.cuh - the reciprocal-space step of PME fused into one pass:
// the last forward 1D FFT, the multiplication by the influence function G and
// the first backward 1D FFT, all along the same axis while the column tile is
// on chip.
//
// Paper mapping.  The paper's application (Sec. 1) is particle-mesh Ewald: the
// charge grid is transformed forward (Eq. 1), multiplied point by point by a
// real influence function and transformed back (Eq. 2, unnormalised here).
// Because the three 1D transforms of a 3D DFT commute (separability, Sec. 2.1),
// the backward transform may start with the axis the forward one ended with.
// Doing both on that axis inside one CTA removes one HBM round trip of the
// grid (the forward pass's write and the backward pass's read) and the
// separate multiply pass; the other axes run as ordinary passes.
//
// Tile: W adjacent columns of the axis (COL layout, croft_internal.h; W fixed per
// length by croft_conv_width), the
// matching W columns of G (real, same layout as the grid) and the twiddles.
// G is copied to shared memory with cp.async at the start, so its latency
// hides behind the forward stages.  The backward transform is conj(F(conj(.))):
// the last forward stage stores conj(G * Y) into the tile, the forward stages
// run again on it, and the final store conjugates.
#pragma once
#include <type_traits>

#include "croft_fft_core.cuh"
#include "croft_internal.h"

namespace croft {

// Store of the last forward stage: element a of this column times G(a), conjugated.
template <class C, int W>
struct ScaleConjCol {
    using value_type = C;
    using R = typename CxScalar<C>::T;
    C* s;        // tile + c
    const R* g;  // G tile + c
    __device__ __forceinline__ void store(int a, C v) const {
        const R ga = g[a * W];
        s[a * W] = mkc<C>(v.x * ga, -(v.y * ga));
    }
};

template <class R>
__device__ __forceinline__ void conv_cp_async(R* dst_smem, const R* src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst_smem);
    if constexpr (sizeof(R) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}

// Launch shape: W = croft_conv_width(N) columns of T threads (a compile-time
// constant, so every shared-memory index folds into constants).  For complex64
// power-of-two lengths with 16-thread pencils (W = 16, 256-thread CTAs), asking
// for four CTAs per SM keeps the kernel at 64 registers (72 at N = 256
// otherwise: three CTAs per SM).  Complex64 pencils of 32 threads make 512-thread
// CTAs whose tiles (data + G, ~100 KB at N = 512) allow two per SM, so they are
// bound to two (64 registers).  Other lengths keep the 128-register bound:
// radix-3/5 stages and complex128 spill at 64.
template <int N, class C>
struct ConvShape {
    static constexpr int T = croft_threads_per_pencil(N);
    static constexpr int W = croft_conv_width(N, (int)sizeof(C));
    static constexpr int THREADS = W * T;
    static constexpr bool TIGHT = sizeof(C) == 8 && THREADS == 256 && T <= 16 && (N & (N - 1)) == 0;
    // 0: no minimum in the launch bound (an explicit minimum of one or two lets ptxas
    // take far more registers than it does without one)
    static constexpr int MIN_BLOCKS = TIGHT ? 4 : ((sizeof(C) == 8 && T == 32) ? 2 : 0);
};

// The last forward stage, the multiply by G and the first backward stage, in registers.
// Valid when the schedule's first and last radices are equal (R): the last stage's
// butterfly b (b < N/R, so k = b) produces outputs b + j*N/R, which are exactly the
// inputs of butterfly b of the first stage of the next transform.  Reads the last
// forward stage's input from `src`, multiplies its outputs by G (from the G tile) and
// conjugates them, applies the first stage of the backward transform (no twiddles)
// and stores its outputs (index b*R + j) to `dst`.  `mid` separates all reads from
// the stores (and publishes the G copies).
template <class SchedT, int T, int W, class Src, class Mid, class Dst, class R>
__device__ __forceinline__ void conv_middle(const Src& src, const Mid& mid, const Dst& dst, const R* gcol,
                                            const typename Src::value_type* stw, int lane, bool ok) {
    using C = typename Src::value_type;
    constexpr int N = SchedT::N;
    constexpr CroftSched sc = SchedT::get();
    constexpr int S = sc.count - 1;
    constexpr int RAD = sc.r[S];
    constexpr int P = croft_sched_p(sc, S);
    constexpr int NB = N / RAD;
    static_assert(sc.r[0] == RAD && P == NB, "first and last radix must agree");
    constexpr int QM = (NB + T - 1) / T;
    C v[QM][RAD];
#pragma unroll
    for (int q = 0; q < QM; ++q) {
        const int b = lane + q * T;
        if (ok && (NB % T == 0 || b < NB)) {
#pragma unroll
            for (int j = 0; j < RAD; ++j) v[q][j] = src.load(b + j * NB);
        }
    }
    mid();
#pragma unroll
    for (int q = 0; q < QM; ++q) {
        const int b = lane + q * T;
        if (ok && (NB % T == 0 || b < NB)) {
            if (P > 1) {
                const C* w = stw + (P - 1) + b;
#pragma unroll
                for (int j = 1; j < RAD; ++j) v[q][j] = cmul(v[q][j], w[(j - 1) * P]);
            }
            dft<RAD>(v[q]);
#pragma unroll
            for (int j = 0; j < RAD; ++j) {
                const R ga = gcol[(b + j * P) * W];
                v[q][j] = mkc<C>(v[q][j].x * ga, -(v[q][j].y * ga));
            }
            dft<RAD>(v[q]);
#pragma unroll
            for (int j = 0; j < RAD; ++j) dst.store(b * RAD + j, v[q][j]);
        }
    }
}

// The schedule of the fused pass: the column passes' (croft_pass_sched).
template <int N, class C>
struct ConvSched {
    static constexpr int N_ = N;
    static constexpr bool even = croft_even_pow2_pass(N, LAYOUT_COL, (int)sizeof(C));
};
template <int N, class C>
using ConvSchedT = typename std::conditional<ConvSched<N, C>::even, EvenPow2Sched<N>, DefaultSched<N>>::type;

template <class SchedT>
constexpr bool conv_fuses_middle() {
    return SchedT::get().count >= 1 && SchedT::get().r[0] == SchedT::get().r[SchedT::get().count - 1];
}

// Shared memory: [twiddles: tw_pad][tile: N x W complex][G tile: N x W real].
template <int N, class C>
__device__ __forceinline__ void conv_body(const C* in, C* out, const typename CxScalar<C>::T* g, const PassArgs& A) {
    using R = typename CxScalar<C>::T;
    constexpr int T = ConvShape<N, C>::T;
    constexpr int W = ConvShape<N, C>::W;
    using CS = ConvSchedT<N, C>;
    constexpr CroftSched sc = CS::get();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* stw = reinterpret_cast<C*>(smem_raw);
    C* tile = stw + A.tw_pad;
    R* gtile = reinterpret_cast<R*>(tile + (long long)N * W);
    const C* twg;
    if constexpr (sizeof(C) == 16) twg = A.tw64;
    else twg = A.tw;

    const int c = threadIdx.x % W;
    const int lane = threadIdx.x / W;
    const long long col = (long long)blockIdx.x * W + c;
    const bool ok = col < A.ncols;
    long long b, m;
    col_split(col, A, b, m);
    const long long base = b * (long long)N * A.M + m;

    pdl_allow_dependents();
    if (ok)
        for (int a = lane; a < N; a += T) conv_cp_async(gtile + a * W + c, g + base + (long long)a * A.M);
    asm volatile("cp.async.commit_group;" ::: "memory");
    if (sc.count > 1)
        for (int i = threadIdx.x; i < N - 1; i += blockDim.x) stw[i] = twg[i];
    pdl_wait();  // (G and the twiddles are not written by the previous pass)

    const GlobalInT<C> src{in + base, A.M, 1.f};
    const SmemColFixed<C, W> work{tile + c};
    const ScaleConjCol<C, W> scaled{tile + c, gtile + c};
    const GlobalOutT<C> dst{out + base, A.M, -1.f};

    if constexpr (conv_fuses_middle<CS>()) {
        // forward stages but the last; the last, G and the first backward stage in registers
        // (conv_middle); the remaining backward stages
        if constexpr (sc.count == 1) {
            asm volatile("cp.async.wait_all;" ::: "memory");
            conv_middle<CS, T, W>(src, CtaBarrier{}, dst, gtile + c, stw, lane, ok);
        } else {
            fft_stage_s<CS, 0, T>(src, NoBarrier{}, work, stw, lane, ok);
            __syncthreads();
            smem_stages_s<CS, 1, sc.count - 1, T>(work, stw, lane, ok);
            asm volatile("cp.async.wait_all;" ::: "memory");
            conv_middle<CS, T, W>(work, CtaBarrier{}, work, gtile + c, stw, lane, ok);
            __syncthreads();
            smem_stages_s<CS, 1, sc.count - 1, T>(work, stw, lane, ok);
            fft_stage_s<CS, sc.count - 1, T>(work, NoBarrier{}, dst, stw, lane, ok);
        }
        return;
    }
    // forward transform of the column; its last stage leaves conj(G * Y) in the tile.
    // (The barrier inside the last stage also publishes every thread's G copies.)
    if constexpr (sc.count == 1) {
        asm volatile("cp.async.wait_all;" ::: "memory");
        fft_stage_s<CS, 0, T>(src, CtaBarrier{}, scaled, stw, lane, ok);
    } else {
        fft_stage_s<CS, 0, T>(src, NoBarrier{}, work, stw, lane, ok);
        __syncthreads();
        smem_stages_s<CS, 1, sc.count - 1, T>(work, stw, lane, ok);
        asm volatile("cp.async.wait_all;" ::: "memory");
        fft_stage_s<CS, sc.count - 1, T>(work, CtaBarrier{}, scaled, stw, lane, ok);
    }
    __syncthreads();
    // backward transform along the same axis: forward stages on the conjugated tile, conjugated store
    if constexpr (sc.count == 1) {
        fft_stage_s<CS, 0, T>(work, NoBarrier{}, dst, stw, lane, ok);
    } else {
        fft_stage_s<CS, 0, T>(work, CtaBarrier{}, work, stw, lane, ok);
        __syncthreads();
        smem_stages_s<CS, 1, sc.count - 1, T>(work, stw, lane, ok);
        fft_stage_s<CS, sc.count - 1, T>(work, NoBarrier{}, dst, stw, lane, ok);
    }
}

template <int N, class C = float2>
__global__ void __launch_bounds__(ConvShape<N, C>::THREADS)
    croft_conv_kernel(const C* in, C* out, const typename CxScalar<C>::T* g, const __grid_constant__ PassArgs A) {
    conv_body<N, C>(in, out, g, A);
}

template <int N, class C = float2>
__global__ void __launch_bounds__(ConvShape<N, C>::THREADS, ConvShape<N, C>::MIN_BLOCKS > 0 ? ConvShape<N, C>::MIN_BLOCKS : 1)
    croft_conv_kernel_bounded(const C* in, C* out, const typename CxScalar<C>::T* g, const __grid_constant__ PassArgs A) {
    conv_body<N, C>(in, out, g, A);
}

// The kernel of length N: bounded when ConvShape asks for a minimum of CTAs per SM.
template <int N, class C>
constexpr auto conv_kernel_of() {
    if constexpr (ConvShape<N, C>::MIN_BLOCKS > 0) return croft_conv_kernel_bounded<N, C>;
    else return croft_conv_kernel<N, C>;
}

// out[i] = in[i] * g[i] (the multiply on its own, for plans whose last pass cannot
// take it: a grid of one point, a last pass that is a fused plane or a
// tensor-core pass).  Grid-stride loop.
template <class C>
__global__ void croft_scale_kernel(const C* in, C* out, const typename CxScalar<C>::T* g, long long n) {
    pdl_allow_dependents();
    pdl_wait();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const C v = in[i];
        const typename CxScalar<C>::T s = g[i];
        out[i] = mkc<C>(v.x * s, v.y * s);
    }
}

}  // namespace croft
