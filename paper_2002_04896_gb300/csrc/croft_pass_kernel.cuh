// croft_pass_kernel.cuh - one pass = a batched 1D FFT over all pencils of one axis.
//
// Paper mapping (Sec. 4.1): steps 1, 5 and 9 are the per-axis batched 1D FFTs;
// steps 2-4 and 6-8 (pack, all-to-all, unpack) only exist to make the next
// axis local to a process.  On one GPU every axis is addressable, so the
// rearrangement is fused into the FFT pass itself: a CTA gathers W whole
// pencils of a strided axis straight from HBM (W consecutive columns, i.e.
// W*8-byte contiguous row segments), transforms them on chip and writes them
// back to the same place.  The grid therefore stays in its natural layout
// between passes and after the last one (the paper's closing transposes,
// Sec. 4.2, are not needed).
//
// Inside a CTA each pencil is transformed with the Stockham auto-sort
// formulation: stage s with radix R combines R sub-transforms of length p
// into one of length pR.  Butterfly b (0 <= b < n/R), k = b mod p, reads
// x[b + j*n/R] (j = 0..R-1), multiplies input j by w_{pR}^{jk}, applies the
// radix-R DFT and writes output j to y[(b-k)*R + k + j*p].  The first stage
// reads HBM straight into registers and the last stage writes HBM straight
// from registers (unit-stride lanes in both cases); the stages in between
// exchange through shared memory in place.  Kernels are specialised on n, so
// the radix schedule, strides and twiddle offsets are compile-time constants.
#pragma once
#include "croft_fft_core.cuh"
#include "croft_internal.h"

namespace croft {

// Shared memory: [twiddles: tw_pad elements][tile: W pencils].  C = float2
// (complex64, the default) or double2 (complex128, twiddles from A.tw64).
// COL kernels are specialised on the column-tile width WC as well (so the
// shared-memory indices fold into constants); ROW kernels take W from A.W.
template <int LAYOUT, int N, class C, int WC, int SV = 0, int TH = 0>
__device__ __forceinline__ void pass_body(const C* in, C* out, const PassArgs& A) {
    constexpr int T = TH > 0 ? TH : croft_threads_per_pencil(N);  // TH: threads per pencil, if not the rule's
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* smem = reinterpret_cast<C*>(smem_raw);
    C* stw = smem;
    C* sbuf = smem + A.tw_pad;
    const C* twg;
    if constexpr (sizeof(C) == 16) twg = A.tw64;
    else twg = A.tw;
    pdl_allow_dependents();
    if (croft_make_sched(N).count > 1)
        for (int i = threadIdx.x; i < N - 1; i += blockDim.x) stw[i] = twg[i];
    pdl_wait();

    if (LAYOUT == LAYOUT_ROW) {
        const int c = threadIdx.x / T;
        const int lane = threadIdx.x - c * T;
        const long long col = (long long)blockIdx.x * A.W + c;
        const bool ok = col < A.ncols;
        const long long base = col * N;
        fft_pencil_row<N, T>(GlobalInUnitT<C>{in + base, A.isign}, sbuf + c * croft_row_ld_staged(N),
                             GlobalOutUnitT<C>{out + base, A.isign}, stw, lane, ok);
    } else {
        static_assert(LAYOUT == LAYOUT_ROW || WC > 0, "COL kernels need a compile-time tile width");
        const int c = threadIdx.x % WC;
        const int lane = threadIdx.x / WC;
        const long long col = (long long)blockIdx.x * WC + c;
        const bool ok = col < A.ncols;
        long long b, m;
        col_split(col, A, b, m);
        const long long base = b * (long long)N * A.M + m;
        const GlobalInT<C> src{in + base, A.M, A.isign};
        const SmemColFixed<C, (WC > 0 ? WC : 1)> work{sbuf + c};
        const GlobalOutT<C> dst{out + base, A.M, A.isign};
        // the column schedule (croft_pass_sched_v: SV = 1 the radix-16-first variant, SV = 2 one
        // radix-16 stage then the near-equal split)
        if constexpr (SV == 2)
            fft_pencil_s<Mixed16Sched<N>, T>(src, work, dst, stw, lane, ok);
        else if constexpr (SV == 0 && croft_even_pow2_pass(N, LAYOUT_COL, (int)sizeof(C)))
            fft_pencil_s<EvenPow2Sched<N>, T>(src, work, dst, stw, lane, ok);
        else
            fft_pencil<N, T>(src, work, dst, stw, lane, ok);
    }
}

// The pass kernel.  (Its launch bound names no minimum of CTAs per SM: with an
// explicit minimum of one, ptxas allocates far more registers - 83 instead of 52
// for the 256-point COL kernel - and the pass slows from 46 to 60 us.)
template <int LAYOUT, int N, class C = float2, int WC = 0>
__global__ void __launch_bounds__(512) croft_pass_kernel(const C* in, C* out, const __grid_constant__ PassArgs A) {
    pass_body<LAYOUT, N, C, WC>(in, out, A);
}

// The same with registers bounded for MINB CTAs of MAXT threads per SM (croft_col_minb,
// croft_pass_minb); SV selects the schedule variant (croft_pass_sched_v).
template <int LAYOUT, int N, class C, int WC, int MINB, int MAXT = 512, int SV = 0, int TH = 0>
__global__ void __launch_bounds__(MAXT, MINB) croft_pass_kernel_bounded(const C* in, C* out,
                                                                         const __grid_constant__ PassArgs A) {
    pass_body<LAYOUT, N, C, WC, SV, TH>(in, out, A);
}

}  // namespace croft
