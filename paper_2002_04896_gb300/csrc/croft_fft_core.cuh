// croft_fft_core.cuh - one Stockham stage of a length-N FFT, with pluggable operand access.
//
// Stage S of the length-N schedule (radix R = sched.r[S], sub-transform length
// P = product of the earlier radices) on one pencil: butterfly b in
// [0, N/R), k = b mod P, reads x[b + j*N/R] (j = 0..R-1), multiplies input j
// by w_{PR}^{jk} (table entry P-1 + (j-1)*P + k), applies the radix-R DFT and
// writes output j to y[(b-k)*R + k + j*P].  After the last stage the pencil is
// in natural order (Stockham auto-sort).
//
// Where x and y live is up to the caller: `Src::load(a)` / `Dst::store(a, v)`
// address element a of this thread's pencil in HBM, in this CTA's shared
// memory, or in another CTA's shared memory of the same cluster.  `Mid` is the
// barrier between the reads and the writes of the stage (needed when the
// writes overwrite data other threads still have to read).
#pragma once
#include <type_traits>
#include <cooperative_groups.h>

#include "croft_butterflies.cuh"
#include "croft_sched.h"

namespace croft {

// ---------------------------------------------------------------------------
// operand accessors
// ---------------------------------------------------------------------------

// Accessors are templates on the complex type C (float2 or double2); the
// float2 names below are the complex64 instances.

// Pencil in HBM with element stride `stride`; conj() on the way in/out when isign = -1.
template <class C>
struct GlobalInT {
    using value_type = C;
    const C* p;
    long long stride;
    float isign;
    __device__ __forceinline__ C load(int a) const {
        C t = p[(long long)a * stride];
        t.y *= isign;
        return t;
    }
};
template <class C>
struct GlobalInUnitT {  // unit stride (contiguous pencil)
    using value_type = C;
    const C* p;
    float isign;
    __device__ __forceinline__ C load(int a) const {
        C t = p[a];
        t.y *= isign;
        return t;
    }
};
// As GlobalIn, but read through L2 only (ld.global.cg): for data another CTA
// wrote earlier in the same launch (the batched persistent kernel).
struct GlobalInCG {
    using value_type = float2;
    const float2* p;
    long long stride;
    float isign;
    __device__ __forceinline__ float2 load(int a) const {
        float2 t = __ldcg(p + (long long)a * stride);
        t.y *= isign;
        return t;
    }
};
template <class C>
struct GlobalOutT {
    using value_type = C;
    C* p;
    long long stride;
    float isign;
    __device__ __forceinline__ void store(int a, C v) const {
        v.y *= isign;
        p[(long long)a * stride] = v;
    }
};
template <class C>
struct GlobalOutUnitT {
    using value_type = C;
    C* p;
    float isign;
    __device__ __forceinline__ void store(int a, C v) const {
        v.y *= isign;
        p[a] = v;
    }
};
using GlobalIn = GlobalInT<float2>;
using GlobalInUnit = GlobalInUnitT<float2>;
using GlobalOut = GlobalOutT<float2>;
using GlobalOutUnit = GlobalOutUnitT<float2>;

// Row-major pencil in shared memory, one pad slot per 16 elements (conflict-free
// for the stride-R writes of the early stages).
__host__ __device__ constexpr int row_ld(int n) { return croft_row_ld(n); }
struct SmemRow {
    using value_type = float2;
    float2* s;  // start of this pencil
    __device__ __forceinline__ float2 load(int a) const { return s[a + (a >> 4)]; }
    __device__ __forceinline__ void store(int a, float2 v) const { s[a + (a >> 4)] = v; }
};
// Row pencil stored with the padding of one stage's output (croft_row_layouts.h).
template <int L, int D, class C = float2>
struct SmemRowP {
    using value_type = C;
    C* s;
    __device__ __forceinline__ int idx(int a) const { return D == 0 ? a : a + (a / L) * D; }
    __device__ __forceinline__ C load(int a) const { return s[idx(a)]; }
    __device__ __forceinline__ void store(int a, C v) const { s[idx(a)] = v; }
};
// Column c of a [N][W] tile (W pencils side by side).
template <class C>
struct SmemColT {
    using value_type = C;
    C* s;  // tile + c
    int W;
    __device__ __forceinline__ C load(int a) const { return s[a * W]; }
    __device__ __forceinline__ void store(int a, C v) const { s[a * W] = v; }
};
using SmemCol = SmemColT<float2>;
// The same with a compile-time width (the index arithmetic folds into constants).
template <class C, int W>
struct SmemColFixed {
    using value_type = C;
    // Rows of 64 bytes cover half of the banks: a first stage with an even radix R0 then
    // writes rows R0*b + j of consecutive butterflies b all on one half, unless odd
    // butterflies store their pairs of outputs in swapped order (fft_stage_s).
    static constexpr bool kPairSwap = W * (int)sizeof(C) == 64;
    C* s;  // tile + c
    __device__ __forceinline__ C load(int a) const { return s[a * W]; }
    __device__ __forceinline__ void store(int a, C v) const { s[a * W] = v; }
};

// ---------------------------------------------------------------------------
// programmatic dependent launch
// ---------------------------------------------------------------------------
// Passes after the first of an exec are launched with programmatic stream
// serialisation: their CTAs may become resident while the previous pass drains.
// Every such kernel loads what the previous pass does not write (twiddles, the
// influence function), then waits here for the previous grid to complete and its
// writes to become visible, before it reads the grid.  Without the launch
// attribute both instructions return at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_allow_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---------------------------------------------------------------------------
// barriers
// ---------------------------------------------------------------------------
struct NoBarrier {
    __device__ __forceinline__ void operator()() const {}
};
struct CtaBarrier {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

// ---------------------------------------------------------------------------
// schedules (which radix each stage of a length-N transform uses)
// ---------------------------------------------------------------------------
template <int N_>
struct DefaultSched {
    static constexpr int N = N_;
    __host__ __device__ static constexpr CroftSched get() { return croft_make_sched(N_); }
};
template <int N_>
struct EvenPow2Sched {  // the near-equal power-of-two split (croft_pass_sched)
    static constexpr int N = N_;
    __host__ __device__ static constexpr CroftSched get() { return croft_make_sched(N_, true); }
};
template <int N_>
struct Mixed16Sched {  // one radix-16 stage, then the near-equal split of the rest
    static constexpr int N = N_;
    __host__ __device__ static constexpr CroftSched get() { return croft_make_sched_mixed(N_); }
};
template <int N_>
struct Tc16Sched {
    static constexpr int N = N_;
    __host__ __device__ static constexpr CroftSched get() { return croft_make_sched_tc(N_); }
};

// ---------------------------------------------------------------------------
// the stage
// ---------------------------------------------------------------------------
// Whether a destination wants the pair-swapped store order of a first stage (kPairSwap).
template <class D, class = void>
struct PairSwapStores : std::false_type {};
template <class D>
struct PairSwapStores<D, std::void_t<decltype(D::kPairSwap)>> : std::bool_constant<D::kPairSwap> {};

template <class SchedT, int S, int T, class Src, class Mid, class Dst>
__device__ __forceinline__ void fft_stage_s(const Src& src, const Mid& mid, const Dst& dst,
                                            const typename Src::value_type* stw, int lane, bool ok) {
    using C = typename Src::value_type;
    constexpr int N = SchedT::N;
    constexpr CroftSched sc = SchedT::get();
    constexpr int R = sc.r[S];
    constexpr int P = croft_sched_p(sc, S);
    constexpr int NB = N / R;
    constexpr int QM = (NB + T - 1) / T;
    C v[QM][R];
#pragma unroll
    for (int q = 0; q < QM; ++q) {
        const int b = lane + q * T;
        if (ok && (NB % T == 0 || b < NB)) {
#pragma unroll
            for (int j = 0; j < R; ++j) v[q][j] = src.load(b + j * NB);
        }
    }
    mid();
#pragma unroll
    for (int q = 0; q < QM; ++q) {
        const int b = lane + q * T;
        if (ok && (NB % T == 0 || b < NB)) {
            const int k = (P == 1) ? 0 : b % P;
            if (P > 1) {
                const C* w = stw + (P - 1) + k;
#pragma unroll
                for (int j = 1; j < R; ++j) v[q][j] = cmul(v[q][j], w[(j - 1) * P]);
            }
            dft<R>(v[q]);
            const int o = (b - k) * R + k;
            if constexpr (P == 1 && R % 2 == 0 && PairSwapStores<Dst>::value) {
                // same stores, odd butterflies take each pair (j, j+1) in swapped order: the
                // rows one instruction writes then alternate between the two bank halves
                const int odd = b & 1;
#pragma unroll
                for (int j = 0; j < R; j += 2) {
                    const C first = odd ? v[q][j + 1] : v[q][j];
                    const C second = odd ? v[q][j] : v[q][j + 1];
                    dst.store(o + odd + j, first);
                    dst.store(o + 1 - odd + j, second);
                }
            } else {
#pragma unroll
                for (int j = 0; j < R; ++j) dst.store(o + j * P, v[q][j]);
            }
        }
    }
}

template <int N, int S, int T, class Src, class Mid, class Dst>
__device__ __forceinline__ void fft_stage(const Src& src, const Mid& mid, const Dst& dst,
                                          const typename Src::value_type* stw, int lane, bool ok) {
    fft_stage_s<DefaultSched<N>, S, T>(src, mid, dst, stw, lane, ok);
}

// Stages [S, E) of a length-N FFT entirely in shared memory (in place), each
// followed by a CTA barrier.  `Sm` is SmemRow or SmemCol.
template <int N, int S, int E, int T, class Sm>
__device__ __forceinline__ void smem_stages(const Sm& sm, const typename Sm::value_type* stw, int lane, bool ok) {
    if constexpr (S < E) {
        fft_stage<N, S, T>(sm, CtaBarrier{}, sm, stw, lane, ok);
        __syncthreads();
        smem_stages<N, S + 1, E, T>(sm, stw, lane, ok);
    }
}

// A full length-N FFT of one pencil per thread group: first stage src -> work
// (shared memory), inner stages in `work`, last stage work -> dst.  With a
// single-stage schedule src -> dst directly.  `work` must not alias src/dst.
// Ends without a trailing barrier when dst is not shared memory.
template <int N, int T, class Src, class Sm, class Dst>
__device__ __forceinline__ void fft_pencil(const Src& src, const Sm& work, const Dst& dst,
                                           const typename Src::value_type* stw, int lane, bool ok) {
    constexpr CroftSched sc = croft_make_sched(N);
    if constexpr (sc.count == 1) {
        fft_stage<N, 0, T>(src, NoBarrier{}, dst, stw, lane, ok);
    } else {
        fft_stage<N, 0, T>(src, NoBarrier{}, work, stw, lane, ok);
        __syncthreads();
        smem_stages<N, 1, sc.count - 1, T>(work, stw, lane, ok);
        fft_stage<N, sc.count - 1, T>(work, NoBarrier{}, dst, stw, lane, ok);
    }
}

// smem_stages / fft_pencil for an explicit schedule type (SchedT::N, SchedT::get()).
template <class SchedT, int S, int E, int T, class Sm>
__device__ __forceinline__ void smem_stages_s(const Sm& sm, const typename Sm::value_type* stw, int lane, bool ok) {
    if constexpr (S < E) {
        fft_stage_s<SchedT, S, T>(sm, CtaBarrier{}, sm, stw, lane, ok);
        __syncthreads();
        smem_stages_s<SchedT, S + 1, E, T>(sm, stw, lane, ok);
    }
}
template <class SchedT, int T, class Src, class Sm, class Dst>
__device__ __forceinline__ void fft_pencil_s(const Src& src, const Sm& work, const Dst& dst,
                                             const typename Src::value_type* stw, int lane, bool ok) {
    constexpr CroftSched sc = SchedT::get();
    if constexpr (sc.count == 1) {
        fft_stage_s<SchedT, 0, T>(src, NoBarrier{}, dst, stw, lane, ok);
    } else {
        fft_stage_s<SchedT, 0, T>(src, NoBarrier{}, work, stw, lane, ok);
        __syncthreads();
        smem_stages_s<SchedT, 1, sc.count - 1, T>(work, stw, lane, ok);
        fft_stage_s<SchedT, sc.count - 1, T>(work, NoBarrier{}, dst, stw, lane, ok);
    }
}

// Padding of the buffer written by stage S of the length-N schedule.
template <int N, int S, class C = float2>
struct RowPadOf {
    static constexpr int L = croft_row_layout(N).L[S];
    static constexpr int D = croft_row_layout(N).D[S];
    using type = SmemRowP<L, D, C>;
};

// Stages [S, E) of a length-N row transform in shared memory: stage S reads the
// layout of stage S-1's output and writes its own layout (in place, the data
// passes through registers between the two barriers).
template <int N, int S, int E, int T, class C>
__device__ __forceinline__ void row_stages(C* base, const C* stw, int lane, bool ok) {
    if constexpr (S < E) {
        const typename RowPadOf<N, S - 1, C>::type src{base};
        const typename RowPadOf<N, S, C>::type dst{base};
        fft_stage<N, S, T>(src, CtaBarrier{}, dst, stw, lane, ok);
        __syncthreads();
        row_stages<N, S + 1, E, T>(base, stw, lane, ok);
    }
}

// A full length-N FFT of one row pencil: stage 0 src -> shared memory (pencil
// base `base`, stride croft_row_ld_staged(N) between pencils), inner stages in
// place, last stage -> dst.  Ends without a trailing barrier.
template <int N, int T, class Src, class Dst>
__device__ __forceinline__ void fft_pencil_row(const Src& src, typename Src::value_type* base, const Dst& dst,
                                               const typename Src::value_type* stw, int lane, bool ok) {
    using C = typename Src::value_type;
    constexpr CroftSched sc = croft_make_sched(N);
    if constexpr (sc.count == 1) {
        fft_stage<N, 0, T>(src, NoBarrier{}, dst, stw, lane, ok);
    } else {
        const typename RowPadOf<N, 0, C>::type w0{base};
        fft_stage<N, 0, T>(src, NoBarrier{}, w0, stw, lane, ok);
        __syncthreads();
        row_stages<N, 1, sc.count - 1, T>(base, stw, lane, ok);
        const typename RowPadOf<N, sc.count - 2, C>::type wl{base};
        fft_stage<N, sc.count - 1, T>(wl, NoBarrier{}, dst, stw, lane, ok);
    }
}

}  // namespace croft
