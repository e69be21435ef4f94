// croft_kernels.cu - instantiates the pass kernel for one group of axis lengths.
// Compiled once per group (-DCROFT_GROUP=0..3) so the instantiations build in parallel.
#include "croft_pass_kernel.cuh"
#include "croft_sizes.h"

#ifndef CROFT_GROUP
#error "compile with -DCROFT_GROUP=<0..3>"
#endif

#define CROFT_CAT_(a, b) a##b
#define CROFT_CAT(a, b) CROFT_CAT_(a, b)

namespace croft {

// One COL kernel per length: tile width croft_col_width, launch bound croft_col_minb;
// lengths of 32-thread pencils add the narrow short-stride kernel (croft_col_width_at) and,
// for tuned plans, both widths with the other schedule variant (sv = 1).
// w: the width asked for (nullptr when no kernel is built for it).
template <int N>
static pass_fn col_kernel(int w, int sv, int th) {
    constexpr int W = croft_col_width(N, 8);
    // 24 threads per pencil (croft_col_t24): 192-thread narrow CTAs, six per SM; 384-thread
    // 16-column CTAs, three per SM (56 registers both)
    if (th == 24) {
        if constexpr (croft_threads_per_pencil(N) == 32 && croft_col_t24(N, true))
            if (w == kColNarrowWidth)
                return sv ? croft_pass_kernel_bounded<LAYOUT_COL, N, float2, kColNarrowWidth, 6, kColNarrowWidth * 24, 1, 24>
                          : croft_pass_kernel_bounded<LAYOUT_COL, N, float2, kColNarrowWidth, 6, kColNarrowWidth * 24, 0, 24>;
        if constexpr (croft_threads_per_pencil(N) == 32 && croft_col_t24(N, false) && W == 16)
            if (w == 16)
                return sv ? croft_pass_kernel_bounded<LAYOUT_COL, N, float2, 16, 3, 16 * 24, 1, 24>
                          : croft_pass_kernel_bounded<LAYOUT_COL, N, float2, 16, 3, 16 * 24, 0, 24>;
        return nullptr;
    }
    if constexpr (croft_threads_per_pencil(N) == 32 && W != kColNarrowWidth) {
        // 16 threads per pencil (32 elements each): 256-thread CTAs of 16 columns, three per SM
        if (th == 16 && w == W)
            return sv ? croft_pass_kernel_bounded<LAYOUT_COL, N, float2, W, 3, W * 16, 1, 16>
                      : croft_pass_kernel_bounded<LAYOUT_COL, N, float2, W, 3, W * 16, 0, 16>;
        if (th) return nullptr;
        if constexpr (N == 512)
            if (w == kColNarrowWidth && sv == 2)
                return croft_pass_kernel_bounded<LAYOUT_COL, N, float2, kColNarrowWidth, croft_col_narrow_minb(N),
                                                 kColNarrowWidth * 32, 2>;
        if (w == kColNarrowWidth)
            return sv ? croft_pass_kernel_bounded<LAYOUT_COL, N, float2, kColNarrowWidth, croft_col_narrow_minb(N),
                                                  kColNarrowWidth * 32, 1>
                      : croft_pass_kernel_bounded<LAYOUT_COL, N, float2, kColNarrowWidth, croft_col_narrow_minb(N),
                                                  kColNarrowWidth * 32>;
        if (w == W && sv) return croft_pass_kernel_bounded<LAYOUT_COL, N, float2, W, croft_col_minb(N, 8), 512, 1>;
    }
    if (w != W || sv || th) return nullptr;
    if constexpr (croft_col_minb(N, 8) > 1) return croft_pass_kernel_bounded<LAYOUT_COL, N, float2, W, croft_col_minb(N, 8)>;
    else if constexpr (croft_pass_minb(N, 8) > 0)
        return croft_pass_kernel_bounded<LAYOUT_COL, N, float2, W, croft_pass_minb(N, 8), 256>;
    else return croft_pass_kernel<LAYOUT_COL, N, float2, W>;
}

template <int N>
static pass_fn row_kernel() {
    if constexpr (croft_pass_minb(N, 8) > 0) return croft_pass_kernel_bounded<LAYOUT_ROW, N, float2, 0, croft_pass_minb(N, 8), 256>;
    else return croft_pass_kernel<LAYOUT_ROW, N>;
}

pass_fn CROFT_CAT(lookup_pass_kernel_group_, CROFT_GROUP)(int layout, int n, int w, int sv, int th) {
#define CROFT_CASE(N) \
    case N: return layout == LAYOUT_ROW ? ((sv || th) ? nullptr : row_kernel<N>()) : col_kernel<N>(w, sv, th);
    switch (n) {
        CROFT_CAT(CROFT_SIZES_, CROFT_GROUP)(CROFT_CASE)
        default: return nullptr;
    }
#undef CROFT_CASE
}

}  // namespace croft
