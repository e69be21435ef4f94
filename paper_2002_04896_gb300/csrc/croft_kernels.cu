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

// COL kernels exist for the two tile widths the planner can pick (croft_col_width with
// close or distant rows; one kernel when they agree).  w: the width asked for.
template <int N>
static pass_fn col_kernel(int w) {
    constexpr int W_NEAR = croft_col_width(N, 8, true);
    constexpr int W_FAR = croft_col_width(N, 8, false);
    if (w == W_FAR) return croft_pass_kernel<LAYOUT_COL, N, float2, W_FAR>;
    if (w == W_NEAR) return croft_pass_kernel<LAYOUT_COL, N, float2, W_NEAR>;
    return nullptr;
}

pass_fn CROFT_CAT(lookup_pass_kernel_group_, CROFT_GROUP)(int layout, int n, int w) {
#define CROFT_CASE(N) \
    case N: return layout == LAYOUT_ROW ? croft_pass_kernel<LAYOUT_ROW, N> : col_kernel<N>(w);
    switch (n) {
        CROFT_CAT(CROFT_SIZES_, CROFT_GROUP)(CROFT_CASE)
        default: return nullptr;
    }
#undef CROFT_CASE
}

}  // namespace croft
