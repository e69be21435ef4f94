// croft_kernels64.cu - complex128 instantiations of the pass kernel.
//
// Double precision is the paper's own precision (Sec. 5: double complex data).
// On GB300 the FP64 units are a small fraction of the FP32 ones, so these
// passes are arithmetic-bound rather than HBM-bound; they exist for the
// paper's accuracy and for a like-for-like comparison with its FFTW3-based
// double-complex runs, not as a fast path.  Lengths: every power of two up to
// 1024 and a few mixed-radix ones.
#include "croft_pass_kernel.cuh"
#include "croft_sizes.h"

namespace croft {

template <int N>
static pass64_fn col64_kernel(int w) {
    constexpr int W = croft_col_width(N, 16);
    return (w == W || w == 0) ? croft_pass_kernel<LAYOUT_COL, N, double2, W> : nullptr;
}

pass64_fn pass64_kernel_for(int layout, int n, int w) {
#define CROFT_CASE64(N)                                                                 \
    case N:                                                                             \
        return layout == LAYOUT_ROW ? croft_pass_kernel<LAYOUT_ROW, N, double2> : col64_kernel<N>(w);
    switch (n) {
        CROFT_SIZES64(CROFT_CASE64)
        default: return nullptr;
    }
#undef CROFT_CASE64
}

}  // namespace croft
