// croft_tc.cu - instantiations of the tensor-core pass kernel and the DFT-16 operand.
#include <math.h>
#include <string.h>

#include "croft_tc_kernel.cuh"
#include "croft_tc_operand.h"

namespace croft {

// Every length <= 1024 with a factor 16 (a radix-16 stage) and 2^a 3^b 5^c: the tensor-core
// stages need at most one butterfly per thread (N / 16 <= threads per pencil), which holds up
// to 1024 points.  Compiled in four groups (-DCROFT_TC_GROUP=0..3) so they build in parallel.
#define CROFT_TC_SIZES_0(X) X(16) X(80) X(160) X(288) X(432) X(640) X(864)
#define CROFT_TC_SIZES_1(X) X(32) X(96) X(192) X(320) X(480) X(720) X(960)
#define CROFT_TC_SIZES_2(X) X(48) X(128) X(240) X(384) X(512) X(768) X(1024)
#define CROFT_TC_SIZES_3(X) X(64) X(144) X(256) X(400) X(576) X(800)

#ifdef CROFT_TC_GROUP
#define CROFT_TCAT_(a, b) a##b
#define CROFT_TCAT(a, b) CROFT_TCAT_(a, b)

pass_fn CROFT_TCAT(lookup_tc_kernel_group_, CROFT_TC_GROUP)(int layout, int n, int prec) {
#define CROFT_TC_CASE(N)                                                                                     \
    case N:                                                                                                  \
        if (prec == TC_BF16X3)                                                                               \
            return layout == LAYOUT_ROW ? croft_pass_kernel_tc<LAYOUT_ROW, N, TC_BF16X3>                     \
                                        : croft_pass_kernel_tc<LAYOUT_COL, N, TC_BF16X3>;                    \
        return layout == LAYOUT_ROW ? croft_pass_kernel_tc<LAYOUT_ROW, N, TC_FP16X3>                         \
                                    : croft_pass_kernel_tc<LAYOUT_COL, N, TC_FP16X3>;
    switch (n) {
        CROFT_TCAT(CROFT_TC_SIZES_, CROFT_TC_GROUP)(CROFT_TC_CASE)
        default: return nullptr;
    }
#undef CROFT_TC_CASE
}

#else  // the lookup and the DFT-16 operands (one translation unit)

pass_fn lookup_tc_kernel_group_0(int layout, int n, int prec);
pass_fn lookup_tc_kernel_group_1(int layout, int n, int prec);
pass_fn lookup_tc_kernel_group_2(int layout, int n, int prec);
pass_fn lookup_tc_kernel_group_3(int layout, int n, int prec);

pass_fn tc_pass_kernel_for(int layout, int n, int prec) {
    if (prec != TC_BF16X3 && prec != TC_FP16X3) return nullptr;
    pass_fn f = lookup_tc_kernel_group_0(layout, n, prec);
    if (!f) f = lookup_tc_kernel_group_1(layout, n, prec);
    if (!f) f = lookup_tc_kernel_group_2(layout, n, prec);
    if (!f) f = lookup_tc_kernel_group_3(layout, n, prec);
    return f;
}

void tc_dft16_matrix(unsigned char* out, int prec) { tc_dft16_operand(out, prec == TC_FP16X3); }

#endif  // CROFT_TC_GROUP

}  // namespace croft
