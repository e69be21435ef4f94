// croft_pipe.cu - instantiations of the TMA-pipelined pass kernel (even lengths 64..1024),
// compiled once per group (-DCROFT_PIPE_GROUP=0/1) so the two halves build in parallel.
#include "croft_pipe_kernel.cuh"

#ifndef CROFT_PIPE_GROUP
#error "compile with -DCROFT_PIPE_GROUP=<0|1>"
#endif

#define CROFT_PIPE_SIZES_0(X)                                                                              \
    X(64) X(80) X(96) X(108) X(128) X(150) X(162) X(192) X(216) X(250) X(270) X(300) X(324) X(384) X(432)   \
    X(480) X(500) X(540) X(600) X(648) X(750) X(800) X(864) X(960) X(1000)
#define CROFT_PIPE_SIZES_1(X)                                                                              \
    X(72) X(90) X(100) X(120) X(144) X(160) X(180) X(200) X(240) X(256) X(288) X(320) X(360) X(400) X(450)  \
    X(486) X(512) X(576) X(640) X(720) X(768) X(810) X(900) X(972) X(1024)

#define CROFT_PCAT_(a, b) a##b
#define CROFT_PCAT(a, b) CROFT_PCAT_(a, b)

namespace croft {

pipe_fn CROFT_PCAT(lookup_pipe_kernel_group_, CROFT_PIPE_GROUP)(int layout, int n) {
#define CROFT_PIPE_CASE(N) \
    case N: return layout == LAYOUT_ROW ? croft_pipe_kernel<LAYOUT_ROW, N> : croft_pipe_kernel<LAYOUT_COL, N>;
    switch (n) {
        CROFT_PCAT(CROFT_PIPE_SIZES_, CROFT_PIPE_GROUP)(CROFT_PIPE_CASE)
        default: return nullptr;
    }
#undef CROFT_PIPE_CASE
}

}  // namespace croft
