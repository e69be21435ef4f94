// croft_pair.cu - instantiations of the cluster-pair column kernel (croft_pair_kernel.cuh) for
// the even lengths whose pencils take 32 threads (the half lengths take 16).
#include "croft_pair_kernel.cuh"

namespace croft {

#define CROFT_PAIR_SIZES(X) \
    X(270) X(288) X(300) X(320) X(324) X(360) X(384) X(400) X(432) X(450) X(480) X(486) X(500) X(512)

pass_fn pair_kernel_for(int n) {
#define CROFT_PAIR_CASE(N) \
    case N: return croft_pair_kernel<N>;
    switch (n) {
        CROFT_PAIR_SIZES(CROFT_PAIR_CASE)
        default: return nullptr;
    }
#undef CROFT_PAIR_CASE
}

}  // namespace croft
