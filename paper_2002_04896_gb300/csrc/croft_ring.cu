// croft_ring.cu - instantiations of the tensor-copy ring column kernel (croft_ring_kernel.cuh)
// for the lengths whose pencils take 32 threads (270 .. 512).
#include "croft_ring_kernel.cuh"

namespace croft {

#define CROFT_RING_SIZES(X) \
    X(270) X(288) X(300) X(320) X(324) X(360) X(375) X(384) X(400) X(405) X(432) X(450) X(480) X(486) X(500) X(512)

ring_fn ring_kernel_for(int n) {
#define CROFT_RING_CASE(N) \
    case N: return croft_ring_kernel<N>;
    switch (n) {
        CROFT_RING_SIZES(CROFT_RING_CASE)
        default: return nullptr;
    }
#undef CROFT_RING_CASE
}

}  // namespace croft
