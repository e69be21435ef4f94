// croft_plan_internal.h - the plan object behind the opaque croft_plan handle.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/croft.h"
#include "croft_internal.h"

namespace croft {
struct BatchState;  // croft_batch_plan.cu
void batch_state_destroy(BatchState* b);
struct StreamState;  // croft_stream.cu
void stream_state_destroy(StreamState* st);
size_t stream_state_bytes(const StreamState* st);
}  // namespace croft

struct croft_plan_s {
    int dims[3];          // nx, ny, nz
    croft_dtype dtype;
    int device;
    std::vector<croft::PassLaunch> passes;   // execution order (z, y, x; length-1 axes skipped)
    std::vector<int> pass_axis;       // axis index of each pass (2 = z, 1 = y, 0 = x)
    float2* tw_dev[3];                // per-axis twiddle tables (NULL for length <= 1)
    float2* tw_pair[3];               // pair column passes: [half-length table | combine twiddles], else NULL
    float2* tw_conv;                  // fused convolution: its axis's table in the convolution kernel's
                                      // schedule when the axis's passes follow another one, else NULL
    bool timing;
    std::vector<cudaEvent_t> ev;      // one per logical pass + 1 (created when timing is enabled)
    int ev_count;                     // events recorded by the last exec
    int ngroups;                      // logical passes (launches of one group are timed together)
    bool ran;
    croft::BatchState* batch;         // batched plans only (NULL for a single-grid plan)
    croft::StreamState* stream;       // host-streaming executor state (created on first use)
    unsigned char* tc_b;              // tensor-core plans: DFT-16 operand (4 KB), else NULL
    int* d_status;                    // tensor-core plans: device status word, else NULL
    bool axis_tc[3];                  // axis runs the tensor-core pass kernel
    int tc_prec;                      // tensor-core operand precision (TcPrec) of such axes
    croft::PassLaunch conv;           // fused convolution pass (croft_conv_kernel.cuh), valid when conv_fused
    int conv_axis;                    // its axis (the plan's last pass)
    bool conv_fused;                  // false: croft_exec_convolve runs F, a multiply and B instead
    bool pdl;                         // launches after the first of an exec use programmatic dependent launch
    // per-axis kernel choice (CROFT_SCHEDULE_TUNED): kind -1 the library's rules, 0 the plain pass
    // kernel with tile width axis_w and schedule variant axis_sv, 1 the tensor-copy ring kernel,
    // 2 the cluster-pair kernel
    int axis_kind[3];
    int axis_w[3];
    int axis_sv[3];
    int axis_th[3];                   // threads per pencil of a tuned plain column kernel (0: the rule's)
    std::string tuned;                // the tuner's choice and measurements (describe)
};

