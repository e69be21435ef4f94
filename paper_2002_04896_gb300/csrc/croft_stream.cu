// croft_stream.cu - streaming executor: host-resident grids through the GPU with
// the host->device copy, the transform and the device->host copy of different
// grids in flight at the same time.
//
// Paper mapping: the paper overlaps packing and computation with the MPI
// all-to-all by splitting the exchange into K chunks handled by a dedicated
// communication thread (Sec. 5.1, Sec. 5.2).  On one GPU the slow link is the
// host link (NVLink-C2C), and the same idea becomes a three-stage software
// pipeline over grids: while grid i is transformed, grid i+1 is uploaded and
// grid i-1 downloaded, each on its own CUDA stream, ordered by events.  The
// upload and download directions of the link run concurrently.
//
// Resources (allocated on the first call, kept by the plan, reported by
// croft_plan_workspace_bytes): kSlots device buffers of one grid each, three
// streams and the per-slot events.
#include <cuda_runtime.h>

#include <new>

#include "croft_plan_internal.h"

namespace croft {

constexpr int kSlots = 3;

struct StreamState {
    float2* slot[kSlots] = {nullptr, nullptr, nullptr};
    cudaStream_t s_in = nullptr, s_comp = nullptr, s_out = nullptr;
    cudaEvent_t ev_in[kSlots] = {}, ev_comp[kSlots] = {}, ev_out[kSlots] = {};
    cudaEvent_t ev_start = nullptr, ev_end_comp = nullptr, ev_end_out = nullptr;
    size_t bytes = 0;
};

void stream_state_destroy(StreamState* st) {
    if (!st) return;
    for (int k = 0; k < kSlots; ++k) {
        dev_free(st->slot[k]);
        if (st->ev_in[k]) cudaEventDestroy(st->ev_in[k]);
        if (st->ev_comp[k]) cudaEventDestroy(st->ev_comp[k]);
        if (st->ev_out[k]) cudaEventDestroy(st->ev_out[k]);
    }
    if (st->ev_start) cudaEventDestroy(st->ev_start);
    if (st->ev_end_comp) cudaEventDestroy(st->ev_end_comp);
    if (st->ev_end_out) cudaEventDestroy(st->ev_end_out);
    if (st->s_in) cudaStreamDestroy(st->s_in);
    if (st->s_comp) cudaStreamDestroy(st->s_comp);
    if (st->s_out) cudaStreamDestroy(st->s_out);
    delete st;
}

size_t stream_state_bytes(const StreamState* st) { return st ? kSlots * st->bytes : 0; }

static croft_status stream_state_create(croft_plan plan, StreamState** out) {
    StreamState* st = new (std::nothrow) StreamState();
    if (!st) return CROFT_ERR_OOM;
    st->bytes = (size_t)plan->dims[0] * plan->dims[1] * plan->dims[2] *
                (plan->dtype == CROFT_C2C_F64 ? sizeof(double2) : sizeof(float2));
    for (int k = 0; k < kSlots; ++k)
        if (dev_alloc((void**)&st->slot[k], st->bytes) != cudaSuccess) {
            cudaGetLastError();
            stream_state_destroy(st);
            return CROFT_ERR_OOM;
        }
    bool ok = cudaStreamCreateWithFlags(&st->s_in, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&st->s_comp, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&st->s_out, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&st->ev_start, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&st->ev_end_comp, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&st->ev_end_out, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; ok && k < kSlots; ++k)
        ok = cudaEventCreateWithFlags(&st->ev_in[k], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&st->ev_comp[k], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&st->ev_out[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        stream_state_destroy(st);
        return CROFT_ERR_CUDA;
    }
    *out = st;
    return CROFT_OK;
}

croft_status exec_forward_impl(croft_plan plan, const void* in, void* out, void* stream);
croft_status exec_backward_impl(croft_plan plan, const void* in, void* out, void* stream);

}  // namespace croft

using namespace croft;

#define CROFT_CK(x)                      \
    do {                                 \
        if ((x) != cudaSuccess) {        \
            cudaGetLastError();          \
            return CROFT_ERR_CUDA;       \
        }                                \
    } while (0)

extern "C" croft_status croft_exec_host_pipeline(croft_plan plan, int count, const void* const* host_in,
                                                 void* const* host_out, int ops, void* stream) {
    if (!plan || plan->batch || count < 0 || (count > 0 && (!host_in || !host_out))) return CROFT_ERR_INVALID_ARG;
    if ((ops & ~(CROFT_OP_FORWARD | CROFT_OP_BACKWARD)) != 0 || ops == 0) return CROFT_ERR_INVALID_ARG;
    for (int i = 0; i < count; ++i)
        if (!host_in[i] || !host_out[i]) return CROFT_ERR_INVALID_ARG;
    if (count == 0) return CROFT_OK;
    if (!plan->stream) {
        croft_status s = stream_state_create(plan, &plan->stream);
        if (s != CROFT_OK) return s;
    }
    StreamState* st = plan->stream;
    cudaStream_t caller = (cudaStream_t)stream;
    // the pipeline starts after the caller's prior work and the caller's stream waits for its end
    CROFT_CK(cudaEventRecord(st->ev_start, caller));
    CROFT_CK(cudaStreamWaitEvent(st->s_in, st->ev_start, 0));
    CROFT_CK(cudaStreamWaitEvent(st->s_comp, st->ev_start, 0));
    CROFT_CK(cudaStreamWaitEvent(st->s_out, st->ev_start, 0));
    for (int i = 0; i < count; ++i) {
        const int k = i % kSlots;
        if (i >= kSlots) CROFT_CK(cudaStreamWaitEvent(st->s_in, st->ev_out[k], 0));  // slot downloaded
        CROFT_CK(cudaMemcpyAsync(st->slot[k], host_in[i], st->bytes, cudaMemcpyHostToDevice, st->s_in));
        CROFT_CK(cudaEventRecord(st->ev_in[k], st->s_in));
        CROFT_CK(cudaStreamWaitEvent(st->s_comp, st->ev_in[k], 0));
        if (ops & CROFT_OP_FORWARD) {
            croft_status s = exec_forward_impl(plan, st->slot[k], st->slot[k], st->s_comp);
            if (s != CROFT_OK) return s;
        }
        if (ops & CROFT_OP_BACKWARD) {
            croft_status s = exec_backward_impl(plan, st->slot[k], st->slot[k], st->s_comp);
            if (s != CROFT_OK) return s;
        }
        CROFT_CK(cudaEventRecord(st->ev_comp[k], st->s_comp));
        CROFT_CK(cudaStreamWaitEvent(st->s_out, st->ev_comp[k], 0));
        CROFT_CK(cudaMemcpyAsync(host_out[i], st->slot[k], st->bytes, cudaMemcpyDeviceToHost, st->s_out));
        CROFT_CK(cudaEventRecord(st->ev_out[k], st->s_out));
    }
    CROFT_CK(cudaEventRecord(st->ev_end_out, st->s_out));
    CROFT_CK(cudaStreamWaitEvent(caller, st->ev_end_out, 0));
    CROFT_CK(cudaEventRecord(st->ev_end_comp, st->s_comp));  // (the download stream already waited on it)
    CROFT_CK(cudaStreamWaitEvent(caller, st->ev_end_comp, 0));
    return CROFT_OK;
}
