// croft_batch_noalloc.cu - the batched transform for callers that cannot allocate device memory.
//
// Same persistent kernel and work decomposition as a CROFT_BATCH_ONE_LAUNCH
// plan, but every buffer the kernel needs besides the caller's grids (work
// counter, per-grid completion counts, status word, grid descriptors, work
// list, twiddle tables) lives in one file-scope __device__ array below.  The
// call itself allocates nothing on the device: it copies the host-built tables
// into the array and launches.
#include <cuda_runtime.h>

#include <stdint.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "../../include/croft.h"
#include "croft_batched_kernel.cuh"

namespace croft {

croft_status build_batch_tables(const std::vector<int>& dims, const std::vector<int>& pgrid,
                                std::vector<BatchGrid>& hgrid, std::vector<BatchItem>& items,
                                std::vector<float>& pool, int pass_begin[4]);
bool batch_size_supported(int n);
int batch_smem_bytes();
cudaError_t batched_prepare(int smem);
int batched_blocks_per_sm(int smem);
cudaError_t launch_batched(const BatchArgs& A, int blocks, int smem, cudaStream_t s);

// Capacity of the static scratch (held by every GPU that loads the library until exit).
constexpr int kNaMaxGrids = CROFT_NOALLOC_MAX_GRIDS;
constexpr int kNaMaxItems = CROFT_NOALLOC_MAX_ITEMS;
constexpr int kNaMaxTw = 8192;         // float2 slots; all 37 supported lengths <= 128 need < 2500
constexpr int kNaCounterInts = 1024;   // [0] work counter, [4] status, [8 + 3 g + pass] completion counts
constexpr size_t kNaCounters = sizeof(int) * kNaCounterInts;
constexpr size_t kNaGridsOff = kNaCounters;
constexpr size_t kNaItemsOff = kNaGridsOff + sizeof(BatchGrid) * kNaMaxGrids;
constexpr size_t kNaTwOff = kNaItemsOff + sizeof(BatchItem) * kNaMaxItems;
constexpr size_t kNaBytes = kNaTwOff + sizeof(float2) * kNaMaxTw;
static_assert(8 + 3 * kNaMaxGrids <= kNaCounterInts, "counter region too small");
static_assert(kNaGridsOff % 16 == 0 && kNaItemsOff % 16 == 0 && kNaTwOff % 16 == 0, "region alignment");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

// Device address of g_noalloc_scratch on the current device, looked up once per
// device and kept for the life of the process (host code may not use the symbol
// itself as a device pointer; after a cudaDeviceReset the kept address is stale).
static croft_status noalloc_scratch(unsigned char** out) {
    static std::mutex mu;
    static void* addr[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return CROFT_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return CROFT_ERR_CUDA;
        }
        addr[dev] = p;
    }
    *out = (unsigned char*)addr[dev];
    return CROFT_OK;
}

}  // namespace croft

using namespace croft;

extern "C" croft_status croft_exec_batched_noalloc(int count, const int* dims, void* const* in, void* const* out,
                                                   int direction, void* stream) {
    if (count < 1 || !dims || !in || !out || (direction != 1 && direction != -1)) return CROFT_ERR_INVALID_ARG;
    // The host tables below live only for this call: a copy captured into a graph would read
    // freed memory on every replay, so a capturing stream is refused before any device work.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cap) != cudaSuccess) {
        cudaGetLastError();
        return CROFT_ERR_INVALID_ARG;
    }
    if (cap != cudaStreamCaptureStatusNone) return CROFT_ERR_INVALID_ARG;
    if (count > kNaMaxGrids) return CROFT_ERR_UNSUPPORTED_SIZE;
    for (int i = 0; i < 3 * count; ++i)
        if (dims[i] != 1 && !batch_size_supported(dims[i])) return CROFT_ERR_UNSUPPORTED_SIZE;
    std::vector<int> dv(dims, dims + 3 * count);
    std::vector<int> pgrid;
    for (int g = 0; g < count; ++g) {
        const char* x = (const char*)in[g];
        const char* y = (const char*)out[g];
        if (!x || !y || ((uintptr_t)x & 15) || ((uintptr_t)y & 15)) return CROFT_ERR_INVALID_ARG;
        const size_t nb = (size_t)dims[3 * g] * dims[3 * g + 1] * dims[3 * g + 2] * sizeof(float2);
        if (x != y && x < y + nb && y < x + nb) return CROFT_ERR_INVALID_ARG;
        if (nb > sizeof(float2)) pgrid.push_back(g);
    }
    std::vector<BatchGrid> hgrid;
    std::vector<BatchItem> items;
    std::vector<float> pool;
    int pass_begin[4];
    const croft_status st = build_batch_tables(dv, pgrid, hgrid, items, pool, pass_begin);
    if (st != CROFT_OK) return st;
    if ((int)items.size() > kNaMaxItems || pool.size() / 2 > (size_t)kNaMaxTw) return CROFT_ERR_UNSUPPORTED_SIZE;
    for (size_t i = 0; i < pgrid.size(); ++i) {
        hgrid[i].in = (const float2*)in[pgrid[i]];
        hgrid[i].out = (float2*)out[pgrid[i]];
    }
    unsigned char* base = nullptr;
    if (noalloc_scratch(&base) != CROFT_OK) return CROFT_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    // single-point grids are copies
    for (int g = 0; g < count; ++g) {
        const size_t nb = (size_t)dims[3 * g] * dims[3 * g + 1] * dims[3 * g + 2] * sizeof(float2);
        if (nb == sizeof(float2) && in[g] != out[g] &&
            cudaMemcpyAsync(out[g], in[g], nb, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
            cudaGetLastError();
            return CROFT_ERR_CUDA;
        }
    }
    if (items.empty()) return CROFT_OK;
    const int smem = batch_smem_bytes();
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || batched_prepare(smem) != cudaSuccess) {
        cudaGetLastError();
        return CROFT_ERR_CUDA;
    }
    const int per_sm = batched_blocks_per_sm(smem);
    if (per_sm < 1) return CROFT_ERR_CUDA;
    // counters start at zero; tables overwrite the previous call's
    if (cudaMemsetAsync(base, 0, kNaCounters, s) != cudaSuccess ||
        cudaMemcpyAsync(base + kNaGridsOff, hgrid.data(), sizeof(BatchGrid) * hgrid.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(base + kNaItemsOff, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        (!pool.empty() &&
         cudaMemcpyAsync(base + kNaTwOff, pool.data(), sizeof(float) * pool.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)) {
        cudaGetLastError();
        return CROFT_ERR_CUDA;
    }
    BatchArgs A;
    memset(&A, 0, sizeof(A));
    A.grids = (const BatchGrid*)(base + kNaGridsOff);
    A.items = (const BatchItem*)(base + kNaItemsOff);
    A.tw_pool = (const float2*)(base + kNaTwOff);
    A.queue = (int*)base;
    A.status = (int*)base + 4;
    A.done = (int*)base + 8;
    A.wait_cycles = 4000000000LL;
    A.item_begin = 0;
    A.item_end = (int)items.size();
    A.extra_wait = 0;
    A.isign = direction == -1 ? 1.f : -1.f;  // -1: forward, Eq. (1); +1: backward, Eq. (2)
    const int blocks = sms * per_sm < (int)items.size() ? sms * per_sm : (int)items.size();
    if (launch_batched(A, blocks, smem, s) != cudaSuccess) {
        cudaGetLastError();
        return CROFT_ERR_CUDA;
    }
    return CROFT_OK;
}
