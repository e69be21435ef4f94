// croft_batch_plan.cu - batched plans: many independent grids of uneven sizes.
//
// Schedules (croft_batch_mode):
//   ONE_LAUNCH : every tile of every pass of every grid in one persistent launch
//                (work counter + bounded per-grid dependency waits);
//   PER_PASS   : the same work list in three launches (z, y, x) of one CTA per
//                tile; kernel boundaries order the passes, no counters, no waits;
//   PER_GRID   : one ordinary single-grid plan per grid, launched one after
//                the other (the plain baseline);
//   GROUPED    : per pass, one launch per distinct axis length over every grid
//                that has it (croft_batch_group.cu), the launches of a pass
//                concurrent.
// ONE_LAUNCH, PER_PASS and GROUPED are recorded once into a CUDA graph per direction
// (descriptor upload from pinned memory, counter reset, kernel launch(es));
// an exec fills in the grids' pointers and launches the graph.  AUTO times the
// four schedules on scratch buffers at plan creation and keeps the fastest,
// caching the choice on disk (like FFTW wisdom) keyed by the batch's sizes, the
// GPU name and the CUDA runtime version.
//
// Paper mapping: the K-chunk parameter of Sec. 5.1 (trading the size of an
// overlapped chunk against the number of calls) is the tuner's choice between
// one call for everything, one call per pass and one call per grid.
#include <cuda_runtime.h>

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "croft_batched_kernel.cuh"
#include "croft_plan_internal.h"

namespace croft {

bool batch_size_supported(int n);
int batch_smem_bytes();
int batch_col_width(int n);
cudaError_t batched_prepare(int smem);
int batched_blocks_per_sm(int smem);
void* batched_kernel_ptr();
int host_build_twiddles(int n, float* out);  // croft_plan.cu

struct GroupState;  // croft_batch_group.cu
croft_status group_state_build(const std::vector<int>& dims, const std::vector<int>& pgrid, GroupState** out);
void group_state_destroy(GroupState* s);
void group_state_fill(GroupState* s, void* const* in, void* const* out);
croft_status group_graph_add(GroupState* s, cudaGraph_t g, float isign, bool pdl);
int group_state_launches(const GroupState* s);

struct BatchState {
    int count = 0;
    std::vector<int> dims;
    int mode = 0;
    // persistent path
    std::vector<int> pgrid;          // batch index of each persistent grid
    std::vector<BatchGrid> hgrid;    // descriptors (pointers filled per exec)
    BatchGrid* staging = nullptr;    // pinned copy the graph uploads
    BatchGrid* d_grids = nullptr;
    BatchItem* d_items = nullptr;
    float2* d_tw = nullptr;
    int* d_scratch = nullptr;
    int scratch_ints = 0;
    int nitems = 0;
    int pass_begin[4] = {0, 0, 0, 0};
    int blocks = 0, smem = 0;
    long long wait_cycles = 4000000000LL;  // ~2 s at 2 GHz
    int extra_wait = 0;
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    bool graphs_dirty = true;
    cudaEvent_t staging_free = nullptr;
    bool staging_pending = false;
    // grids on single-grid plans (axes > 128, or PER_GRID mode)
    std::vector<int> sgrid;
    std::vector<croft_plan> subplans;
    GroupState* group = nullptr;      // GROUPED schedule
    double tuned_us[5] = {0, 0, 0, 0, 0};
};

void batch_state_destroy(BatchState* b) {
    if (!b) return;
    for (int d = 0; d < 2; ++d) {
        if (b->gexec[d]) cudaGraphExecDestroy(b->gexec[d]);
        if (b->graph[d]) cudaGraphDestroy(b->graph[d]);
    }
    if (b->staging_free) cudaEventDestroy(b->staging_free);
    if (b->staging) host_free(b->staging);
    dev_free(b->d_grids);
    dev_free(b->d_items);
    dev_free(b->d_tw);
    dev_free(b->d_scratch);
    for (croft_plan p : b->subplans) croft_plan_destroy(p);
    group_state_destroy(b->group);
    delete b;
}

static const int kPassAxis[3] = {2, 1, 0};  // pass 0 = z, 1 = y, 2 = x
croft_status build_batch_tables(const std::vector<int>& dims, const std::vector<int>& pgrid,
                                std::vector<BatchGrid>& hgrid, std::vector<BatchItem>& items,
                                std::vector<float>& pool, int pass_begin[4]);

// Host tables of the persistent schedule for the grids `pgrid` of a batch:
// grid descriptors (pointers left NULL), the work list (pass by pass, biggest
// grids first within a pass), the twiddle pool and the item range of each pass.
croft_status build_batch_tables(const std::vector<int>& dims, const std::vector<int>& pgrid,
                                std::vector<BatchGrid>& hgrid, std::vector<BatchItem>& items,
                                std::vector<float>& pool, int pass_begin[4]) {
    const int G = (int)pgrid.size();
    std::vector<int> lens;
    for (int g : pgrid)
        for (int a = 0; a < 3; ++a) lens.push_back(dims[3 * g + a]);
    std::sort(lens.begin(), lens.end());
    lens.erase(std::unique(lens.begin(), lens.end()), lens.end());
    pool.clear();
    std::vector<int> off(CROFT_BATCH_MAX_N + 1, 0);
    for (int n : lens) {
        if (n > CROFT_BATCH_MAX_N) return CROFT_ERR_UNSUPPORTED_SIZE;
        off[n] = (int)(pool.size() / 2);
        std::vector<float> t(2 * (size_t)n + 2, 0.f);
        if (n > 1 && host_build_twiddles(n, t.data()) != n - 1) return CROFT_ERR_UNSUPPORTED_SIZE;
        pool.insert(pool.end(), t.begin(), t.begin() + 2 * std::max(1, n - 1));
    }
    hgrid.assign(G, BatchGrid{});
    for (int i = 0; i < G; ++i) {
        const int g = pgrid[i];
        const int nx = dims[3 * g], ny = dims[3 * g + 1], nz = dims[3 * g + 2];
        const long long N = (long long)nx * ny * nz;
        BatchGrid& D = hgrid[i];
        D.first_pass = -1;
        int prev = -1;
        for (int p = 0; p < 3; ++p) {
            const int axis = kPassAxis[p];
            const int n = dims[3 * g + axis];
            D.n[p] = n;
            D.M[p] = (axis == 2) ? 1 : (axis == 1 ? (long long)nz : (long long)ny * nz);
            D.ncols[p] = N / n;
            D.tw_off[p] = off[n];
            D.dep[p] = -1;
            if (n == 1) {
                D.W[p] = 1;
                D.ntiles[p] = 0;
                continue;
            }
            const int T = croft_threads_per_pencil(n);
            D.W[p] = (D.M[p] == 1) ? CROFT_BATCH_THREADS / T : batch_col_width(n);
            D.ntiles[p] = (int)((D.ncols[p] + D.W[p] - 1) / D.W[p]);
            D.cdiv[p] = croft_coldiv_make(D.M[p], D.ncols[p] + D.W[p]);
            D.dep[p] = prev;
            if (D.first_pass < 0) D.first_pass = p;
            prev = p;
        }
    }
    std::vector<int> order(G);
    for (int i = 0; i < G; ++i) order[i] = i;
    items.clear();
    for (int p = 0; p < 3; ++p) {
        pass_begin[p] = (int)items.size();
        std::sort(order.begin(), order.end(), [&](int a, int c) {
            return (long long)hgrid[a].ntiles[p] * hgrid[a].n[p] > (long long)hgrid[c].ntiles[p] * hgrid[c].n[p];
        });
        for (int i : order)
            for (int t = 0; t < hgrid[i].ntiles[p]; ++t) items.push_back(BatchItem{i, p, t, 0});
    }
    pass_begin[3] = (int)items.size();
    return CROFT_OK;
}

static croft_status build_persistent(BatchState* b) {
    const int G = (int)b->pgrid.size();
    if (G == 0) return CROFT_OK;
    std::vector<BatchItem> items;
    std::vector<float> pool;
    croft_status st = build_batch_tables(b->dims, b->pgrid, b->hgrid, items, pool, b->pass_begin);
    if (st != CROFT_OK) return st;
    b->nitems = (int)items.size();
    b->scratch_ints = 8 + 3 * G;
    b->smem = batch_smem_bytes();
    if (batched_prepare(b->smem) != cudaSuccess) return CROFT_ERR_CUDA;
    int dev = 0;
    cudaGetDevice(&dev);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int per_sm = batched_blocks_per_sm(b->smem);
    if (per_sm < 1) return CROFT_ERR_CUDA;
    b->blocks = std::max(1, std::min(sms * per_sm, b->nitems));

    if (dev_alloc((void**)&b->d_tw, sizeof(float) * std::max<size_t>(2, pool.size())) != cudaSuccess) return CROFT_ERR_OOM;
    if (dev_alloc((void**)&b->d_items, sizeof(BatchItem) * std::max(1, b->nitems)) != cudaSuccess) return CROFT_ERR_OOM;
    if (dev_alloc((void**)&b->d_grids, sizeof(BatchGrid) * G) != cudaSuccess) return CROFT_ERR_OOM;
    if (dev_alloc((void**)&b->d_scratch, sizeof(int) * b->scratch_ints) != cudaSuccess) return CROFT_ERR_OOM;
    if (host_alloc((void**)&b->staging, sizeof(BatchGrid) * G) != cudaSuccess) return CROFT_ERR_OOM;
    if (cudaEventCreateWithFlags(&b->staging_free, cudaEventDisableTiming) != cudaSuccess) return CROFT_ERR_CUDA;
    if (!pool.empty() && cudaMemcpy(b->d_tw, pool.data(), sizeof(float) * pool.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return CROFT_ERR_CUDA;
    if (b->nitems && cudaMemcpy(b->d_items, items.data(), sizeof(BatchItem) * b->nitems, cudaMemcpyHostToDevice) != cudaSuccess)
        return CROFT_ERR_CUDA;
    memcpy(b->staging, b->hgrid.data(), sizeof(BatchGrid) * G);
    return CROFT_OK;
}

static BatchArgs batch_args(const BatchState* b, int launch, int begin, int end, float isign) {
    BatchArgs A;
    memset(&A, 0, sizeof(A));
    A.grids = b->d_grids;
    A.items = b->d_items;
    A.tw_pool = b->d_tw;
    A.queue = b->d_scratch + launch;
    A.done = b->d_scratch + 8;
    A.status = b->d_scratch + 4;
    A.wait_cycles = b->wait_cycles;
    A.item_begin = begin;
    A.item_end = end;
    A.extra_wait = b->extra_wait;
    A.isign = isign;
    return A;
}

// Graph per direction: [descriptor upload] + [counter reset] -> kernel launch(es).
static croft_status build_graphs(BatchState* b) {
    for (int d = 0; d < 2; ++d) {
        if (b->gexec[d]) cudaGraphExecDestroy(b->gexec[d]);
        if (b->graph[d]) cudaGraphDestroy(b->graph[d]);
        b->gexec[d] = nullptr;
        b->graph[d] = nullptr;
    }
    b->graphs_dirty = false;
    if (b->pgrid.empty() || b->mode == CROFT_BATCH_PER_GRID) return CROFT_OK;
    const int G = (int)b->pgrid.size();
    for (int d = 0; d < 2; ++d) {
        const float isign = d == 0 ? 1.f : -1.f;
        cudaGraph_t g;
        if (cudaGraphCreate(&g, 0) != cudaSuccess) return CROFT_ERR_CUDA;
        b->graph[d] = g;
        if (b->mode == CROFT_BATCH_GROUPED) {
            const char* pdl_env = getenv("CROFT_PDL");  // 0: ordinary graph edges between the passes
            croft_status st = group_graph_add(b->group, g, isign, !(pdl_env && pdl_env[0] == '0'));
            if (st != CROFT_OK) return st;
            if (cudaGraphInstantiate(&b->gexec[d], g, 0) != cudaSuccess) return CROFT_ERR_CUDA;
            continue;
        }
        cudaGraphNode_t up, rs;
        if (cudaGraphAddMemcpyNode1D(&up, g, nullptr, 0, b->d_grids, b->staging, sizeof(BatchGrid) * G,
                                     cudaMemcpyHostToDevice) != cudaSuccess)
            return CROFT_ERR_CUDA;
        cudaMemsetParams ms;
        memset(&ms, 0, sizeof(ms));
        ms.dst = b->d_scratch;
        ms.value = 0;
        ms.elementSize = 4;
        ms.width = (size_t)b->scratch_ints;
        ms.height = 1;
        if (cudaGraphAddMemsetNode(&rs, g, nullptr, 0, &ms) != cudaSuccess) return CROFT_ERR_CUDA;
        std::vector<cudaGraphNode_t> deps = {up, rs};
        const int nl = (b->mode == CROFT_BATCH_PER_PASS) ? 3 : 1;
        for (int l = 0; l < nl; ++l) {
            const int begin = (nl == 1) ? 0 : b->pass_begin[l];
            const int end = (nl == 1) ? b->nitems : b->pass_begin[l + 1];
            if (begin == end) continue;
            BatchArgs A = batch_args(b, l, begin, end, isign);
            A.direct = (b->mode == CROFT_BATCH_PER_PASS) ? 1 : 0;  // per pass: one CTA per tile
            void* params[1] = {&A};
            cudaKernelNodeParams kp;
            memset(&kp, 0, sizeof(kp));
            kp.func = batched_kernel_ptr();
            kp.gridDim = dim3((unsigned)(A.direct ? end - begin : std::min(b->blocks, end - begin)), 1, 1);
            kp.blockDim = dim3(CROFT_BATCH_THREADS, 1, 1);
            kp.sharedMemBytes = (unsigned)b->smem;
            kp.kernelParams = params;
            cudaGraphNode_t kn;
            if (cudaGraphAddKernelNode(&kn, g, deps.data(), deps.size(), &kp) != cudaSuccess) return CROFT_ERR_CUDA;
            deps.assign(1, kn);
        }
        if (cudaGraphInstantiate(&b->gexec[d], g, 0) != cudaSuccess) return CROFT_ERR_CUDA;
    }
    return CROFT_OK;
}

static size_t grid_bytes(const BatchState* b, int g) {
    return (size_t)b->dims[3 * g] * b->dims[3 * g + 1] * b->dims[3 * g + 2] * sizeof(float2);
}

static croft_status exec_batch(croft_plan plan, void* const* in, void* const* out, void* stream, int dir) {
    BatchState* b = plan->batch;
    if (!in || !out) return CROFT_ERR_INVALID_ARG;
    for (int g = 0; g < b->count; ++g) {
        const char* x = (const char*)in[g];
        const char* y = (const char*)out[g];
        if (!x || !y || ((uintptr_t)x & 15) || ((uintptr_t)y & 15)) return CROFT_ERR_INVALID_ARG;
        const size_t nb = grid_bytes(b, g);
        if (x != y && x < y + nb && y < x + nb) return CROFT_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (b->graphs_dirty) {
        croft_status st = build_graphs(b);
        if (st != CROFT_OK) return st;
    }
    const bool tm = plan->timing;
    if (tm && cudaEventRecord(plan->ev[0], s) != cudaSuccess) { cudaGetLastError(); return CROFT_ERR_CUDA; }
    if (b->gexec[dir]) {
        if (b->staging_pending && cudaEventSynchronize(b->staging_free) != cudaSuccess) {
            cudaGetLastError();
            return CROFT_ERR_CUDA;
        }
        if (b->mode == CROFT_BATCH_GROUPED) {
            group_state_fill(b->group, in, out);
        } else {
            for (size_t i = 0; i < b->pgrid.size(); ++i) {
                b->staging[i].in = (const float2*)in[b->pgrid[i]];
                b->staging[i].out = (float2*)out[b->pgrid[i]];
            }
        }
        if (cudaGraphLaunch(b->gexec[dir], s) != cudaSuccess) { cudaGetLastError(); return CROFT_ERR_CUDA; }
        if (cudaEventRecord(b->staging_free, s) != cudaSuccess) { cudaGetLastError(); return CROFT_ERR_CUDA; }
        b->staging_pending = true;
    }
    for (size_t i = 0; i < b->sgrid.size(); ++i) {
        const int g = b->sgrid[i];
        croft_status st = dir == 0 ? croft_exec_forward(b->subplans[i], in[g], out[g], stream)
                                   : croft_exec_backward(b->subplans[i], in[g], out[g], stream);
        if (st != CROFT_OK) return st;
    }
    if (tm) {
        if (cudaEventRecord(plan->ev[1], s) != cudaSuccess) { cudaGetLastError(); return CROFT_ERR_CUDA; }
        plan->ev_count = 2;
    }
    plan->ran = true;
    return CROFT_OK;
}

// ---------------------------------------------------------------------------
// autotuner with an on-disk cache
// ---------------------------------------------------------------------------

static std::string tune_key(const BatchState* b) {
    unsigned long long h = 1469598103934665603ULL;  // FNV-1a over the dims
    for (int v : b->dims) {
        h ^= (unsigned long long)v;
        h *= 1099511628211ULL;
    }
    int dev = 0, rt = 0;
    cudaGetDevice(&dev);
    cudaRuntimeGetVersion(&rt);
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, dev);
    char buf[512];
    snprintf(buf, sizeof(buf), "batch-v2:%d:%016llx:%s:%d", b->count, h, prop.name, rt);
    for (char* c = buf; *c; ++c)
        if (*c == ' ' || *c == '"') *c = '_';
    return buf;
}

static std::string tune_cache_path() {
    const char* p = getenv("CROFT_TUNE_CACHE");
    if (p && *p) return p;
    const char* home = getenv("HOME");
    return std::string(home && *home ? home : "/tmp") + "/.croft_tune_cache.txt";
}

static int tune_lookup(const std::string& key) {
    FILE* f = fopen(tune_cache_path().c_str(), "r");
    if (!f) return 0;
    char line[1024];
    int mode = 0;
    while (fgets(line, sizeof(line), f)) {
        char k[900];
        int m = 0;
        if (sscanf(line, "%899s %d", k, &m) == 2 && key == k) mode = m;
    }
    fclose(f);
    return mode;
}

static void tune_store(const std::string& key, int mode, const double* us) {
    FILE* f = fopen(tune_cache_path().c_str(), "a");
    if (!f) return;
    fprintf(f, "%s %d one_launch_us=%.1f per_pass_us=%.1f per_grid_us=%.1f grouped_us=%.1f\n", key.c_str(), mode, us[1],
            us[2], us[3], us[4]);
    fclose(f);
}

static croft_status configure(BatchState* b, int mode) {
    // (re)build the persistent part and the single-grid plans for `mode`
    for (croft_plan p : b->subplans) croft_plan_destroy(p);
    b->subplans.clear();
    b->sgrid.clear();
    b->pgrid.clear();
    b->mode = mode;
    for (int g = 0; g < b->count; ++g) {
        bool small = true;
        for (int a = 0; a < 3; ++a) small = small && batch_size_supported(b->dims[3 * g + a]);
        const bool all_one = b->dims[3 * g] == 1 && b->dims[3 * g + 1] == 1 && b->dims[3 * g + 2] == 1;
        if (small && !all_one && mode != CROFT_BATCH_PER_GRID) b->pgrid.push_back(g);
        else b->sgrid.push_back(g);
    }
    for (int g : b->sgrid) {
        croft_plan sp = nullptr;
        croft_status st = croft_plan_create(&sp, b->dims[3 * g], b->dims[3 * g + 1], b->dims[3 * g + 2], CROFT_C2C_F32);
        if (st != CROFT_OK) return st;
        b->subplans.push_back(sp);
    }
    if (mode == CROFT_BATCH_GROUPED) {
        if (!b->group && !b->pgrid.empty()) {
            croft_status st = group_state_build(b->dims, b->pgrid, &b->group);
            if (st != CROFT_OK) return st;
        }
        if (!b->staging_free && cudaEventCreateWithFlags(&b->staging_free, cudaEventDisableTiming) != cudaSuccess)
            return CROFT_ERR_CUDA;
    } else if (!b->d_items && !b->pgrid.empty()) {
        croft_status st = build_persistent(b);
        if (st != CROFT_OK) return st;
    }
    b->graphs_dirty = true;
    return CROFT_OK;
}

static croft_status autotune(croft_plan plan) {
    BatchState* b = plan->batch;
    const std::string key = tune_key(b);
    int cached = tune_lookup(key);
    if (cached >= CROFT_BATCH_ONE_LAUNCH && cached <= CROFT_BATCH_GROUPED) return configure(b, cached);
    size_t total = 0;
    std::vector<size_t> offs;
    for (int g = 0; g < b->count; ++g) {
        offs.push_back(total);
        total += (grid_bytes(b, g) + 255) / 256 * 256;
    }
    char* buf = nullptr;
    if (dev_alloc((void**)&buf, total) != cudaSuccess) {
        cudaGetLastError();
        return configure(b, CROFT_BATCH_GROUPED);
    }
    cudaMemset(buf, 0, total);
    std::vector<void*> ptrs(b->count);
    for (int g = 0; g < b->count; ++g) ptrs[g] = buf + offs[g];
    cudaStream_t s;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int modes[4] = {CROFT_BATCH_ONE_LAUNCH, CROFT_BATCH_PER_PASS, CROFT_BATCH_PER_GRID, CROFT_BATCH_GROUPED};
    double best = 1e30;
    int best_mode = CROFT_BATCH_ONE_LAUNCH;
    croft_status st = CROFT_OK;
    const bool tm = plan->timing;
    plan->timing = false;
    for (int m : modes) {
        st = configure(b, m);
        if (st != CROFT_OK) break;
        std::vector<float> t;
        for (int r = 0; r < 7 && st == CROFT_OK; ++r) {
            cudaEventRecord(e0, s);
            st = exec_batch(plan, ptrs.data(), ptrs.data(), s, 0);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r >= 2) t.push_back(ms);
        }
        if (st != CROFT_OK) break;
        std::sort(t.begin(), t.end());
        const double us = 1e3 * t[t.size() / 2];
        b->tuned_us[m] = us;
        if (us < best) {
            best = us;
            best_mode = m;
        }
    }
    plan->timing = tm;
    cudaStreamSynchronize(s);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    dev_free(buf);
    if (st != CROFT_OK) return st;
    tune_store(key, best_mode, b->tuned_us);
    return configure(b, best_mode);
}

}  // namespace croft

using namespace croft;

extern "C" {

croft_status croft_plan_create_batched_mode(croft_plan* out, int count, const int* dims, croft_dtype dtype,
                                            croft_batch_mode mode) {
    if (!out) return CROFT_ERR_INVALID_ARG;
    *out = NULL;
    if (count < 1 || !dims) return CROFT_ERR_INVALID_ARG;
    if (dtype != CROFT_C2C_F32)
        return (dtype == CROFT_C2C_F32_TC_BF16X3 || dtype == CROFT_C2C_F32_TC_FP16X3) ? CROFT_ERR_UNSUPPORTED_SIZE
                                                                                  : CROFT_ERR_INVALID_ARG;
    if (mode < CROFT_BATCH_AUTO || mode > CROFT_BATCH_GROUPED) return CROFT_ERR_INVALID_ARG;
    for (int i = 0; i < 3 * count; ++i)
        if (croft_make_sched(dims[i]).count < 0) return CROFT_ERR_UNSUPPORTED_SIZE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return CROFT_ERR_CUDA; }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) { cudaGetLastError(); return CROFT_ERR_CUDA; }
    if (prop.major < 10) return CROFT_ERR_CUDA;

    croft_plan p = new (std::nothrow) croft_plan_s();
    if (!p) return CROFT_ERR_OOM;
    p->dims[0] = count;
    p->dims[1] = 0;
    p->dims[2] = 0;
    p->dtype = dtype;
    p->device = dev;
    for (int a = 0; a < 3; ++a) p->tw_dev[a] = NULL;
    p->timing = false;
    p->ngroups = 1;
    p->stream = NULL;
    p->tc_b = NULL;
    p->d_status = NULL;
    p->ev_count = 0;
    p->ran = false;
    p->batch = new (std::nothrow) BatchState();
    if (!p->batch) {
        delete p;
        return CROFT_ERR_OOM;
    }
    p->batch->count = count;
    p->batch->dims.assign(dims, dims + 3 * count);
    croft_status st;
    const char* tune = getenv("CROFT_TUNE");
    if (mode == CROFT_BATCH_AUTO && !(tune && strcmp(tune, "off") == 0)) st = autotune(p);
    else st = configure(p->batch, mode == CROFT_BATCH_AUTO ? CROFT_BATCH_GROUPED : mode);  // (the usual winner)
    if (st == CROFT_OK) st = build_graphs(p->batch);
    if (st != CROFT_OK) {
        cudaGetLastError();
        croft_plan_destroy(p);
        return st;
    }
    *out = p;
    return CROFT_OK;
}

croft_status croft_plan_create_batched(croft_plan* out, int count, const int* dims, croft_dtype dtype) {
    return croft_plan_create_batched_mode(out, count, dims, dtype, CROFT_BATCH_AUTO);
}

croft_status croft_exec_batched_forward(croft_plan plan, void* const* in, void* const* out, void* stream) {
    if (!plan || !plan->batch) return CROFT_ERR_INVALID_ARG;
    return exec_batch(plan, in, out, stream, 0);
}

croft_status croft_exec_batched_backward(croft_plan plan, void* const* in, void* const* out, void* stream) {
    if (!plan || !plan->batch) return CROFT_ERR_INVALID_ARG;
    return exec_batch(plan, in, out, stream, 1);
}

croft_status croft_plan_set_wait_limit(croft_plan plan, long long cycles) {
    if (!plan || cycles < 1) return CROFT_ERR_INVALID_ARG;
    if (!plan->batch) return CROFT_OK;
    plan->batch->wait_cycles = cycles;
    plan->batch->graphs_dirty = true;
    return CROFT_OK;
}

croft_status croft_plan_set_test_unsatisfiable_wait(croft_plan plan, int enable) {
    if (!plan || !plan->batch) return CROFT_ERR_INVALID_ARG;
    plan->batch->extra_wait = enable ? 1 : 0;
    plan->batch->graphs_dirty = true;
    return CROFT_OK;
}

}  // extern "C"

namespace croft {

int batch_plan_mode(const croft_plan_s* p) { return p->batch ? p->batch->mode : 0; }

croft_status batch_last_status(croft_plan_s* p) {
    BatchState* b = p->batch;
    if (!b->d_scratch) return CROFT_OK;
    int st = 0;
    if (cudaMemcpy(&st, b->d_scratch + 4, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return CROFT_ERR_CUDA;
    }
    return st == 0 ? CROFT_OK : (croft_status)st;
}

size_t batch_workspace_bytes(const croft_plan_s* p) {
    const BatchState* b = p->batch;
    return b->d_scratch ? sizeof(int) * (size_t)b->scratch_ints : 0;
}

int batch_num_launches(const croft_plan_s* p) {
    const BatchState* b = p->batch;
    int n = 0;
    if (!b->pgrid.empty())
        n += b->mode == CROFT_BATCH_PER_PASS ? 3 : (b->mode == CROFT_BATCH_GROUPED ? group_state_launches(b->group) : 1);
    for (croft_plan sp : b->subplans) n += croft_plan_num_launches(sp);
    return n;
}

std::string batch_describe(const croft_plan_s* p) {
    const BatchState* b = p->batch;
    static const char* names[5] = {"auto", "one_launch", "per_pass", "per_grid", "grouped"};
    char tmp[512];
    snprintf(tmp, sizeof(tmp),
             "batch of %d grids, schedule %s (persistent grids %d, items %d, blocks %d, smem %d; grouped launches %d;"
             " single-grid plans %d) tuned_us one_launch=%.1f per_pass=%.1f per_grid=%.1f grouped=%.1f",
             b->count, names[b->mode], (int)b->pgrid.size(), b->nitems, b->blocks, b->smem,
             group_state_launches(b->group), (int)b->subplans.size(), b->tuned_us[1], b->tuned_us[2], b->tuned_us[3],
             b->tuned_us[4]);
    return tmp;
}

}  // namespace croft
