// croft_batch_group.cu - the grouped schedule of batched plans (CROFT_BATCH_GROUPED):
// for each pass, one launch per distinct axis length over all grids that have it
// (croft_group_kernel.cuh), the launches of a pass concurrent in the plan's CUDA
// graph, the passes ordered by graph edges.
//
// Paper mapping: "option 4" of Sec. 5.1 - one 1D plan (here: one specialised
// kernel) reused for every pencil of that length, across grids as well.
#include <cuda_runtime.h>

#include <string.h>

#include <algorithm>
#include <map>
#include <new>
#include <vector>

#include "../../include/croft.h"
#include "croft_group_kernel.cuh"
#include "croft_sizes.h"

namespace croft {

typedef void (*group_fn)(const GroupArgs);

static group_fn group_kernel_for(int layout, int n) {
    switch (n) {
#define CROFT_G_CASE(N) \
    case N: return layout == LAYOUT_ROW ? croft_group_kernel<LAYOUT_ROW, N> : croft_group_kernel<LAYOUT_COL, N>;
        CROFT_BATCH_SIZES(CROFT_G_CASE)
#undef CROFT_G_CASE
        default: return nullptr;
    }
}

int host_build_twiddles(int n, float* out);  // croft_plan.cu

struct GroupLaunch {
    int pass, layout, n;
    int seg_begin, nseg;  // segments [seg_begin, seg_begin + nseg) of the segment table
    int cta_begin, ctas;  // entries of the CTA map
    int W, block, smem;
    int tw_off;           // float2 offset of N's twiddles in the pool
};

struct GroupState {
    std::vector<GroupLaunch> launches;
    std::vector<int> seg_grid;   // batch index of each segment
    std::vector<int> seg_first;  // 1: the segment's pass is its grid's first pass (reads `in`)
    GroupSeg* staging = nullptr; // pinned, pointers filled per exec
    GroupSeg* d_segs = nullptr;
    unsigned short* d_cta = nullptr;
    float2* d_tw = nullptr;
    int nseg = 0;
};

void group_state_destroy(GroupState* s) {
    if (!s) return;
    if (s->staging) host_free(s->staging);
    dev_free(s->d_segs);
    dev_free(s->d_cta);
    dev_free(s->d_tw);
    delete s;
}

// Builds the launches of the grids `pgrid` (axes all in the batched size list).
croft_status group_state_build(const std::vector<int>& dims, const std::vector<int>& pgrid, GroupState** out) {
    *out = nullptr;
    GroupState* s = new (std::nothrow) GroupState();
    if (!s) return CROFT_ERR_OOM;
    static const int kAxis[3] = {2, 1, 0};
    std::vector<GroupSeg> segs;
    std::vector<unsigned short> cta;
    std::vector<float> pool;
    std::map<int, int> tw_off;
    // first pass of each grid (lowest pass index whose axis is longer than 1)
    std::vector<int> first(pgrid.size(), -1);
    for (size_t i = 0; i < pgrid.size(); ++i)
        for (int p = 0; p < 3 && first[i] < 0; ++p)
            if (dims[3 * pgrid[i] + kAxis[p]] > 1) first[i] = p;
    for (int p = 0; p < 3; ++p) {
        std::map<std::pair<int, int>, std::vector<int>> by_len;  // (layout, n) -> grids
        for (size_t i = 0; i < pgrid.size(); ++i) {
            const int g = pgrid[i];
            const int n = dims[3 * g + kAxis[p]];
            if (n <= 1) continue;
            const int nz = dims[3 * g + 2], ny = dims[3 * g + 1];
            const long long M = kAxis[p] == 2 ? 1 : (kAxis[p] == 1 ? (long long)nz : (long long)ny * nz);
            by_len[{M == 1 ? LAYOUT_ROW : LAYOUT_COL, n}].push_back((int)i);
        }
        for (auto& kv : by_len) {
            const int layout = kv.first.first, n = kv.first.second;
            group_fn f = group_kernel_for(layout, n);
            if (!f) {
                group_state_destroy(s);
                return CROFT_ERR_UNSUPPORTED_SIZE;
            }
            if (!tw_off.count(n)) {
                tw_off[n] = (int)(pool.size() / 2);
                std::vector<float> t(2 * (size_t)n + 2, 0.f);
                if (n > 1 && host_build_twiddles(n, t.data()) != n - 1) {
                    group_state_destroy(s);
                    return CROFT_ERR_UNSUPPORTED_SIZE;
                }
                pool.insert(pool.end(), t.begin(), t.begin() + 2 * std::max(1, n - 1));
            }
            const int T = croft_threads_per_pencil(n);
            const int tw_pad = ((n + 1) / 2) * 2;
            GroupLaunch L;
            L.pass = p;
            L.layout = layout;
            L.n = n;
            L.W = layout == LAYOUT_ROW ? 256 / T : croft_col_width(n, 8);
            L.block = L.W * T;
            const long long tile_elems = layout == LAYOUT_ROW ? (long long)L.W * croft_row_ld_staged(n) : (long long)n * L.W;
            L.smem = (int)((tw_pad + tile_elems) * sizeof(float2));
            L.tw_off = tw_off[n];
            L.seg_begin = (int)segs.size();
            L.cta_begin = (int)cta.size();
            for (int i : kv.second) {
                const int g = pgrid[i];
                const long long N = (long long)dims[3 * g] * dims[3 * g + 1] * dims[3 * g + 2];
                GroupSeg S;
                memset(&S, 0, sizeof(S));
                const int nz = dims[3 * g + 2], ny = dims[3 * g + 1];
                S.M = kAxis[p] == 2 ? 1 : (kAxis[p] == 1 ? (long long)nz : (long long)ny * nz);
                S.ncols = N / n;
                S.cdiv = croft_coldiv_make(S.M, S.ncols + L.W);
                S.first_tile = (int)(cta.size() - L.cta_begin);
                const long long tiles = (S.ncols + L.W - 1) / L.W;
                const int seg_local = (int)segs.size() - L.seg_begin;
                if (seg_local > 65535 || (long long)cta.size() - L.cta_begin + tiles > 0x7fffffffLL) {
                    group_state_destroy(s);
                    return CROFT_ERR_UNSUPPORTED_SIZE;
                }
                for (long long t = 0; t < tiles; ++t) cta.push_back((unsigned short)seg_local);
                segs.push_back(S);
                s->seg_grid.push_back(g);
                s->seg_first.push_back(first[i] == p ? 1 : 0);
            }
            L.nseg = (int)segs.size() - L.seg_begin;
            L.ctas = (int)cta.size() - L.cta_begin;
            if (L.smem > 48 * 1024 && cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, L.smem) != cudaSuccess) {
                cudaGetLastError();
                group_state_destroy(s);
                return CROFT_ERR_CUDA;
            }
            s->launches.push_back(L);
        }
    }
    s->nseg = (int)segs.size();
    if (s->nseg == 0) {
        *out = s;
        return CROFT_OK;
    }
    if (host_alloc((void**)&s->staging, sizeof(GroupSeg) * s->nseg) != cudaSuccess ||
        dev_alloc((void**)&s->d_segs, sizeof(GroupSeg) * s->nseg) != cudaSuccess ||
        dev_alloc((void**)&s->d_cta, sizeof(unsigned short) * std::max<size_t>(1, cta.size())) != cudaSuccess ||
        dev_alloc((void**)&s->d_tw, sizeof(float) * std::max<size_t>(2, pool.size())) != cudaSuccess) {
        cudaGetLastError();
        group_state_destroy(s);
        return CROFT_ERR_OOM;
    }
    memcpy(s->staging, segs.data(), sizeof(GroupSeg) * s->nseg);
    if (cudaMemcpy(s->d_cta, cta.data(), sizeof(unsigned short) * cta.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        (!pool.empty() && cudaMemcpy(s->d_tw, pool.data(), sizeof(float) * pool.size(), cudaMemcpyHostToDevice) != cudaSuccess)) {
        cudaGetLastError();
        group_state_destroy(s);
        return CROFT_ERR_CUDA;
    }
    *out = s;
    return CROFT_OK;
}

// The grids' pointers for one exec (into the pinned staging table the graph uploads).
void group_state_fill(GroupState* s, void* const* in, void* const* out) {
    for (int k = 0; k < s->nseg; ++k) {
        const int g = s->seg_grid[k];
        s->staging[k].in = (const float2*)(s->seg_first[k] ? in[g] : out[g]);
        s->staging[k].out = (float2*)out[g];
    }
}

// Adds [segment upload] -> pass 0 launches -> pass 1 launches -> pass 2 launches to g.
// With pdl, the edges from one pass's launches to the next pass's are programmatic:
// the next pass's CTAs may become resident (and load their twiddles) while the
// previous pass drains, and wait in the kernel (griddepcontrol.wait) for every
// upstream launch to complete before they read the grid.
croft_status group_graph_add(GroupState* s, cudaGraph_t g, float isign, bool pdl) {
    if (s->nseg == 0) return CROFT_OK;
    cudaGraphNode_t up;
    if (cudaGraphAddMemcpyNode1D(&up, g, nullptr, 0, s->d_segs, s->staging, sizeof(GroupSeg) * s->nseg,
                                 cudaMemcpyHostToDevice) != cudaSuccess)
        return CROFT_ERR_CUDA;
    std::vector<cudaGraphNode_t> prev = {up};
    for (int p = 0; p < 3; ++p) {
        std::vector<cudaGraphNode_t> cur;
        for (const GroupLaunch& L : s->launches) {
            if (L.pass != p) continue;
            GroupArgs A;
            memset(&A, 0, sizeof(A));
            A.segs = s->d_segs + L.seg_begin;
            A.cta_seg = s->d_cta + L.cta_begin;
            A.tw = s->d_tw + L.tw_off;
            A.W = L.W;
            A.isign = isign;
            void* params[1] = {&A};
            cudaKernelNodeParams kp;
            memset(&kp, 0, sizeof(kp));
            kp.func = (void*)group_kernel_for(L.layout, L.n);
            kp.gridDim = dim3((unsigned)L.ctas, 1, 1);
            kp.blockDim = dim3((unsigned)L.block, 1, 1);
            kp.sharedMemBytes = (unsigned)L.smem;
            kp.kernelParams = params;
            cudaGraphNode_t kn;
            if (p == 0 || !pdl) {
                if (cudaGraphAddKernelNode(&kn, g, prev.data(), prev.size(), &kp) != cudaSuccess) return CROFT_ERR_CUDA;
            } else {
                if (cudaGraphAddKernelNode(&kn, g, nullptr, 0, &kp) != cudaSuccess) return CROFT_ERR_CUDA;
                std::vector<cudaGraphNode_t> to(prev.size(), kn);
                std::vector<cudaGraphEdgeData> ed(prev.size());
                for (cudaGraphEdgeData& e : ed) {
                    memset(&e, 0, sizeof(e));
                    e.from_port = cudaGraphKernelNodePortProgrammatic;
                    e.type = cudaGraphDependencyTypeProgrammatic;
                }
                if (cudaGraphAddDependencies(g, prev.data(), to.data(), ed.data(), prev.size()) != cudaSuccess) {
                    cudaGetLastError();  // programmatic edges refused: plain edges (the kernel's wait returns at once)
                    if (cudaGraphAddDependencies(g, prev.data(), to.data(), nullptr, prev.size()) != cudaSuccess)
                        return CROFT_ERR_CUDA;
                }
            }
            cur.push_back(kn);
        }
        if (!cur.empty()) prev = cur;
    }
    return CROFT_OK;
}

int group_state_launches(const GroupState* s) { return s ? (int)s->launches.size() : 0; }

}  // namespace croft
