// croft_internal.h - descriptors shared by the planner (host) and the pass kernels.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "croft_coldiv.h"
#include "croft_sched.h"

namespace croft {

// How the pencils of one pass sit in memory.
//  ROW: pencil g occupies elements [g*n, g*n + n)  (the contiguous z axis).
//  COL: pencil g = b*M + m has element a at b*n*M + a*M + m (a strided axis;
//       consecutive pencils are consecutive in memory, so a CTA that takes W
//       consecutive pencils reads W-wide contiguous rows of the tile).
enum PassLayout { LAYOUT_ROW = 0, LAYOUT_COL = 1 };

// One pass = one batched 1D FFT over every pencil of one axis (one kernel launch).
struct PassArgs {
    const float2* tw;   // device twiddle table of the axis, n-1 entries
    long long M;        // COL: pencils per batch row (= element stride of the axis); ROW: 1
    long long ncols;    // number of pencils
    int n;              // FFT length (the kernel is specialised on it; kept for dispatch)
    int W;              // pencils per CTA
    int tw_pad;         // float2 slots reserved for twiddles in shared memory
    float isign;        // +1 forward, -1 backward (conj-in / conj-out)
    const double2* tw64;        // complex128 passes: the twiddle table in double precision
    const unsigned char* tc_b;  // tensor-core passes: 16-point DFT matrix, bf16 hi | lo, core-matrix layout (4 KB)
    int* status;                // tensor-core passes: device status word (bounded waits), may be null
    const float2* tw2;          // pair passes: the combine twiddles w_n^k, k < n/2
    CroftColDiv cdiv;           // COL passes: col / M as a multiply-high (croft_coldiv.h); m = 0: divide
};

#ifdef __CUDACC__
// Batch row b = col / M and column m = col % M of pencil col of a COL pass.
__device__ __forceinline__ void col_split(long long col, const PassArgs& A, long long& b, long long& m) {
    if (A.cdiv.m) {
        const unsigned c32 = (unsigned)col;
        const unsigned q = croft_coldiv_q(A.cdiv.m, A.cdiv.s1, A.cdiv.s2, c32);
        b = q;
        m = c32 - q * (unsigned)A.M;
    } else {
        b = col / A.M;
        m = col - b * A.M;
    }
}
#endif

// Fused z+y pass: 2D FFT of every yz-plane (one plane per cluster of C CTAs).
struct PlaneArgs {
    const float2* tw_z;  // twiddle table of the z axis (nz-1 entries)
    const float2* tw_y;  // twiddle table of the y axis (ny-1 entries)
    int* status;         // device status word for the bounded exchange wait, may be null
    float isign;
};

typedef void (*pass_fn)(const float2*, float2*, const PassArgs);
typedef void (*pass64_fn)(const double2*, double2*, const PassArgs);
// fused convolution pass (croft_conv_kernel.cuh): the extra operand is the real influence function
typedef void (*conv_fn)(const float2*, float2*, const float*, const PassArgs);
typedef void (*conv64_fn)(const double2*, double2*, const double*, const PassArgs);

constexpr int kRingTileWidth = 16;  // columns per tile of the ring column kernel (128-byte rows)
constexpr int kPairTileWidth = 16;  // columns per tile of the cluster-pair column kernel

// Column pass fed by tensor copies through a ring of tile buffers (croft_ring_kernel.cuh).
struct RingArgs {
    const float2* tw;          // twiddle table of the axis (N-1 entries, the column schedule)
    long long M;               // element stride of the axis (inner extent of the tensor map)
    long long ntiles;          // batch rows x tiles_per_row
    long long tiles_per_row;   // ceil(M / 16)
    long long wait_cycles;     // bound of every mbarrier wait (SM clocks)
    int* status;               // device status word (CROFT_ERR_TIMEOUT), may be null
    int box_rows;              // rows per tensor-map box (divides N, <= 256)
    int tw_pad;                // float2 slots reserved for twiddles in shared memory
    float isign;               // +1 forward, -1 backward (conj-in / conj-out)
};
typedef void (*ring_fn)(const float2*, float2*, const RingArgs, const CUtensorMap);
typedef void (*plane_fn)(const float2*, float2*, const PlaneArgs);

struct PlaneKernel {
    plane_fn fn;
    int ny, nz, cluster, threads, smem;
};

enum PassKind { PASS_AXIS = 0, PASS_PLANE = 1 };

struct PassLaunch {
    int kind;           // PASS_AXIS or PASS_PLANE
    long long offset;   // element offset of this launch's sub-grid (slab schedule), 0 otherwise
    int src_in;         // 1: reads the exec's `in` (first pass over its elements); 0: reads `out`
    int group;          // logical pass this launch belongs to (per-pass timing)
    PassArgs args;      // PASS_AXIS
    PlaneArgs pargs;    // PASS_PLANE
    PlaneKernel pk;     // PASS_PLANE
    int layout;
    int tc;             // tensor-core variant of the pass kernel: 0 none, 1 + operand precision (TcPrec)
    int f64;            // 1: complex128 pass kernel
    int sv;             // schedule variant of a plain pass kernel (croft_pass_sched_v)
    int th;             // threads per pencil of a plain COL pass kernel if not the rule's (0: the rule's)
    int pair;           // 1: cluster-pair column kernel (croft_pair_kernel.cuh)
    int ring;           // 1: tensor-copy ring kernel (RingArgs below)
    RingArgs ra;
    long long B;        // ring: outer extent of the tensor map (batch rows)
    int T;              // threads per pencil (fixed by the kernel: croft_threads_per_pencil)
    int grid;
    int block;
    int smem;           // dynamic shared memory bytes
};

// croft_planes.cu
// fused kernel for an ny x nz plane with the given cluster size (<= 0: the default one); NULL if none
const PlaneKernel* find_plane_kernel(int ny, int nz, int cluster);

// croft_ring.cu: the tensor-copy ring column kernel (NULL if not instantiated for n)
ring_fn ring_kernel_for(int n);
// croft_pair.cu: the cluster-pair column kernel (NULL if not instantiated for n)
pass_fn pair_kernel_for(int n);
// Launch shape of a pair column pass (2-CTA clusters over 16-column tiles); false when the
// pass does not qualify or no cluster fits.
bool shape_pair(PassLaunch& L, int n, long long M, long long ncols);

// croft_kernels.cu, one per size group (w: the COL tile width, ignored for ROW; sv: the
// schedule variant, croft_pass_sched_v; th: threads per pencil if not the rule's, else 0)
pass_fn lookup_pass_kernel_group_0(int layout, int n, int w, int sv, int th);
pass_fn lookup_pass_kernel_group_1(int layout, int n, int w, int sv, int th);
pass_fn lookup_pass_kernel_group_2(int layout, int n, int w, int sv, int th);
pass_fn lookup_pass_kernel_group_3(int layout, int n, int w, int sv, int th);

// croft_tc.cu: tensor-core pass kernels (NULL when n has no instantiation); prec 0 = split
// bf16, 1 = split fp16 with per-butterfly power-of-two scaling (TcPrec)
pass_fn tc_pass_kernel_for(int layout, int n, int prec);
void tc_dft16_matrix(unsigned char* out4096, int prec);  // B operand (hi | lo) in the kernels' smem layout

// croft_alloc.cu: all library allocations (failure injection for tests)
cudaError_t dev_alloc(void** p, size_t bytes);
void dev_free(void* p);
cudaError_t host_alloc(void** p, size_t bytes);
void host_free(void* p);

// croft_kernels64.cu: complex128 pass kernels (NULL when n has no instantiation; w: COL tile
// width, 0 = the default one)
pass64_fn pass64_kernel_for(int layout, int n, int w = 0);

// croft_conv.cu: fused convolution pass kernels (NULL when n has no instantiation)
conv_fn lookup_conv_kernel_group_0(int n);
conv_fn lookup_conv_kernel_group_1(int n);
conv_fn lookup_conv_kernel_group_2(int n);
conv_fn lookup_conv_kernel_group_3(int n);
conv64_fn conv64_kernel_for(int n);
// out = in * g elementwise (complex times real), n elements
cudaError_t launch_scale(const void* in, void* out, const void* g, long long n, bool f64, cudaStream_t s,
                         bool pdl = false);

// croft_passes.cu
extern int g_max_smem;  // the device's opt-in shared memory per block (set by plan creation)
// Launch shape of one axis pass (tile width, block, grid, shared memory); false when no shape fits.
bool shape_pass(PassLaunch& L, int layout, int n, long long M, long long ncols, int tc = 0, bool f64 = false,
                int want_w = 0, int sv = 0, int th = 0);
pass_fn pass_kernel_for(int layout, int n, int w, int sv = 0, int th = 0);
conv_fn conv_kernel_for(int n);
// Launch shape of a ring column pass (one persistent CTA per SM); false when the pass does not
// qualify (length, odd stride, shared memory).
bool shape_ring(PassLaunch& L, int n, long long M, long long ncols);
cudaError_t prepare_pass(const PassLaunch& L);  // once per plan: shared-memory / cluster opt-ins, occupancy check
// pdl: launch with programmatic stream serialisation (ignored for kernels that do not wait for it)
cudaError_t launch_pass(const PassLaunch& L, const void* in, void* out, cudaStream_t s, bool pdl = false);
bool pass_supports_pdl(const PassLaunch& L);
// the fused convolution pass (args/shape of a COL pass; g: the real influence function)
cudaError_t launch_conv(const PassLaunch& L, const void* in, void* out, const void* g, cudaStream_t s, bool pdl = false);
int active_clusters(const PassLaunch& L);  // co-resident clusters of a plane pass (0 for axis passes)

}  // namespace croft
