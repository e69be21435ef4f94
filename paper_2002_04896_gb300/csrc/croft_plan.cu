// croft_plan.cu - planner, twiddle tables and the C ABI entry points (include/croft.h).
//
// A plan is the GPU counterpart of the paper's single reusable 1D FFT plan that
// covers every pencil of an axis ("option 4", Sec. 5.1), extended to the whole
// three-axis schedule of Sec. 4.1: it fixes, per axis, the radix order, the
// twiddle table and the launch shape of the pass, and uploads the tables once.
// Exec then only launches the passes (z, then y, then x).
#include <cuda_runtime.h>

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "../../include/croft.h"
#include "croft_internal.h"
#include "croft_plan_internal.h"

using namespace croft;

// ---------------------------------------------------------------------------
// host planning helpers
// ---------------------------------------------------------------------------

static bool axis_supported(int n) { return croft_make_sched(n).count >= 0; }

static int factorize(int n, int* r, int cap) {
    CroftSched sc = croft_make_sched(n);
    if (sc.count < 0 || sc.count > cap) return -1;
    for (int i = 0; i < sc.count; ++i) r[i] = sc.r[i];
    return sc.count;
}

// exp(-2 pi i r / N) in float64, 0 <= r < N, with the angle reduced to the
// first quadrant by integer arithmetic so that multiples of a quarter turn
// are exact (1, -i, -1, i) and the two halves of a quadrant are mirror images.
static void twiddle64(long long r, long long N, double* re, double* im) {
    long long q = (4 * r) / N;
    long long rem = 4 * r - q * N;  // angle = (q + rem/N) * pi/2
    double c, s;
    if (2 * rem <= N) {
        double ph = (M_PI / 2.0) * (double)rem / (double)N;
        c = cos(ph);
        s = sin(ph);
    } else {
        double ph = (M_PI / 2.0) * (double)(N - rem) / (double)N;
        c = sin(ph);
        s = cos(ph);
    }
    double x = c, y = -s;  // exp(-i phi)
    for (long long t = 0; t < (q & 3); ++t) {  // times (-i)^q
        double nx = y, ny = -x;
        x = nx;
        y = ny;
    }
    *re = x;
    *im = y;
}

// The same table in double precision (complex128 plans).
static int build_twiddles64(int n, const int* radices, int ns, double* out) {
    int p = 1;
    for (int s = 0; s < ns; ++s) {
        int R = radices[s];
        if (R < 2 || p * R > n) return -1;
        for (int j = 1; j < R; ++j)
            for (int k = 0; k < p; ++k) {
                double re, im;
                twiddle64((long long)j * k, (long long)p * R, &re, &im);
                long long idx = (long long)(p - 1) + (long long)(j - 1) * p + k;
                out[2 * idx] = re;
                out[2 * idx + 1] = im;
            }
        p *= R;
    }
    return p == n ? n - 1 : -1;
}

static int build_twiddles(int n, const int* radices, int ns, float* out) {
    int p = 1;
    for (int s = 0; s < ns; ++s) {
        int R = radices[s];
        if (R < 2 || p * R > n) return -1;
        for (int j = 1; j < R; ++j)
            for (int k = 0; k < p; ++k) {
                double re, im;
                twiddle64((long long)j * k, (long long)p * R, &re, &im);
                long long idx = (long long)(p - 1) + (long long)(j - 1) * p + k;
                out[2 * idx] = (float)re;
                out[2 * idx + 1] = (float)im;
            }
        p *= R;
    }
    return p == n ? n - 1 : -1;
}

namespace croft {
// twiddle table of a length-n axis in the library's schedule (n-1 entries); used by batched plans
int host_build_twiddles(int n, float* out) {
    int rad[CROFT_MAX_STAGES];
    const int ns = factorize(n, rad, CROFT_MAX_STAGES);
    if (ns < 1) return -1;
    return build_twiddles(n, rad, ns, out);
}
int batch_plan_mode(const croft_plan_s* p);
croft_status batch_last_status(croft_plan_s* p);
size_t batch_workspace_bytes(const croft_plan_s* p);
int batch_num_launches(const croft_plan_s* p);
std::string batch_describe(const croft_plan_s* p);
}  // namespace croft

// (shape_pass and the device's shared-memory limit g_max_smem live in croft_passes.cu)

extern "C" {

const char* croft_status_string(croft_status s) {
    switch (s) {
        case CROFT_OK: return "CROFT_OK";
        case CROFT_ERR_INVALID_ARG: return "CROFT_ERR_INVALID_ARG";
        case CROFT_ERR_UNSUPPORTED_SIZE: return "CROFT_ERR_UNSUPPORTED_SIZE";
        case CROFT_ERR_OOM: return "CROFT_ERR_OOM";
        case CROFT_ERR_CUDA: return "CROFT_ERR_CUDA";
        case CROFT_ERR_TIMEOUT: return "CROFT_ERR_TIMEOUT";
    }
    return "CROFT_ERR_UNKNOWN";
}

int croft_factorize(int n, int* radices, int cap) {
    if (!radices || cap < 0) return -1;
    return factorize(n, radices, cap);
}

int croft_twiddle_table(int n, const int* radices, int nstages, float* out) {
    if (!out || (!radices && nstages > 0) || n < 1 || n > CROFT_MAX_N) return -1;
    if (n == 1) return nstages == 0 ? 0 : -1;
    return build_twiddles(n, radices, nstages, out);
}

croft_status croft_plan_destroy(croft_plan plan) {
    if (!plan) return CROFT_OK;
    int cur = -1;
    cudaGetDevice(&cur);
    cudaSetDevice(plan->device);
    for (int a = 0; a < 3; ++a) {
        dev_free(plan->tw_dev[a]);
        dev_free(plan->tw_pair[a]);
    }
    dev_free(plan->tw_conv);
    for (cudaEvent_t e : plan->ev)
        if (e) cudaEventDestroy(e);
    if (plan->batch) batch_state_destroy(plan->batch);
    if (plan->stream) stream_state_destroy(plan->stream);
    dev_free(plan->tc_b);
    dev_free(plan->d_status);
    if (cur >= 0) cudaSetDevice(cur);
    delete plan;
    return CROFT_OK;
}

static croft_status fail(croft_plan p, croft_status st) {
    cudaGetLastError();
    croft_plan_destroy(p);
    return st;
}

// Axis pass (z: ROW; y, x: COL) of the three-pass schedule, or the x pass of the fused one.
// Axis pass over x-planes [x0, x0 + nxs) (the whole grid unless the slab schedule asks for less).
// Whether an axis's column passes run the tensor-copy ring kernel (croft_ring_default, a tuned
// plan's choice, or CROFT_RING=1 / 0 for measurement).
static bool ring_selected(croft_plan p, int axis) {
    const int n = p->dims[axis];
    const long long M = (axis == 2) ? 1 : (axis == 1 ? (long long)p->dims[2] : (long long)p->dims[1] * p->dims[2]);
    if (M == 1 || p->dtype == CROFT_C2C_F64 || p->axis_tc[axis]) return false;
    const int kind = p->axis_kind[axis];
    const char* re = getenv("CROFT_RING");
    return kind >= 0 ? kind == 1 : (re ? re[0] == '1' : croft_ring_default(n, 8, M * 8));
}

// The schedule variant of an axis's plain passes under the rules (croft_col_sv_default): complex64
// column passes of 32-thread pencils only (tensor-core axes take their own schedule, the ring
// kernel the rule's split, both from the axis's table).
static int rules_sv(croft_plan p, int axis) {
    const int n = p->dims[axis];
    const long long M = (axis == 2) ? 1 : (axis == 1 ? (long long)p->dims[2] : (long long)p->dims[1] * p->dims[2]);
    if (M == 1 || p->dtype == CROFT_C2C_F64 || p->axis_tc[axis] || croft_threads_per_pencil(n) != 32) return 0;
    if (ring_selected(p, axis)) return 0;
    return croft_col_sv_default(n, 8, M * 8);
}

static croft_status add_axis_pass(croft_plan p, int axis, int x0 = 0, int nxs = -1, int group = -1, int src_in = -1) {
    const int nx = nxs < 0 ? p->dims[0] : nxs, ny = p->dims[1], nz = p->dims[2];
    const long long N = (long long)nx * ny * nz;
    const long long offset = (long long)x0 * ny * nz;
    const int grp = group < 0 ? p->ngroups : group;
    const int sin = src_in < 0 ? (p->passes.empty() ? 1 : 0) : src_in;
    const int n = p->dims[axis];
    // element stride of the axis; a unit stride means the pencils are contiguous rows
    const long long M = (axis == 2) ? 1 : (axis == 1 ? (long long)nz : (long long)ny * nz);
    const int layout = M == 1 ? LAYOUT_ROW : LAYOUT_COL;
    const bool f64 = p->dtype == CROFT_C2C_F64;
    // The tensor-copy ring kernel serves column passes of 32-thread pencils when the rules
    // (croft_ring_default) or a tuned plan pick it; CROFT_RING=1 takes it for every such column
    // pass, CROFT_RING=0 for none (both for measurement).
    const int kind = p->axis_kind[axis];
    const bool ring_pass = layout == LAYOUT_COL && ring_selected(p, axis);
    // The cluster-pair kernel (croft_pair_kernel.cuh): tuned plans (kind 2) or CROFT_PAIR=1.
    const char* pe = getenv("CROFT_PAIR");
    const bool pair_pass = layout == LAYOUT_COL && !f64 && !p->axis_tc[axis] && !ring_pass &&
                           (kind >= 0 ? kind == 2 : (pe ? pe[0] == '1' : croft_pair_default(n, 8, M * 8)));
    if (pair_pass) {
        PassLaunch L;
        if (shape_pair(L, n, M, N / n)) {
            const int n2 = n / 2;
            if (!p->tw_pair[axis]) {
                // [the half length's table in its column schedule | w_n^k, k < n/2], float64 -> float32
                std::vector<float> tw(4 * (size_t)n2 + 2, 0.f);
                const CroftSched hs = croft_pass_sched(n2, LAYOUT_COL, 8);
                if (n2 > 1 && build_twiddles(n2, hs.r, hs.count, tw.data()) != n2 - 1) return CROFT_ERR_UNSUPPORTED_SIZE;
                for (int k = 0; k < n2; ++k) {
                    double re, im;
                    twiddle64(k, n, &re, &im);
                    tw[2 * ((size_t)n2 + k)] = (float)re;
                    tw[2 * ((size_t)n2 + k) + 1] = (float)im;
                }
                if (dev_alloc((void**)&p->tw_pair[axis], sizeof(float2) * 2 * (size_t)n2) != cudaSuccess) return CROFT_ERR_OOM;
                if (cudaMemcpy(p->tw_pair[axis], tw.data(), sizeof(float2) * 2 * (size_t)n2, cudaMemcpyHostToDevice) != cudaSuccess)
                    return CROFT_ERR_CUDA;
            }
            L.args.tw = p->tw_pair[axis];
            L.args.tw2 = p->tw_pair[axis] + n2;
            L.args.status = p->d_status;
            L.offset = offset;
            L.src_in = sin;
            L.group = grp;
            if (prepare_pass(L) == cudaSuccess) {
                p->passes.push_back(L);
                p->pass_axis.push_back(axis);
                if (grp >= p->ngroups) p->ngroups = grp + 1;
                return CROFT_OK;
            }
            cudaGetLastError();
        }
    }
    if (ring_pass) {
        PassLaunch L;
        if (shape_ring(L, n, M, N / n)) {
            L.args.tw = p->tw_dev[axis];
            L.args.status = p->d_status;
            L.offset = offset;
            L.src_in = sin;
            L.group = grp;
            if (prepare_pass(L) == cudaSuccess) {
                p->passes.push_back(L);
                p->pass_axis.push_back(axis);
                if (grp >= p->ngroups) p->ngroups = grp + 1;
                return CROFT_OK;
            }
            cudaGetLastError();
        }
    }
    PassLaunch L;
    int want_w = kind == 0 ? p->axis_w[axis] : 0, sv = kind == 0 ? p->axis_sv[axis] : rules_sv(p, axis);
    int th = kind == 0 ? p->axis_th[axis] : 0;
    // CROFT_COL_TH=16 (measurement): 16-column tiles with 16 threads per pencil for every column
    // pass of 32-thread pencils that a plan's rules would give the plain kernel
    const char* te = getenv("CROFT_COL_TH");
    if (kind < 0 && te && atoi(te) == 16 && layout == LAYOUT_COL && !f64 && !p->axis_tc[axis] &&
        croft_threads_per_pencil(n) == 32) {
        th = 16;
        want_w = croft_col_width(n, 8);
    }
    // the rules' 24- and 16-thread pencils (croft_col_t24, croft_col_t16), unless CROFT_COL_TH
    // asked for 16
    if (kind < 0 && th == 0 && layout == LAYOUT_COL && !f64 && !p->axis_tc[axis] && croft_threads_per_pencil(n) == 32) {
        const int w = croft_col_width_at(n, 8, M * 8);
        if (croft_col_t24(n, M * 8 <= 16 * 1024)) {
            th = 24;
            want_w = w;
        } else if (croft_col_t16(n, 8, M * 8)) {
            th = 16;
            want_w = croft_col_width(n, 8);
        }
    }
    if (!shape_pass(L, layout, n, M, N / n, p->axis_tc[axis] ? 1 + p->tc_prec : 0, f64, want_w, sv, th))
        return CROFT_ERR_UNSUPPORTED_SIZE;
    L.kind = PASS_AXIS;
    L.args.tw = p->tw_dev[axis];
    L.args.tw64 = f64 ? (const double2*)p->tw_dev[axis] : nullptr;
    L.args.tc_b = p->tc_b;
    L.args.status = p->d_status;
    L.offset = offset;
    L.src_in = sin;
    L.group = grp;
    if (prepare_pass(L) != cudaSuccess) return CROFT_ERR_CUDA;
    p->passes.push_back(L);
    p->pass_axis.push_back(axis);
    if (grp >= p->ngroups) p->ngroups = grp + 1;
    return CROFT_OK;
}

// Slab schedule: for each slab of x-planes the z pass then the y pass (the y pass
// finds the z output in L2), all in logical pass 0; then the x pass.
static croft_status add_slab_passes(croft_plan p, int planes) {
    const int nx = p->dims[0], ny = p->dims[1], nz = p->dims[2];
    for (int x0 = 0; x0 < nx; x0 += planes) {
        const int nxs = (nx - x0 < planes) ? nx - x0 : planes;
        bool first = true;
        if (nz > 1) {
            croft_status st = add_axis_pass(p, 2, x0, nxs, 0, 1);
            if (st != CROFT_OK) return st;
            first = false;
        }
        if (ny > 1) {
            croft_status st = add_axis_pass(p, 1, x0, nxs, 0, first ? 1 : 0);
            if (st != CROFT_OK) return st;
        }
    }
    if (nx > 1) return add_axis_pass(p, 0, 0, -1, p->passes.empty() ? 0 : 1, p->passes.empty() ? 1 : 0);
    return CROFT_OK;
}

// Fused z+y pass over every yz-plane (croft_plane_kernel.cuh).
static croft_status add_plane_pass(croft_plan p, const PlaneKernel* pk) {
    PassLaunch L;
    memset(&L, 0, sizeof(L));
    L.kind = PASS_PLANE;
    L.pk = *pk;
    L.pargs.tw_z = p->tw_dev[2];
    L.pargs.tw_y = p->tw_dev[1];
    L.pargs.status = p->d_status;
    L.grid = p->dims[0] * pk->cluster;
    L.block = pk->threads;
    L.smem = pk->smem;
    L.args.n = pk->ny * pk->nz;
    L.src_in = 1;
    L.group = p->ngroups;
    if (L.smem > g_max_smem) return CROFT_ERR_UNSUPPORTED_SIZE;
    if (prepare_pass(L) != cudaSuccess) return CROFT_ERR_CUDA;
    p->passes.push_back(L);
    p->pass_axis.push_back(3);
    p->ngroups += 1;
    return CROFT_OK;
}

// Fused convolution pass for croft_exec_convolve: it replaces the plan's last pass
// when that pass is a plain (CUDA-core, non-pipelined) axis pass over the whole grid
// that forms a logical pass of its own; otherwise convolve runs F, multiply, B.
static void plan_conv(croft_plan p) {
    p->conv_fused = false;
    p->conv_axis = -1;
    if (p->passes.empty()) return;
    const size_t last = p->passes.size() - 1;
    const PassLaunch& Lp = p->passes[last];
    const int axis = p->pass_axis[last];
    if (Lp.kind != PASS_AXIS || Lp.offset != 0 || axis < 0 || axis > 2 || Lp.tc || p->axis_tc[axis]) return;
    if (last > 0 && p->passes[last - 1].group == Lp.group) return;
    const bool f64 = p->dtype == CROFT_C2C_F64;
    const int n = p->dims[axis];
    const long long N = (long long)p->dims[0] * p->dims[1] * p->dims[2];
    const long long M = (axis == 2) ? 1 : (axis == 1 ? (long long)p->dims[2] : (long long)p->dims[1] * p->dims[2]);
    if (f64 ? !conv64_kernel_for(n) : !conv_kernel_for(n)) return;
    // the fused kernel runs the column schedule; the axis's twiddle table follows its pass's,
    // so a pass on another schedule (the rules' or a tuned radix-16-first split) gives the
    // convolution a table of its own (complex64)
    const CroftSched sa = croft_pass_sched_v(n, Lp.layout, f64 ? 16 : 8, Lp.sv),
                     sb = croft_pass_sched(n, LAYOUT_COL, f64 ? 16 : 8);
    bool same = sa.count == sb.count;
    for (int i = 0; same && i < sa.count; ++i) same = sa.r[i] == sb.r[i];
    if (!same && f64) return;
    PassLaunch L;
    // the kernel's column width is a compile-time constant (croft_conv_width)
    const int want_w = croft_conv_width(n, f64 ? 16 : 8);
    if (!shape_pass(L, LAYOUT_COL, n, M, N / n, false, f64, want_w) || L.args.W != want_w) return;
    const long long es = f64 ? 16 : 8;
    const long long smem = ((long long)L.args.tw_pad + (long long)n * L.args.W) * es + (long long)n * L.args.W * (es / 2);
    if (smem > g_max_smem) return;
    L.smem = (int)smem;
    L.kind = PASS_AXIS;
    L.args.tw = p->tw_dev[axis];
    if (!same) {
        std::vector<float> tw(2 * (size_t)(n - 1) + 2, 0.f);
        if (build_twiddles(n, sb.r, sb.count, tw.data()) != n - 1) return;
        if (!p->tw_conv) {
            if (dev_alloc((void**)&p->tw_conv, sizeof(float2) * (size_t)n) != cudaSuccess) {
                p->tw_conv = NULL;
                return;
            }
            if (cudaMemcpy(p->tw_conv, tw.data(), sizeof(float2) * (size_t)(n - 1), cudaMemcpyHostToDevice) != cudaSuccess)
                return;
        }
        L.args.tw = p->tw_conv;
    }
    L.args.tw64 = f64 ? (const double2*)p->tw_dev[axis] : nullptr;
    L.args.status = p->d_status;
    L.group = Lp.group;
    L.src_in = Lp.src_in;
    const void* fn = f64 ? (const void*)conv64_kernel_for(n) : (const void*)conv_kernel_for(n);
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess || L.block > fa.maxThreadsPerBlock) {
        cudaGetLastError();
        return;
    }
    if (L.smem > 48 * 1024 && cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, L.smem) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    p->conv = L;
    p->conv_axis = axis;
    p->conv_fused = true;
}

// Per-axis kernel choice of a tuned plan (croft_plan_s::axis_kind / axis_w / axis_sv).
struct AxisChoice {
    int kind[3] = {-1, -1, -1};
    int w[3] = {0, 0, 0};
    int sv[3] = {0, 0, 0};
    int th[3] = {0, 0, 0};
};

static croft_status create_impl(croft_plan* out, int nx, int ny, int nz, croft_dtype dtype, croft_schedule sched,
                                const AxisChoice* choice = nullptr) {
    if (!out) return CROFT_ERR_INVALID_ARG;
    *out = NULL;
    if (dtype != CROFT_C2C_F32 && dtype != CROFT_C2C_F32_TC_BF16X3 && dtype != CROFT_C2C_F32_TC_FP16X3 &&
        dtype != CROFT_C2C_F64)
        return CROFT_ERR_INVALID_ARG;
    if (dtype == CROFT_C2C_F64) {
        // complex128: three-pass schedule on the instantiated lengths only
        if (sched == CROFT_SCHEDULE_PLANE_FUSED || sched == CROFT_SCHEDULE_SLAB_L2) return CROFT_ERR_UNSUPPORTED_SIZE;
        for (int v : {nx, ny, nz})
            if (v > 1 && !pass64_kernel_for(LAYOUT_ROW, v)) return CROFT_ERR_UNSUPPORTED_SIZE;
    }
    if (sched != CROFT_SCHEDULE_AUTO && sched != CROFT_SCHEDULE_THREE_PASS && sched != CROFT_SCHEDULE_PLANE_FUSED &&
        sched != CROFT_SCHEDULE_SLAB_L2)
        return CROFT_ERR_INVALID_ARG;  // (CROFT_SCHEDULE_TUNED resolves to one of these first)
    if (!axis_supported(nx) || !axis_supported(ny) || !axis_supported(nz)) return CROFT_ERR_UNSUPPORTED_SIZE;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return CROFT_ERR_CUDA; }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) { cudaGetLastError(); return CROFT_ERR_CUDA; }
    if (prop.major < 10) return CROFT_ERR_CUDA;  // built for sm_103a only
    g_max_smem = (int)prop.sharedMemPerBlockOptin;

    croft_plan p = new (std::nothrow) croft_plan_s();
    if (!p) return CROFT_ERR_OOM;
    p->dims[0] = nx;
    p->dims[1] = ny;
    p->dims[2] = nz;
    p->dtype = dtype;
    p->device = dev;
    for (int a = 0; a < 3; ++a) {
        p->tw_dev[a] = NULL;
        p->tw_pair[a] = NULL;
    }
    p->tw_conv = NULL;
    p->timing = false;
    p->ev_count = 0;
    p->ngroups = 0;
    p->ran = false;
    p->batch = NULL;
    p->stream = NULL;
    p->tc_b = NULL;
    p->d_status = NULL;
    p->conv_fused = false;
    p->conv_axis = -1;
    for (int a = 0; a < 3; ++a) {
        p->axis_kind[a] = choice ? choice->kind[a] : -1;
        p->axis_w[a] = choice ? choice->w[a] : 0;
        p->axis_sv[a] = choice ? choice->sv[a] : 0;
        p->axis_th[a] = choice ? choice->th[a] : 0;
    }
    const char* pdl_env = getenv("CROFT_PDL");  // 0: ordinary stream ordering between passes (for measurement)
    p->pdl = !(pdl_env && pdl_env[0] == '0');
    const bool want_tc = dtype == CROFT_C2C_F32_TC_BF16X3 || dtype == CROFT_C2C_F32_TC_FP16X3;
    const int tc_prec = dtype == CROFT_C2C_F32_TC_FP16X3 ? 1 : 0;  // TcPrec
    p->tc_prec = tc_prec;
    for (int axis = 0; axis < 3; ++axis) {
        const long long M = (axis == 2) ? 1 : (axis == 1 ? (long long)nz : (long long)ny * nz);
        // an axis with a radix-16 stage runs it on the tensor cores, or the plan is refused (no
        // silent FP32 stand-in); an axis without one has no stage to put there
        const bool radix16 = p->dims[axis] % 16 == 0;
        p->axis_tc[axis] = want_tc && radix16;
        if (p->axis_tc[axis] && !tc_pass_kernel_for(M == 1 ? LAYOUT_ROW : LAYOUT_COL, p->dims[axis], tc_prec))
            return fail(p, CROFT_ERR_UNSUPPORTED_SIZE);
    }
    if (want_tc) {
        unsigned char hb[4096];
        tc_dft16_matrix(hb, tc_prec);
        if (dev_alloc((void**)&p->tc_b, 4096) != cudaSuccess) return fail(p, CROFT_ERR_OOM);
        if (dev_alloc((void**)&p->d_status, sizeof(int)) != cudaSuccess) return fail(p, CROFT_ERR_OOM);
        if (cudaMemcpy(p->tc_b, hb, 4096, cudaMemcpyHostToDevice) != cudaSuccess) return fail(p, CROFT_ERR_CUDA);
        if (cudaMemset(p->d_status, 0, sizeof(int)) != cudaSuccess) return fail(p, CROFT_ERR_CUDA);
    }

    // twiddle tables, one per axis of length > 1 (tensor-core axes: radix-16-first schedule)
    for (int axis = 0; axis < 3; ++axis) {
        const int n = p->dims[axis];
        if (n == 1) continue;
        int rad[CROFT_MAX_STAGES];
        int ns;
        if (p->axis_tc[axis]) {
            const CroftSched sc = croft_make_sched_tc(n);
            ns = sc.count;
            for (int i = 0; i < ns; ++i) rad[i] = sc.r[i];
        } else {
            // the schedule of the axis's pass (a unit element stride makes it a row pass)
            const long long M = (axis == 2) ? 1 : (axis == 1 ? (long long)nz : (long long)ny * nz);
            const CroftSched sc = croft_pass_sched_v(n, M == 1 ? LAYOUT_ROW : LAYOUT_COL, dtype == CROFT_C2C_F64 ? 16 : 8,
                                                     p->axis_kind[axis] == 0 ? p->axis_sv[axis] : rules_sv(p, axis));
            ns = sc.count;
            for (int i = 0; i < ns; ++i) rad[i] = sc.r[i];
        }
        if (ns < 1) return fail(p, CROFT_ERR_UNSUPPORTED_SIZE);
        if (dtype == CROFT_C2C_F64) {
            std::vector<double> tw(2 * (size_t)(n - 1) + 2, 0.0);
            if (build_twiddles64(n, rad, ns, tw.data()) != n - 1) return fail(p, CROFT_ERR_UNSUPPORTED_SIZE);
            if (dev_alloc((void**)&p->tw_dev[axis], sizeof(double2) * (size_t)n) != cudaSuccess) return fail(p, CROFT_ERR_OOM);
            if (cudaMemcpy(p->tw_dev[axis], tw.data(), sizeof(double2) * (size_t)(n - 1), cudaMemcpyHostToDevice) != cudaSuccess)
                return fail(p, CROFT_ERR_CUDA);
            continue;
        }
        std::vector<float> tw(2 * (size_t)(n - 1) + 2, 0.f);
        if (build_twiddles(n, rad, ns, tw.data()) != n - 1) return fail(p, CROFT_ERR_UNSUPPORTED_SIZE);
        if (dev_alloc((void**)&p->tw_dev[axis], sizeof(float2) * (size_t)n) != cudaSuccess) return fail(p, CROFT_ERR_OOM);
        if (cudaMemcpy(p->tw_dev[axis], tw.data(), sizeof(float2) * (size_t)(n - 1), cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(p, CROFT_ERR_CUDA);
    }

    // schedule: fused yz-plane pass + x pass when a plane kernel exists for (ny, nz)
    // and its cluster fits on this device, else one pass per axis (z, y, x)
    const char* envc = getenv("CROFT_PLANE_CLUSTER");
    const int want_cluster = envc ? atoi(envc) : 0;
    const PlaneKernel* pk = (ny > 1 && nz > 1 && !want_tc && dtype != CROFT_C2C_F64) ? find_plane_kernel(ny, nz, want_cluster) : NULL;
    if (sched == CROFT_SCHEDULE_PLANE_FUSED && !pk) return fail(p, CROFT_ERR_UNSUPPORTED_SIZE);
    // AUTO takes the fused pass only when asked to (CROFT_SCHEDULE_AUTO_FUSED=1): on GB300 the
    // cluster exchange currently costs more than the HBM pass it saves.
    const char* af = getenv("CROFT_SCHEDULE_AUTO_FUSED");
    const bool auto_fused = af && af[0] == '1';
    bool fused = false;
    if (pk && (sched == CROFT_SCHEDULE_PLANE_FUSED || (sched == CROFT_SCHEDULE_AUTO && auto_fused))) {
        croft_status st = add_plane_pass(p, pk);
        if (st == CROFT_OK) {
            fused = true;
        } else {
            cudaGetLastError();
            p->passes.clear();
            p->pass_axis.clear();
            if (sched == CROFT_SCHEDULE_PLANE_FUSED) return fail(p, st);
        }
    }
    if (sched == CROFT_SCHEDULE_SLAB_L2) {
        const char* mb = getenv("CROFT_SLAB_MB");
        const double slab_bytes = (mb && atof(mb) > 0 ? atof(mb) : 16.0) * 1048576.0;
        const double plane_bytes = (double)ny * nz * sizeof(float2);
        int planes = (int)(slab_bytes / plane_bytes);
        if (planes < 1) planes = 1;
        if (planes > nx) planes = nx;
        croft_status st = add_slab_passes(p, planes);
        if (st != CROFT_OK) return fail(p, st);
        plan_conv(p);
        *out = p;
        return CROFT_OK;
    }
    const int axes_fused[1] = {0};
    const int axes_all[3] = {2, 1, 0};
    const int* axes = fused ? axes_fused : axes_all;
    const int naxes = fused ? 1 : 3;
    for (int i = 0; i < naxes; ++i) {
        if (p->dims[axes[i]] == 1) continue;
        croft_status st = add_axis_pass(p, axes[i]);
        if (st != CROFT_OK) return fail(p, st);
    }
    plan_conv(p);
    const char* log = getenv("CROFT_LOG");
    if (log && log[0] == '1') {
        char buf[2048];
        croft_plan_describe(p, buf, sizeof(buf));
        fprintf(stderr, "croft: %s\n", buf);
    }
    *out = p;
    return CROFT_OK;
}

croft_status croft_plan_create(croft_plan* out, int nx, int ny, int nz, croft_dtype dtype) {
    return create_impl(out, nx, ny, nz, dtype, CROFT_SCHEDULE_AUTO);
}

static croft_status exec_dir(croft_plan plan, const void* in, void* out, void* stream, float isign);

}  // extern "C"

// ---------------------------------------------------------------------------
// CROFT_SCHEDULE_TUNED: measure the alternatives at plan creation, keep the fastest
// ---------------------------------------------------------------------------
// The paper tunes its implementation by hand through options 1-4 and the chunk count K
// (Sec. 5.1); here the choices a plan can make are timed on the device at creation:
//  * per axis, the pass kernel: for the column passes of 32-thread pencils (270..512 points)
//    the 16- or 8-column tile, each with the near-equal or the radix-16-first power-of-two
//    split, and the tensor-copy ring kernel; every other pass has one kernel;
//  * the schedule (the transpose fusion): three passes with the chosen kernels, z+y per L2
//    slab, or the fused yz-plane pass, as whole forward+backward transforms.
// Each candidate axis kernel is timed inside a three-pass plan by that plan's per-pass events
// (the other axes on the rules), five runs after two warm-ups, median.  The choice is cached
// on disk (CROFT_TUNE_CACHE, as for batched plans) keyed by the shape, dtype, GPU name and
// CUDA runtime version.

static std::string plan_tune_key(int nx, int ny, int nz, croft_dtype dtype) {
    int dev = 0, rt = 0;
    cudaGetDevice(&dev);
    cudaRuntimeGetVersion(&rt);
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, dev);
    char buf[512];
    snprintf(buf, sizeof(buf), "plan-v2:%dx%dx%d:%d:%s:%d", nx, ny, nz, (int)dtype, prop.name, rt);
    for (char* c = buf; *c; ++c)
        if (*c == ' ' || *c == '"') *c = '_';
    return buf;
}

static std::string plan_tune_cache_path() {
    const char* p = getenv("CROFT_TUNE_CACHE");
    if (p && *p) return p;
    const char* home = getenv("HOME");
    return std::string(home && *home ? home : "/tmp") + "/.croft_tune_cache.txt";
}

static bool plan_tune_lookup(const std::string& key, int* sched, AxisChoice* ch) {
    FILE* f = fopen(plan_tune_cache_path().c_str(), "r");
    if (!f) return false;
    char line[2048];
    bool found = false;
    while (fgets(line, sizeof(line), f)) {
        char k[900];
        int v[13];
        if (sscanf(line, "%899s %d %d %d %d %d %d %d %d %d %d %d %d %d", k, &v[0], &v[1], &v[2], &v[3], &v[4], &v[5],
                   &v[6], &v[7], &v[8], &v[9], &v[10], &v[11], &v[12]) == 14 &&
            key == k) {
            *sched = v[0];
            for (int a = 0; a < 3; ++a) {
                ch->kind[a] = v[1 + 4 * a];
                ch->w[a] = v[2 + 4 * a];
                ch->sv[a] = v[3 + 4 * a];
                ch->th[a] = v[4 + 4 * a];
            }
            found = true;  // the last matching line wins
        }
    }
    fclose(f);
    return found;
}

static void plan_tune_store(const std::string& key, int sched, const AxisChoice& ch, const std::string& info) {
    FILE* f = fopen(plan_tune_cache_path().c_str(), "a");
    if (!f) return;
    fprintf(f, "%s %d", key.c_str(), sched);
    for (int a = 0; a < 3; ++a) fprintf(f, " %d %d %d %d", ch.kind[a], ch.w[a], ch.sv[a], ch.th[a]);
    fprintf(f, " %s\n", info.c_str());
    fclose(f);
}

// Median of `reps` timings (ms) of fn() on stream s after `warm` untimed runs; < 0 on failure.
template <class F>
static double time_median(F fn, cudaStream_t s, int warm, int reps) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    std::vector<float> t;
    bool ok = true;
    for (int r = 0; r < warm + reps && ok; ++r) {
        cudaEventRecord(a, s);
        ok = fn();
        cudaEventRecord(b, s);
        if (cudaEventSynchronize(b) != cudaSuccess) ok = false;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (r >= warm) t.push_back(ms);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (!ok) {
        cudaGetLastError();
        return -1;
    }
    std::sort(t.begin(), t.end());
    return t[t.size() / 2];
}

// ms of the pass of `axis` in a three-pass plan with kernel choice ch (median of per-pass events).
static double time_axis_pass(int nx, int ny, int nz, const AxisChoice& ch, int axis, void* x, void* y, cudaStream_t s) {
    croft_plan p = nullptr;
    if (create_impl(&p, nx, ny, nz, CROFT_C2C_F32, CROFT_SCHEDULE_THREE_PASS, &ch) != CROFT_OK) {
        cudaGetLastError();
        return -1;
    }
    int idx = -1;
    for (size_t i = 0; i < p->passes.size(); ++i)
        if (p->pass_axis[i] == axis) idx = (int)i;
    std::vector<float> t;
    if (idx >= 0 && croft_plan_set_timing(p, 1) == CROFT_OK) {
        for (int r = 0; r < 7; ++r) {
            if (exec_dir(p, x, y, s, 1.0f) != CROFT_OK) break;
            float ms[8];
            const int np = croft_plan_pass_times(p, ms, 8);
            if (np <= idx) break;
            if (r >= 2) t.push_back(ms[idx]);
        }
    }
    croft_plan_destroy(p);
    if (t.size() < 5) return -1;
    std::sort(t.begin(), t.end());
    return t[t.size() / 2];
}

static croft_status create_tuned(croft_plan* out, int nx, int ny, int nz, croft_dtype dtype) {
    if (!out) return CROFT_ERR_INVALID_ARG;
    // tensor-core and complex128 plans have one kernel per pass: nothing to choose
    if (dtype != CROFT_C2C_F32) return create_impl(out, nx, ny, nz, dtype, CROFT_SCHEDULE_THREE_PASS);
    if (!axis_supported(nx) || !axis_supported(ny) || !axis_supported(nz)) return CROFT_ERR_UNSUPPORTED_SIZE;
    const std::string key = plan_tune_key(nx, ny, nz, dtype);
    int sched = CROFT_SCHEDULE_THREE_PASS;
    AxisChoice ch;
    if (plan_tune_lookup(key, &sched, &ch)) {
        croft_status st = create_impl(out, nx, ny, nz, dtype, (croft_schedule)sched, &ch);
        if (st == CROFT_OK) (*out)->tuned = "tuned (cached)";
        return st;
    }
    const long long N = (long long)nx * ny * nz;
    const size_t bytes = (size_t)N * sizeof(float2);
    void* x = nullptr;
    void* y = nullptr;
    if (dev_alloc(&x, bytes) != cudaSuccess || dev_alloc(&y, bytes) != cudaSuccess) {
        cudaGetLastError();
        dev_free(x);
        dev_free(y);
        return create_impl(out, nx, ny, nz, dtype, CROFT_SCHEDULE_AUTO);  // no room to measure: the rules
    }
    cudaStream_t s = nullptr;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    cudaMemsetAsync(x, 0, bytes, s);
    std::string info;
    char tmp[256];
    static const char* an[3] = {"x", "y", "z"};
    const int dims[3] = {nx, ny, nz};
    for (int axis = 2; axis >= 0; --axis) {
        const int n = dims[axis];
        const long long M = (axis == 2) ? 1 : (axis == 1 ? (long long)nz : (long long)ny * nz);
        if (n == 1 || M == 1 || croft_threads_per_pencil(n) != 32) continue;  // one kernel: nothing to choose
        struct Cand {
            int kind, w, sv, th;
        };
        std::vector<Cand> cands = {{-1, 0, 0, 0}};
        for (int sv = 0; sv < croft_sched_variants(n, LAYOUT_COL, 8); ++sv) {
            for (int w : {croft_col_width(n, 8), kColNarrowWidth}) cands.push_back({0, w, sv, 0});
            cands.push_back({0, croft_col_width(n, 8), sv, 16});  // 16 threads per pencil
        }
        cands.push_back({1, 16, 0, 0});
        if (n % 2 == 0) cands.push_back({2, 16, 0, 0});  // the cluster pair
        double best = 1e30;
        Cand pick = cands[0];
        for (const Cand& c : cands) {
            AxisChoice trial = ch;
            trial.kind[axis] = c.kind;
            trial.w[axis] = c.w;
            trial.sv[axis] = c.sv;
            trial.th[axis] = c.th;
            const double ms = time_axis_pass(nx, ny, nz, trial, axis, x, y, s);
            snprintf(tmp, sizeof(tmp), "%s%s:%s", info.empty() ? "" : " ", an[axis],
                     c.kind < 0 ? "rules" : (c.kind == 1 ? "ring" : (c.kind == 2 ? "pair" : (c.sv ? "r16" : "even"))));
            info += tmp;
            if (c.kind == 0) {
                snprintf(tmp, sizeof(tmp), "/w%d%s", c.w, c.th ? "/t16" : "");
                info += tmp;
            }
            snprintf(tmp, sizeof(tmp), "=%.1fus", ms < 0 ? -1.0 : ms * 1e3);
            info += tmp;
            if (ms > 0 && ms < best * 0.995) {  // a candidate must win by more than noise to replace an earlier one
                best = ms;
                pick = c;
            }
        }
        ch.kind[axis] = pick.kind;
        ch.w[axis] = pick.w;
        ch.sv[axis] = pick.sv;
        ch.th[axis] = pick.th;
    }
    // the schedule, as whole forward+backward transforms
    const croft_schedule scheds[3] = {CROFT_SCHEDULE_THREE_PASS, CROFT_SCHEDULE_SLAB_L2, CROFT_SCHEDULE_PLANE_FUSED};
    static const char* sn[3] = {"three_pass", "slab_l2", "plane_fused"};
    double best = 1e30;
    for (int k = 0; k < 3; ++k) {
        croft_plan p = nullptr;
        const croft_status st = create_impl(&p, nx, ny, nz, dtype, scheds[k], k == 0 ? &ch : nullptr);
        if (st != CROFT_OK) {
            cudaGetLastError();
            continue;
        }
        const double ms = time_median(
            [&]() { return exec_dir(p, x, y, s, 1.0f) == CROFT_OK && exec_dir(p, y, y, s, -1.0f) == CROFT_OK; }, s, 2, 5);
        croft_plan_destroy(p);
        snprintf(tmp, sizeof(tmp), " %s=%.1fus", sn[k], ms * 1e3);
        info += tmp;
        if (ms > 0 && ms < best * 0.995) {
            best = ms;
            sched = scheds[k];
        }
    }
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    dev_free(x);
    dev_free(y);
    cudaGetLastError();
    if (sched != CROFT_SCHEDULE_THREE_PASS) ch = AxisChoice();  // the other schedules run the rules' kernels
    plan_tune_store(key, sched, ch, info);
    croft_status st = create_impl(out, nx, ny, nz, dtype, (croft_schedule)sched, &ch);
    if (st == CROFT_OK) (*out)->tuned = "tuned: " + info;
    return st;
}

extern "C" {

croft_status croft_plan_create_schedule(croft_plan* out, int nx, int ny, int nz, croft_dtype dtype,
                                        croft_schedule schedule) {
    if (schedule == CROFT_SCHEDULE_TUNED) return create_tuned(out, nx, ny, nz, dtype);
    return create_impl(out, nx, ny, nz, dtype, schedule);
}

int croft_plan_describe(croft_plan plan, char* buf, int cap) {
    if (!plan) return -1;
    std::string s;
    char tmp[256];
    if (plan->batch) s = batch_describe(plan);
    else {
    snprintf(tmp, sizeof(tmp), "grid %dx%dx%d dtype %d passes %d", plan->dims[0], plan->dims[1], plan->dims[2],
             (int)plan->dtype, (int)plan->passes.size());
    s += tmp;
    static const char* an[3] = {"x", "y", "z"};
    for (size_t i = 0; i < plan->passes.size(); ++i) {
        const PassLaunch& L = plan->passes[i];
        if (L.kind == PASS_PLANE) {
            snprintf(tmp, sizeof(tmp), " | yz:plane %dx%d cluster=%d block=%d grid=%d smem=%d active_clusters=%d",
                     L.pk.ny, L.pk.nz, L.pk.cluster, L.block, L.grid, L.smem, active_clusters(L));
            s += tmp;
            continue;
        }
        snprintf(tmp, sizeof(tmp), " | %s:%s%s%s n=%d radix=", an[plan->pass_axis[i]], L.layout == LAYOUT_ROW ? "row" : "col",
                 L.tc ? (L.tc == 2 ? "+tc_fp16x3" : "+tc_bf16x3") : "", L.ring ? "+ring" : (L.pair ? "+pair" : ""),
                 L.args.n);
        s += tmp;
        CroftSched sc = L.tc ? croft_make_sched_tc(L.args.n) : croft_pass_sched_v(L.args.n, L.layout, L.f64 ? 16 : 8, L.sv);
        if (L.pair) {  // radix 2 across the pair over the half length's schedule
            sc = croft_pass_sched(L.args.n / 2, LAYOUT_COL, 8);
            s += "2|";
        }
        for (int st = 0; st < sc.count; ++st) {
            snprintf(tmp, sizeof(tmp), "%s%d", st ? "x" : "", sc.r[st]);
            s += tmp;
        }
        snprintf(tmp, sizeof(tmp), " T=%d W=%d block=%d grid=%d smem=%d", L.T, L.args.W, L.block, L.grid, L.smem);
        s += tmp;
    }
    if (plan->conv_fused) {
        const PassLaunch& L = plan->conv;
        snprintf(tmp, sizeof(tmp), " | convolve: %s fwd*G*bwd fused W=%d block=%d grid=%d smem=%d", an[plan->conv_axis],
                 L.args.W, L.block, L.grid, L.smem);
        s += tmp;
    } else {
        s += " | convolve: forward, multiply, backward";
    }
    if (!plan->tuned.empty()) s += " | " + plan->tuned;
    }
    if (buf && cap > 0) {
        size_t m = s.size() < (size_t)(cap - 1) ? s.size() : (size_t)(cap - 1);
        memcpy(buf, s.data(), m);
        buf[m] = 0;
    }
    return (int)s.size();
}

int croft_plan_tc_axes(croft_plan plan) {
    if (!plan || plan->batch) return 0;
    int m = 0;
    for (size_t i = 0; i < plan->passes.size(); ++i)
        if (plan->passes[i].tc && plan->pass_axis[i] >= 0 && plan->pass_axis[i] <= 2) m |= 1 << plan->pass_axis[i];
    return m;
}

size_t croft_plan_workspace_bytes(croft_plan plan) {
    if (!plan) return 0;
    if (plan->batch) return batch_workspace_bytes(plan);
    return stream_state_bytes(plan->stream);
}

int croft_plan_num_launches(croft_plan plan) {
    if (!plan) return -1;
    if (plan->batch) return batch_num_launches(plan);
    return plan->passes.empty() ? 0 : (int)plan->passes.size();
}

croft_status croft_plan_set_timing(croft_plan plan, int enable) {
    if (!plan) return CROFT_ERR_INVALID_ARG;
    // (a convolution records up to 2 * ngroups + 1 logical passes)
    const size_t need = (size_t)(plan->batch ? 2 : 2 * plan->ngroups + 2);
    if (enable && plan->ev.size() < need) {
        while (plan->ev.size() < need) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return CROFT_ERR_CUDA; }
            plan->ev.push_back(e);
        }
    }
    plan->timing = enable != 0;
    plan->ev_count = 0;
    return CROFT_OK;
}

int croft_plan_pass_times(croft_plan plan, float* ms, int cap) {
    if (!plan || !plan->timing || plan->ev_count < 2) return 0;
    if (cudaEventSynchronize(plan->ev[plan->ev_count - 1]) != cudaSuccess) { cudaGetLastError(); return -1; }
    int np = plan->ev_count - 1;
    for (int i = 0; i < np && i < cap; ++i) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, plan->ev[i], plan->ev[i + 1]) != cudaSuccess) { cudaGetLastError(); return -1; }
        if (ms) ms[i] = t;
    }
    return np;
}

croft_status croft_plan_last_device_status(croft_plan plan) {
    if (!plan) return CROFT_ERR_INVALID_ARG;
    if (plan->batch) return batch_last_status(plan);
    if (plan->d_status) {
        int st = 0;
        if (cudaMemcpy(&st, plan->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            return CROFT_ERR_CUDA;
        }
        return st == 0 ? CROFT_OK : (croft_status)st;
    }
    return CROFT_OK;
}

// Launches passes [i0, i1) with the given sign.  A pass marked src_in reads `in`
// unless force_out (every pass after the first logical one reads `out`).  With
// evi, records the next timing event at the end of every logical pass.  Every
// launch after the first of an exec (`started`) may use programmatic dependent
// launch: it becomes resident while the previous pass drains and waits on the
// device for that pass's results.  The first launch of an exec is ordered after
// the caller's earlier work in the ordinary way.
static croft_status run_passes(croft_plan plan, size_t i0, size_t i1, const void* in, void* out, cudaStream_t s,
                               float isign, bool force_out, int* evi, bool& started) {
    for (size_t i = i0; i < i1; ++i) {
        PassLaunch L = plan->passes[i];
        L.args.isign = isign;
        L.pargs.isign = isign;
        const size_t es = L.f64 ? sizeof(double2) : sizeof(float2);
        const char* src = ((L.src_in && !force_out) ? (const char*)in : (const char*)out) + (size_t)L.offset * es;
        char* dst = (char*)out + (size_t)L.offset * es;
        const bool pdl = plan->pdl && started;
        started = true;
        if (launch_pass(L, src, dst, s, pdl) != cudaSuccess) { cudaGetLastError(); return CROFT_ERR_CUDA; }
        const bool group_end = (i + 1 == i1) || plan->passes[i + 1].group != L.group;
        if (evi && group_end && cudaEventRecord(plan->ev[(*evi)++], s) != cudaSuccess) {
            cudaGetLastError();
            return CROFT_ERR_CUDA;
        }
    }
    return CROFT_OK;
}

static size_t elem_bytes(const croft_plan plan) { return plan->dtype == CROFT_C2C_F64 ? sizeof(double2) : sizeof(float2); }

static bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
    const char* x = (const char*)a;
    const char* y = (const char*)b;
    return x < y + nb && y < x + na;
}

static croft_status exec_dir(croft_plan plan, const void* in, void* out, void* stream, float isign) {
    if (!plan || !in || !out || plan->batch) return CROFT_ERR_INVALID_ARG;
    if (((uintptr_t)in & 15) || ((uintptr_t)out & 15)) return CROFT_ERR_INVALID_ARG;
    const long long N = (long long)plan->dims[0] * plan->dims[1] * plan->dims[2];
    const size_t bytes = (size_t)N * elem_bytes(plan);
    if (in != out && overlaps(in, bytes, out, bytes)) return CROFT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (plan->passes.empty()) {
        if (in != out && cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
            cudaGetLastError();
            return CROFT_ERR_CUDA;
        }
        plan->ev_count = 0;
        return CROFT_OK;
    }
    const bool tm = plan->timing;
    if (plan->d_status && cudaMemsetAsync(plan->d_status, 0, sizeof(int), s) != cudaSuccess) {
        cudaGetLastError();
        return CROFT_ERR_CUDA;
    }
    int evi = 0;
    if (tm) {
        if (cudaEventRecord(plan->ev[0], s) != cudaSuccess) { cudaGetLastError(); return CROFT_ERR_CUDA; }
        evi = 1;
    }
    bool started = false;
    croft_status st = run_passes(plan, 0, plan->passes.size(), in, out, s, isign, false, tm ? &evi : nullptr, started);
    if (st != CROFT_OK) return st;
    plan->ev_count = tm ? evi : 0;
    plan->ran = true;
    return CROFT_OK;
}

croft_status croft_exec_convolve(croft_plan plan, const void* in, void* out, const void* g, void* stream) {
    if (!plan || !in || !out || !g || plan->batch) return CROFT_ERR_INVALID_ARG;
    const bool f64 = plan->dtype == CROFT_C2C_F64;
    const size_t rs = f64 ? sizeof(double) : sizeof(float);
    if (((uintptr_t)in & 15) || ((uintptr_t)out & 15) || ((uintptr_t)g & (rs - 1))) return CROFT_ERR_INVALID_ARG;
    const long long N = (long long)plan->dims[0] * plan->dims[1] * plan->dims[2];
    const size_t bytes = (size_t)N * elem_bytes(plan);
    if (in != out && overlaps(in, bytes, out, bytes)) return CROFT_ERR_INVALID_ARG;
    if (overlaps(g, (size_t)N * rs, out, bytes)) return CROFT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const bool tm = plan->timing;
    if (plan->d_status && cudaMemsetAsync(plan->d_status, 0, sizeof(int), s) != cudaSuccess) {
        cudaGetLastError();
        return CROFT_ERR_CUDA;
    }
    int evi = 0;
    int* pe = tm ? &evi : nullptr;
    if (tm) {
        if (cudaEventRecord(plan->ev[0], s) != cudaSuccess) { cudaGetLastError(); return CROFT_ERR_CUDA; }
        evi = 1;
    }
    croft_status st = CROFT_OK;
    bool started = false;
    if (plan->conv_fused) {
        // forward passes but the last, the fused last-axis pass, backward passes of the other axes
        const size_t last = plan->passes.size() - 1;
        st = run_passes(plan, 0, last, in, out, s, 1.0f, false, pe, started);
        if (st != CROFT_OK) return st;
        const PassLaunch& L = plan->conv;
        if (launch_conv(L, L.src_in ? in : out, out, g, s, plan->pdl && started) != cudaSuccess) {
            cudaGetLastError();
            return CROFT_ERR_CUDA;
        }
        started = true;
        if (tm && cudaEventRecord(plan->ev[evi++], s) != cudaSuccess) { cudaGetLastError(); return CROFT_ERR_CUDA; }
        st = run_passes(plan, 0, last, in, out, s, -1.0f, true, pe, started);
        if (st != CROFT_OK) return st;
    } else {
        // F, multiply, B (a one-point grid has no passes: the multiply reads `in`)
        st = run_passes(plan, 0, plan->passes.size(), in, out, s, 1.0f, false, pe, started);
        if (st != CROFT_OK) return st;
        // (after a tensor-core pass, which does not wait on the device, the multiply is ordered normally)
        const bool pdl = plan->pdl && started && pass_supports_pdl(plan->passes.back());
        if (launch_scale(plan->passes.empty() ? in : out, out, g, N, f64, s, pdl) != cudaSuccess) {
            cudaGetLastError();
            return CROFT_ERR_CUDA;
        }
        started = true;
        if (tm && cudaEventRecord(plan->ev[evi++], s) != cudaSuccess) { cudaGetLastError(); return CROFT_ERR_CUDA; }
        st = run_passes(plan, 0, plan->passes.size(), in, out, s, -1.0f, true, pe, started);
        if (st != CROFT_OK) return st;
    }
    plan->ev_count = tm ? evi : 0;
    plan->ran = true;
    return CROFT_OK;
}

croft_status croft_exec_forward(croft_plan plan, const void* in, void* out, void* stream) {
    return exec_dir(plan, in, out, stream, 1.0f);
}

croft_status croft_exec_axes(croft_plan plan, const void* in, void* out, int axes, int direction, void* stream) {
    if (!plan || !in || !out || plan->batch || (axes & ~7) || (direction != 1 && direction != -1))
        return CROFT_ERR_INVALID_ARG;
    if (((uintptr_t)in & 15) || ((uintptr_t)out & 15)) return CROFT_ERR_INVALID_ARG;
    const long long N = (long long)plan->dims[0] * plan->dims[1] * plan->dims[2];
    const size_t bytes = (size_t)N * elem_bytes(plan);
    if (in != out && overlaps(in, bytes, out, bytes)) return CROFT_ERR_INVALID_ARG;
    // one launch per axis, over the whole grid (the three-pass schedule) - anything else cannot
    // run a subset of its axes
    for (size_t i = 0; i < plan->passes.size(); ++i)
        if (plan->passes[i].kind != PASS_AXIS || plan->passes[i].offset != 0 || plan->pass_axis[i] > 2)
            return CROFT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (plan->d_status && cudaMemsetAsync(plan->d_status, 0, sizeof(int), s) != cudaSuccess) {
        cudaGetLastError();
        return CROFT_ERR_CUDA;
    }
    const float isign = direction == -1 ? 1.0f : -1.0f;
    const bool tm = plan->timing;  // per-pass events as for exec (croft_plan_pass_times)
    int evi = 0;
    if (tm) {
        if (cudaEventRecord(plan->ev[0], s) != cudaSuccess) { cudaGetLastError(); return CROFT_ERR_CUDA; }
        evi = 1;
    }
    bool started = false, first = true;
    for (size_t i = 0; i < plan->passes.size(); ++i) {
        if (!(axes & (1 << plan->pass_axis[i]))) continue;
        PassLaunch L = plan->passes[i];
        L.args.isign = isign;
        const bool pdl = plan->pdl && started;
        started = true;
        if (launch_pass(L, first ? in : out, out, s, pdl) != cudaSuccess) {
            cudaGetLastError();
            return CROFT_ERR_CUDA;
        }
        first = false;
        if (tm && cudaEventRecord(plan->ev[evi++], s) != cudaSuccess) {
            cudaGetLastError();
            return CROFT_ERR_CUDA;
        }
    }
    // no pass ran (no selected axis longer than 1): the selected transforms are the identity
    if (first && in != out && cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
        cudaGetLastError();
        return CROFT_ERR_CUDA;
    }
    plan->ev_count = tm ? evi : 0;
    plan->ran = true;
    return CROFT_OK;
}

croft_status croft_transpose_blocks(const void* in, void* out, long long d0, long long d1, long long block_bytes,
                                    void* stream) {
    if (!in || !out || d0 < 1 || d1 < 1 || block_bytes < 1) return CROFT_ERR_INVALID_ARG;
    const size_t bytes = (size_t)d0 * (size_t)d1 * (size_t)block_bytes;
    if (overlaps(in, bytes, out, bytes)) return CROFT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const char* src = (const char*)in;
    char* dst = (char*)out;
    const size_t w = (size_t)block_bytes;
    // out[j][i] = in[i][j]: one pitched copy per index of the shorter dimension
    if (d1 <= d0) {
        for (long long j = 0; j < d1; ++j)  // column j of `in` -> row j of `out`
            if (cudaMemcpy2DAsync(dst + (size_t)j * d0 * w, w, src + (size_t)j * w, (size_t)d1 * w, w, (size_t)d0,
                                  cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
                cudaGetLastError();
                return CROFT_ERR_CUDA;
            }
    } else {
        for (long long i = 0; i < d0; ++i)  // row i of `in` -> column i of `out`
            if (cudaMemcpy2DAsync(dst + (size_t)i * w, (size_t)d0 * w, src + (size_t)i * d1 * w, w, w, (size_t)d1,
                                  cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
                cudaGetLastError();
                return CROFT_ERR_CUDA;
            }
    }
    return CROFT_OK;
}

}  // extern "C"

namespace croft {
croft_status exec_forward_impl(croft_plan plan, const void* in, void* out, void* stream) {
    return exec_dir(plan, in, out, stream, 1.0f);
}
croft_status exec_backward_impl(croft_plan plan, const void* in, void* out, void* stream) {
    return exec_dir(plan, in, out, stream, -1.0f);
}
}  // namespace croft

extern "C" {

croft_status croft_exec_backward(croft_plan plan, const void* in, void* out, void* stream) {
    return exec_dir(plan, in, out, stream, -1.0f);
}

}  // extern "C"
