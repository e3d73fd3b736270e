// C-ABI host side of seisgb: validation, padded layout, TMA tensor maps,
// launch configuration, CUDA-graph time loop (run_shot).
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/seisgb.h"
#include "aux_kernels.cuh"
#include "step_kernel.cuh"
#include "step_config.cuh"
#include "two_step.cuh"
#include "flow_step.cuh"

using namespace sgb;

// ---------------------------------------------------------------------------
// errors, counters
// ---------------------------------------------------------------------------
static thread_local std::string t_last_error;
static thread_local int64_t t_launches = 0;

static int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_last_error = buf;
    return code;
}

#define CUDA_TRY(expr)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (expr);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(e_ == cudaErrorMemoryAllocation ? SGB_ERR_OUT_OF_MEMORY           \
                                                        : SGB_ERR_CUDA,                  \
                        "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__,         \
                        __LINE__);                                                       \
    } while (0)

// Launch of a step kernel (one that calls grid_dependency_sync first). Issued
// directly on a stream, it allows programmatic stream serialisation: its CTAs
// may be placed while the previous kernel of the stream drains, so launch
// latency and CTA set-up overlap that kernel's last wave (measured 2-5% per
// step at 192^3-256^3, 2% on the adjoint's step loop). Inside a stream capture
// it is a plain launch: graph replays already launch back to back, and there
// the early CTAs cost up to 3% at 128^3.
#ifndef SGB_PDL
#define SGB_PDL 1
#endif
template <typename... KArgs, typename... Args>
cudaError_t launch_dependent(void (*kern)(KArgs...), int grid, int block, size_t smem,
                             cudaStream_t st, Args... args)
{
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed =
        SGB_PDL && cap == cudaStreamCaptureStatusNone ? 1 : 0;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

extern "C" const char *sgb_last_error(void) { return t_last_error.c_str(); }

extern "C" int64_t sgb_launch_count(int reset)
{
    int64_t v = t_launches;
    if (reset) t_launches = 0;
    return v;
}

// Host-side fault injection (a test hook, process-wide): the library's pool
// allocations are numbered from the moment the hook is armed; numbers
// [after, after + count) fail as out of memory, the others succeed.
static std::mutex g_inject_mu;
static long long g_inject_seen = 0, g_inject_after = 0, g_inject_count = 0;

// True when the armed hook says this allocation fails.
static bool injected_alloc_failure()
{
    std::lock_guard<std::mutex> lk(g_inject_mu);
    if (g_inject_count <= 0) return false;
    const long long k = g_inject_seen++;
    return k >= g_inject_after && k < g_inject_after + g_inject_count;
}

extern "C" int sgb_debug_fail_allocations(int64_t after, int64_t count)
{
    if (after < 0 || count < 0) return fail(SGB_ERR_INVALID_ARG, "after and count must be >= 0");
    std::lock_guard<std::mutex> lk(g_inject_mu);
    g_inject_seen = 0;
    g_inject_after = after;
    g_inject_count = count;
    return SGB_OK;
}

// Device error word of stencil_step (bounded-wait timeouts, non-finite
// samples), read and cleared by sgb_device_status.  run_shot, run_shot_noalloc,
// adjoint_shot, the self-test and every served shot have words of their own.
static __device__ int g_dev_err;

// ---------------------------------------------------------------------------
// per-device state
// ---------------------------------------------------------------------------
namespace {



struct DevState {
    bool ready = false;
    int sms = 0;
    int occ = 0;     // resident CTAs of the fp32 step kernel per SM
    int occ_h = 0;   // ... fp16 storage
    int occ_b = 0;   // ... bf16 storage
    int occ_df = 0;  // ... difference form, fp32 storage
    int occ_db = 0;  // ... difference form, bf16 storage
    int occ_dh = 0;  // ... difference form, fp16 storage (scaled)
    int *err = nullptr;
    cudaMemPool_t pool = nullptr;
};

std::mutex g_mu;
DevState g_dev[64];
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

// Allow the step kernel for storage T its dynamic shared memory; report how
// many of its CTAs fit on one SM.
template <class T, bool DIFF = false>
auto step_kernel_of()
{
    if constexpr (DIFF) return diff_step_kernel<Cfg, T>;
    else return fused_step_kernel<Cfg, T>;
}

template <class T, bool DIFF = false>
int prepare_step_kernel(int *occ)
{
    using G = Stage<Cfg, T>;
    const auto kern = step_kernel_of<T, DIFF>();
    CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)G::SMEM_BYTES));
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, kern, Cfg::BLOCK, G::SMEM_BYTES));
    if (*occ < 1) return fail(SGB_ERR_CUDA, "step kernel does not fit on an SM");
    return SGB_OK;
}

int device_state(DevState **out)
{
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(SGB_ERR_CUDA, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    DevState &s = g_dev[dev];
    if (!s.ready) {
        CUDA_TRY(cudaDeviceGetAttribute(&s.sms, cudaDevAttrMultiProcessorCount, dev));
        int rc0;
        if ((rc0 = prepare_step_kernel<float>(&s.occ))) return rc0;
        if ((rc0 = prepare_step_kernel<__half>(&s.occ_h))) return rc0;
        if ((rc0 = prepare_step_kernel<__nv_bfloat16>(&s.occ_b))) return rc0;
        if ((rc0 = prepare_step_kernel<float, true>(&s.occ_df))) return rc0;
        if ((rc0 = prepare_step_kernel<__nv_bfloat16, true>(&s.occ_db))) return rc0;
        if ((rc0 = prepare_step_kernel<__half, true>(&s.occ_dh))) return rc0;
        CUDA_TRY(cudaGetSymbolAddress((void **)&s.err, g_dev_err));
        cudaMemPoolProps props;
        memset(&props, 0, sizeof props);
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        CUDA_TRY(cudaMemPoolCreate(&s.pool, &props));
        uint64_t thr = UINT64_MAX;
        CUDA_TRY(cudaMemPoolSetAttribute(s.pool, cudaMemPoolAttrReleaseThreshold, &thr));
        if (!g_encode) {
            cudaDriverEntryPointQueryResult q;
            void *fn = nullptr;
            CUDA_TRY(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                      cudaEnableDefault, &q));
            if (q != cudaDriverEntryPointSuccess || !fn)
                return fail(SGB_ERR_CUDA, "cuTensorMapEncodeTiled not available");
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        }
        s.ready = true;
    }
    *out = &s;
    return SGB_OK;
}

// ---------------------------------------------------------------------------
// layout and validation
// ---------------------------------------------------------------------------
void compute_layout(const sgb_grid *g, sgb_layout_info *L)
{
    L->Nx = g->nx + 2 * g->nb;
    L->Ny = g->ny + 2 * g->nb;
    L->Nz = g->nz + 2 * g->nb;
    L->halo_lo_x = HALO_LO_X;
    L->halo = HALO;
    L->sx = ((int64_t)HALO_LO_X + L->Nx + HALO + 31) / 32 * 32;
    L->sy = (int64_t)L->Ny + 2 * HALO;
    L->sz = (int64_t)L->Nz + 2 * HALO;
    L->stride_y = L->sx;
    L->stride_z = L->sx * L->sy;
    L->origin = (int64_t)HALO * L->stride_z + (int64_t)HALO * L->sx + HALO_LO_X;
    L->elems = L->sx * L->sy * L->sz;
}

bool finite_pos(float v) { return std::isfinite(v) && v > 0.0f; }

int check_grid(const sgb_grid *g, sgb_layout_info *L)
{
    if (!g) return fail(SGB_ERR_INVALID_ARG, "grid is NULL");
    if (g->nx < 1 || g->ny < 1 || g->nz < 1)
        return fail(SGB_ERR_INVALID_ARG, "inner extents must be >= 1 (got %d %d %d)", g->nx,
                    g->ny, g->nz);
    if (g->nb < 0) return fail(SGB_ERR_INVALID_ARG, "PML width must be >= 0 (got %d)", g->nb);
    const int64_t lim = 1 << 20;
    if ((int64_t)g->nx + 2 * g->nb > lim || (int64_t)g->ny + 2 * g->nb > lim ||
        (int64_t)g->nz + 2 * g->nb > lim)
        return fail(SGB_ERR_INVALID_ARG, "computed extent above 2^20 points");
    if (!finite_pos(g->dx) || !finite_pos(g->dy) || !finite_pos(g->dz))
        return fail(SGB_ERR_INVALID_ARG, "spacing must be finite and > 0");
    if (!finite_pos(g->dt)) return fail(SGB_ERR_INVALID_ARG, "dt must be finite and > 0");
    if (!finite_pos(g->vmax)) return fail(SGB_ERR_INVALID_ARG, "vmax must be finite and > 0");
    if (!(g->pml_r0 > 0.0f && g->pml_r0 <= 1.0f))
        return fail(SGB_ERR_INVALID_ARG, "pml_r0 must be in (0, 1] (got %g)", (double)g->pml_r0);
    if (g->storage < SGB_FP32 || g->storage > SGB_FP16_DIFF)
        return fail(SGB_ERR_INVALID_ARG, "unknown storage format %d", g->storage);
    if (g->schedule < SGB_SCHED_AUTO || g->schedule > SGB_SCHED_FLOW)
        return fail(SGB_ERR_INVALID_ARG, "unknown schedule %d", g->schedule);
    if (g->schedule == SGB_SCHED_PAIRS && g->storage != SGB_FP32)
        return fail(SGB_ERR_INVALID_ARG, "SGB_SCHED_PAIRS needs SGB_FP32 storage");
    if (g->schedule == SGB_SCHED_FLOW && g->storage != SGB_FP32 && g->storage != SGB_BF16)
        return fail(SGB_ERR_INVALID_ARG, "SGB_SCHED_FLOW needs SGB_FP32 or SGB_BF16 storage");
    compute_layout(g, L);
    if (L->elems > (int64_t(1) << 40)) return fail(SGB_ERR_INVALID_ARG, "field too large");
    return SGB_OK;
}

// 8th-order central second-derivative weights (standard table).
const double W8[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0};
// Peak of the 1D symbol -(w0 + 2 sum w_m cos(m theta)), reached at theta = pi.
const double SYMBOL_MAX = 2048.0 / 315.0;

double cfl_limit(const sgb_grid *g, double vmax)
{
    const double s = 1.0 / ((double)g->dx * g->dx) + 1.0 / ((double)g->dy * g->dy) +
                     1.0 / ((double)g->dz * g->dz);
    return 2.0 / (vmax * std::sqrt(SYMBOL_MAX * s));
}

bool in_inner(const sgb_grid *g, int i, int j, int k)
{
    return i >= g->nb && i < g->nb + g->nx && j >= g->nb && j < g->nb + g->ny && k >= g->nb &&
           k < g->nb + g->nz;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Fill the parts of StepArgs that depend on the grid only.
void fill_step_constants(const sgb_grid *g, const sgb_layout_info &L, StepArgs &a)
{
    memset(&a, 0, sizeof a);
    a.Nx = L.Nx;
    a.Ny = L.Ny;
    a.Nz = L.Nz;
    a.nb = g->nb;
    a.nx = g->nx;
    a.ny = g->ny;
    a.nz = g->nz;
    a.sx = L.sx;
    a.sxy = L.stride_z;
    a.origin = L.origin;
    const double ix = 1.0 / ((double)g->dx * g->dx), iy = 1.0 / ((double)g->dy * g->dy),
                 iz = 1.0 / ((double)g->dz * g->dz);
    a.c0 = (float)(W8[0] * (ix + iy + iz));
    for (int m = 1; m <= 4; ++m) {
        a.cx[m - 1] = (float)(W8[m] * ix);
        a.cy[m - 1] = (float)(W8[m] * iy);
        a.cz[m - 1] = (float)(W8[m] * iz);
    }
    // PML profile eta_a = eta_max_a (d / nb)^2, eta_max_a = -3 vmax ln r0 / (2 nb h_a)
    if (g->nb > 0 && g->pml_r0 < 1.0f) {
        const double nb = g->nb, dt = g->dt, lr = std::log((double)g->pml_r0);
        const double h[3] = {g->dx, g->dy, g->dz};
        double aa[3], kk[3];
        for (int q = 0; q < 3; ++q) {
            const double emax = -3.0 * (double)g->vmax * lr / (2.0 * nb * h[q]);
            aa[q] = emax * dt / (nb * nb);
            kk[q] = dt * emax / (4.0 * nb * nb * h[q] * h[q]);
        }
        a.ax = (float)aa[0];
        a.ay = (float)aa[1];
        a.az = (float)aa[2];
        a.kx = (float)kk[0];
        a.ky = (float)kk[1];
        a.kz = (float)kk[2];
    }
    a.si = a.sj = a.sk = -1;
    a.inv_vol = (float)(1.0 / ((double)g->dx * g->dy * g->dz));
}

template <class T>
struct TmaType;
template <>
struct TmaType<float> {
    static constexpr CUtensorMapDataType v = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
};
template <>
struct TmaType<__half> {
    static constexpr CUtensorMapDataType v = CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
};
template <>
struct TmaType<__nv_bfloat16> {
    static constexpr CUtensorMapDataType v = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
};

// 3D tiled map over the computed region of a padded field of element type T.
template <class T>
int encode_map(CUtensorMap *map, const void *padded, const sgb_layout_info &L, int box_x, int box_y,
               CUtensorMapL2promotion promo = SGB_L2PROMO_P)
{
    const size_t es = sizeof(T);
    void *base = const_cast<char *>(static_cast<const char *>(padded)) + L.origin * es;
    cuuint64_t dims[3] = {(cuuint64_t)L.Nx, (cuuint64_t)L.Ny, (cuuint64_t)L.Nz};
    cuuint64_t strides[2] = {(cuuint64_t)(L.sx * es), (cuuint64_t)(L.stride_z * es)};
    cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = g_encode(map, TmaType<T>::v, 3, base, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          promo, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(SGB_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return SGB_OK;
}

struct StepMaps {
    CUtensorMap ucur, ucur_in, uprev, m, phi;
};

template <class T>
int encode_step_maps(StepMaps &mp, const void *u_cur, const void *u_prev, const float *m,
                     const float *phi, const sgb_layout_info &L)
{
    using G = Stage<Cfg, T>;
    int rc;
    if ((rc = encode_map<T>(&mp.ucur, u_cur, L, G::SW, Cfg::SH, SGB_L2PROMO))) return rc;
    if ((rc = encode_map<T>(&mp.ucur_in, u_cur, L, Cfg::BX, Cfg::BY))) return rc;
    if ((rc = encode_map<T>(&mp.uprev, u_prev, L, Cfg::BX, Cfg::BY))) return rc;
    if ((rc = encode_map<float>(&mp.m, m, L, Cfg::BX, Cfg::BY))) return rc;
    if ((rc = encode_map<float>(&mp.phi, phi ? phi : m, L, Cfg::PHI_BW, Cfg::BY))) return rc;
    return SGB_OK;
}

template <class T, bool DIFF = false>
int launch_step(const StepArgs &a, const StepMaps &mp, int grid, cudaStream_t st)
{
    CUDA_TRY(launch_dependent(step_kernel_of<T, DIFF>(), grid, Cfg::BLOCK, Stage<Cfg, T>::SMEM_BYTES,
                              st, a, mp.ucur, mp.ucur_in, mp.uprev, mp.m, mp.phi));
    ++t_launches;
    return SGB_OK;
}

PadGeom pad_geom(const sgb_layout_info &L)
{
    PadGeom pg;
    pg.Nx = L.Nx;
    pg.Ny = L.Ny;
    pg.Nz = L.Nz;
    pg.sx = L.sx;
    pg.sxy = L.stride_z;
    pg.origin = L.origin;
    return pg;
}

int ew_grid(long long n, const DevState &ds)
{
    long long b = (n + 255) / 256;
    long long cap = (long long)ds.sms * 8;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Stream-ordered scratch from the library pool, released in reverse order.
struct Scratch {
    cudaStream_t st;
    cudaMemPool_t pool;
    std::vector<void *> ptrs;
    ~Scratch()
    {
        for (auto it = ptrs.rbegin(); it != ptrs.rend(); ++it) cudaFreeAsync(*it, st);
    }
    int get(void **p, size_t bytes)
    {
        if (injected_alloc_failure())
            return fail(SGB_ERR_OUT_OF_MEMORY, "scratch allocation of %zu bytes failed (injected)", bytes);
        cudaError_t e = cudaMallocFromPoolAsync(p, bytes ? bytes : 16, pool, st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(e == cudaErrorMemoryAllocation ? SGB_ERR_OUT_OF_MEMORY : SGB_ERR_CUDA,
                        "scratch allocation of %zu bytes failed: %s", bytes,
                        cudaGetErrorString(e));
        }
        ptrs.push_back(*p);
        return SGB_OK;
    }
};

// out = err, err = 0 in one atomic step: a bit set by a kernel on another
// stream between a read and a separate clear would otherwise be lost.
__global__ void take_err_kernel(int *err, int *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *out = atomicExch(err, 0);
}

// Read and clear the error word `err` (stream-ordered, then waits for st).
int read_and_clear_dev_err(int *err, const DevState &ds, cudaStream_t st, int *val)
{
    Scratch sc{st, ds.pool, {}};
    int *d_out = nullptr;
    int rc = sc.get((void **)&d_out, sizeof(int));
    if (rc) return rc;
    take_err_kernel<<<1, 32, 0, st>>>(err, d_out);
    CUDA_TRY(cudaGetLastError());
    ++t_launches;
    CUDA_TRY(cudaMemcpyAsync(val, d_out, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return SGB_OK;
}

// Map the bits of an error word to the status a call returns.
int dev_err_status(int v)
{
    if (v & DEV_ERR_TIMEOUT) return fail(SGB_ERR_TIMEOUT, "a kernel wait timed out");
    if (v & DEV_ERR_NONFINITE) return fail(SGB_ERR_NONFINITE, "a receiver sampled NaN/Inf");
    if (v) return fail(SGB_ERR_CUDA, "device error word %d", v);
    return SGB_OK;
}

// A byte range of a caller buffer (host or device: one address space).
struct Span {
    const void *p;
    size_t bytes;
    const char *name;
};

bool spans_overlap(const Span &a, const Span &b)
{
    if (!a.p || !b.p || !a.bytes || !b.bytes) return false;
    const uintptr_t a0 = (uintptr_t)a.p, b0 = (uintptr_t)b.p;
    return a0 < b0 + b.bytes && b0 < a0 + a.bytes;
}

// Outputs may overlap neither an input nor each other.
int check_no_overlap(const Span *outs, int nout, const Span *ins, int nin)
{
    for (int o = 0; o < nout; ++o) {
        for (int i = 0; i < nin; ++i)
            if (spans_overlap(outs[o], ins[i]))
                return fail(SGB_ERR_INVALID_ARG, "%s overlaps %s", outs[o].name, ins[i].name);
        for (int q = o + 1; q < nout; ++q)
            if (spans_overlap(outs[o], outs[q]))
                return fail(SGB_ERR_INVALID_ARG, "%s overlaps %s", outs[o].name, outs[q].name);
    }
    return SGB_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// public entry points
// ---------------------------------------------------------------------------
extern "C" int sgb_layout(const sgb_grid *g, sgb_layout_info *out)
{
    sgb_layout_info L;
    int rc = check_grid(g, &L);
    if (rc) return rc;
    if (!out) return fail(SGB_ERR_INVALID_ARG, "out is NULL");
    *out = L;
    return SGB_OK;
}

extern "C" int sgb_cfl_dt(const sgb_grid *g, float vmax, float *dt_max)
{
    if (!g || !dt_max) return fail(SGB_ERR_INVALID_ARG, "NULL argument");
    if (!finite_pos(vmax)) return fail(SGB_ERR_INVALID_ARG, "vmax must be finite and > 0");
    if (!finite_pos(g->dx) || !finite_pos(g->dy) || !finite_pos(g->dz))
        return fail(SGB_ERR_INVALID_ARG, "spacing must be finite and > 0");
    *dt_max = (float)cfl_limit(g, vmax);
    return SGB_OK;
}

extern "C" int sgb_pack(const sgb_grid *g, const float *compact, float *padded, void *stream)
{
    sgb_layout_info L;
    int rc = check_grid(g, &L);
    if (rc) return rc;
    if (!compact || !padded) return fail(SGB_ERR_INVALID_ARG, "NULL pointer");
    DevState *ds;
    if ((rc = device_state(&ds))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    pack_kernel<<<ew_grid(L.elems, *ds), 256, 0, st>>>(pad_geom(L), compact, padded, L.elems);
    CUDA_TRY(cudaGetLastError());
    ++t_launches;
    return SGB_OK;
}

extern "C" int sgb_unpack(const sgb_grid *g, const float *padded, float *compact, void *stream)
{
    sgb_layout_info L;
    int rc = check_grid(g, &L);
    if (rc) return rc;
    if (!compact || !padded) return fail(SGB_ERR_INVALID_ARG, "NULL pointer");
    DevState *ds;
    if ((rc = device_state(&ds))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    unpack_kernel<<<ew_grid((long long)L.Nx * L.Ny * L.Nz, *ds), 256, 0, st>>>(pad_geom(L), padded,
                                                                               compact);
    CUDA_TRY(cudaGetLastError());
    ++t_launches;
    return SGB_OK;
}

namespace {

// A bounded wait on an mbarrier that nothing completes, exactly as a step
// kernel waits for its copies: after limit_ns it gives up and sets the timeout
// bit of the device error word.
__global__ void wait_timeout_probe_kernel(int *err, unsigned long long limit_ns)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0, limit_ns)) atomicOr(err, DEV_ERR_TIMEOUT);
}

}  // namespace

extern "C" int sgb_selftest_wait_timeout(int32_t limit_us, int32_t *status_out, void *stream)
{
    if (!status_out) return fail(SGB_ERR_INVALID_ARG, "status_out is NULL");
    if (limit_us < 1 || limit_us > 2000000)
        return fail(SGB_ERR_INVALID_ARG, "limit_us must be in 1..2000000 (got %d)", limit_us);
    DevState *ds;
    int rc = device_state(&ds);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Scratch sc{st, ds->pool, {}};
    int *d_err = nullptr;  // this call's own error word
    if ((rc = sc.get((void **)&d_err, sizeof(int)))) return rc;
    CUDA_TRY(cudaMemsetAsync(d_err, 0, sizeof(int), st));
    wait_timeout_probe_kernel<<<1, 32, 0, st>>>(d_err, (unsigned long long)limit_us * 1000ull);
    CUDA_TRY(cudaGetLastError());
    ++t_launches;
    int v = 0;
    CUDA_TRY(cudaMemcpyAsync(&v, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    *status_out = (v & DEV_ERR_TIMEOUT) ? SGB_ERR_TIMEOUT : v ? SGB_ERR_CUDA : SGB_OK;
    return SGB_OK;
}

extern "C" int sgb_pool_used_bytes(int64_t *bytes)
{
    if (!bytes) return fail(SGB_ERR_INVALID_ARG, "bytes is NULL");
    DevState *ds;
    int rc = device_state(&ds);
    if (rc) return rc;
    cuuint64_t v = 0;
    CUDA_TRY(cudaMemPoolGetAttribute(ds->pool, cudaMemPoolAttrUsedMemCurrent, &v));
    *bytes = (int64_t)v;
    return SGB_OK;
}

extern "C" int sgb_device_status(void *stream)
{
    DevState *ds;
    int rc = device_state(&ds);
    if (rc) return rc;
    int v = 0;
    if ((rc = read_and_clear_dev_err(ds->err, *ds, (cudaStream_t)stream, &v))) return rc;
    return dev_err_status(v);
}

namespace {

// One step of storage type T on caller-owned fields (stencil_step,
// stencil_step_scaled and stencil_step_diff after their argument checks). DIFF:
// the difference form, d_io holding d^n on entry and d^{n+1} on exit.
template <class T, bool DIFF = false>
int stencil_step_t(const sgb_grid *g, const sgb_layout_info &L, DevState *ds, cudaStream_t st,
                   const void *u_cur, void *u_out, void *d_io, const float *m, float *phi,
                   ScaleState *scale, int32_t step, const sgb_source *src, const sgb_receivers *rec)
{
    int rc;
    StepArgs a;
    fill_step_constants(g, L, a);
    a.u_out = u_out;
    a.u_cur = u_cur;
    a.d_io = d_io;
    a.phi = phi;
    a.err = ds->err;
    a.step_add = step;
    a.scale = scale;
    if (src) {
        a.si = src->i;
        a.sj = src->j;
        a.sk = src->k;
        a.wavelet = src->wavelet;
        a.m_src = m + L.origin + (long long)src->k * L.stride_z + (long long)src->j * L.sx + src->i;
    }
    const int occ = DIFF ? (std::is_same<T, float>::value ? ds->occ_df : ds->occ_db)
                    : std::is_same<T, float>::value ? ds->occ
                    : std::is_same<T, __half>::value ? ds->occ_h : ds->occ_b;
    int grid = 0;
    choose_decomposition(L.Nx, L.Ny, L.Nz, ds->sms, occ, a, &grid);
    StepMaps mp;
    if ((rc = encode_step_maps<T>(mp, a.u_cur, DIFF ? d_io : a.u_out, m, phi, L))) return rc;
    if ((rc = launch_step<T, DIFF>(a, mp, grid, st))) return rc;
    if (rec && rec->nrec > 0) {
        std::vector<long long> off(rec->nrec);
        for (int r = 0; r < rec->nrec; ++r)
            off[r] = L.origin + (long long)rec->ijk[3 * r + 2] * L.stride_z +
                     (long long)rec->ijk[3 * r + 1] * L.sx + rec->ijk[3 * r];
        void *d_off = nullptr;
        Scratch sc{st, ds->pool, {}};
        if ((rc = sc.get(&d_off, off.size() * sizeof(long long)))) return rc;
        CUDA_TRY(cudaMemcpyAsync(d_off, off.data(), off.size() * sizeof(long long),
                                 cudaMemcpyHostToDevice, st));
        // u^{n+1} times its scale (fp16: s[(step + 1) & 3], written by the step)
        gather_t_kernel<T><<<(rec->nrec + 255) / 256, 256, 0, st>>>(
            static_cast<const T *>(u_out), static_cast<const long long *>(d_off), rec->nrec,
            scale ? &scale->s[(step + 1) & 3] : nullptr, rec->traces, ds->err);
        CUDA_TRY(cudaGetLastError());
        ++t_launches;
        // the pageable copy above is staged before cudaMemcpyAsync returns; the
        // scratch is released stream-ordered after the gather
    }
    return SGB_OK;
}

int stencil_step_common(const sgb_grid *g, const void *u_cur, void *u_prev_to_next, void *d_io,
                        const float *m, float *phi, float *scale, int32_t step,
                        const sgb_source *src, const sgb_receivers *rec, void *stream)
{
    sgb_layout_info L;
    int rc = check_grid(g, &L);
    if (rc) return rc;
    const bool diff = g->storage == SGB_FP32_DIFF || g->storage == SGB_BF16_DIFF ||
                      g->storage == SGB_FP16_DIFF;
    if (g->storage == SGB_FP16_DIFF)
        return fail(SGB_ERR_INVALID_ARG,
                    "stencil_step: SGB_FP16_DIFF keeps scale states for u and d (run_shot only)");
    if (diff && !d_io)
        return fail(SGB_ERR_INVALID_ARG,
                    "stencil_step: the difference-form storage keeps a third field; use "
                    "stencil_step_diff");
    if (!diff && d_io)
        return fail(SGB_ERR_INVALID_ARG,
                    "stencil_step_diff: storage must be SGB_FP32_DIFF or SGB_BF16_DIFF");
    if (d_io && (!aligned16(d_io) || d_io == u_cur || d_io == u_prev_to_next))
        return fail(SGB_ERR_INVALID_ARG, "d must be 16-byte aligned and distinct from u_cur, u_next");
    if (!u_cur || !u_prev_to_next || !m) return fail(SGB_ERR_INVALID_ARG, "NULL field pointer");
    if (g->nb > 0 && !phi) return fail(SGB_ERR_INVALID_ARG, "phi is required when nb > 0");
    if (!aligned16(u_cur) || !aligned16(u_prev_to_next) || !aligned16(m) || (phi && !aligned16(phi)) ||
        (scale && !aligned16(scale)))
        return fail(SGB_ERR_INVALID_ARG, "field pointers must be 16-byte aligned");
    if (u_cur == u_prev_to_next) return fail(SGB_ERR_INVALID_ARG, "u_cur aliases u_prev_to_next");
    if (step < 0) return fail(SGB_ERR_INVALID_ARG, "step must be >= 0");
    if (src) {
        if (!in_inner(g, src->i, src->j, src->k))
            return fail(SGB_ERR_INVALID_ARG, "source (%d,%d,%d) outside the inner region", src->i,
                        src->j, src->k);
        if (!src->wavelet) return fail(SGB_ERR_INVALID_ARG, "source wavelet is NULL");
    }
    if (rec && rec->nrec > 0) {
        if (!rec->ijk || !rec->traces) return fail(SGB_ERR_INVALID_ARG, "receiver arrays NULL");
        for (int r = 0; r < rec->nrec; ++r)
            if (!in_inner(g, rec->ijk[3 * r], rec->ijk[3 * r + 1], rec->ijk[3 * r + 2]))
                return fail(SGB_ERR_INVALID_ARG, "receiver %d outside the inner region", r);
    }
    if (rec && rec->nrec < 0) return fail(SGB_ERR_INVALID_ARG, "nrec < 0");
    if ((double)g->dt > cfl_limit(g, g->vmax))
        return fail(SGB_ERR_UNSTABLE_DT, "dt %g above the CFL limit %g for vmax %g", (double)g->dt,
                    cfl_limit(g, g->vmax), (double)g->vmax);
    DevState *ds;
    if ((rc = device_state(&ds))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    ScaleState *ss = reinterpret_cast<ScaleState *>(scale);
    switch (g->storage) {
    case SGB_FP16_SCALED:
        return stencil_step_t<__half>(g, L, ds, st, u_cur, u_prev_to_next, nullptr, m, phi, ss, step,
                                      src, rec);
    case SGB_BF16:
        return stencil_step_t<__nv_bfloat16>(g, L, ds, st, u_cur, u_prev_to_next, nullptr, m, phi,
                                             nullptr, step, src, rec);
    case SGB_FP32_DIFF:
        return stencil_step_t<float, true>(g, L, ds, st, u_cur, u_prev_to_next, d_io, m, phi,
                                           nullptr, step, src, rec);
    case SGB_BF16_DIFF:
        return stencil_step_t<__nv_bfloat16, true>(g, L, ds, st, u_cur, u_prev_to_next, d_io, m,
                                                   phi, nullptr, step, src, rec);
    default:
        return stencil_step_t<float>(g, L, ds, st, u_cur, u_prev_to_next, nullptr, m, phi, nullptr,
                                     step, src, rec);
    }
}

}  // namespace

extern "C" int stencil_step(const sgb_grid *g, const void *u_cur, void *u_prev_to_next,
                            const float *m, float *phi, int32_t step, const sgb_source *src,
                            const sgb_receivers *rec, void *stream)
{
    if (g && g->storage == SGB_FP16_SCALED)
        return fail(SGB_ERR_INVALID_ARG,
                    "stencil_step: SGB_FP16_SCALED fields carry a scale state; use stencil_step_scaled");
    return stencil_step_common(g, u_cur, u_prev_to_next, nullptr, m, phi, nullptr, step, src, rec,
                               stream);
}

extern "C" int stencil_step_diff(const sgb_grid *g, const void *u_cur, void *u_next, void *d,
                                 const float *m, float *phi, int32_t step, const sgb_source *src,
                                 const sgb_receivers *rec, void *stream)
{
    if (!d) return fail(SGB_ERR_INVALID_ARG, "stencil_step_diff: d is NULL");
    return stencil_step_common(g, u_cur, u_next, d, m, phi, nullptr, step, src, rec, stream);
}

extern "C" int stencil_step_scaled(const sgb_grid *g, const void *u_cur, void *u_prev_to_next,
                                   const float *m, float *phi, float *scale_state, int32_t step,
                                   const sgb_source *src, const sgb_receivers *rec, void *stream)
{
    if (!g || g->storage != SGB_FP16_SCALED)
        return fail(SGB_ERR_INVALID_ARG, "stencil_step_scaled: storage must be SGB_FP16_SCALED");
    if (!scale_state) return fail(SGB_ERR_INVALID_ARG, "stencil_step_scaled: scale_state is NULL");
    return stencil_step_common(g, u_cur, u_prev_to_next, nullptr, m, phi, scale_state, step, src,
                               rec, stream);
}

namespace {

// ---------------------------------------------------------------------------
// Temporally blocked pairs of steps (SGB_SCHED_PAIRS, stencil_step2)
// ---------------------------------------------------------------------------
using TCfg = TwoCfg<56, 16, 8, 8, 6>;

// Work of one pair (steps n, n+1): the two-step kernel on the box B (the inner
// region shrunk by the stencil radius, x bounds on multiples of 4) and two
// single-step shell launches on the standard tiles that reach outside B.
struct PairPlan {
    bool box = false;
    int bx0 = 0, bx1 = 0, by0 = 0, by1 = 0, bz0 = 0, bz1 = 0;
    int tiles_x = 0, tiles_y = 0, zc = 0, grid = 0;
    std::vector<int4> shell;
};

int two_step_prepared = 0;

int prepare_two_step()
{
    if (two_step_prepared) return SGB_OK;
    std::lock_guard<std::mutex> lk(g_mu);
    CUDA_TRY(cudaFuncSetAttribute(two_step_kernel<TCfg>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)TCfg::SMEM_BYTES));
    CUDA_TRY(cudaFuncSetAttribute(shell_step_kernel<Cfg>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)Stage<Cfg, float>::SMEM_BYTES));
    two_step_prepared = 1;
    return SGB_OK;
}

void plan_pair(const sgb_grid *g, const sgb_layout_info &L, const DevState &ds, PairPlan &pp)
{
    const int nb = g->nb;
    pp.bx0 = (nb + R + 3) / 4 * 4;
    pp.bx1 = (nb + g->nx - R) / 4 * 4;
    pp.by0 = nb + R;
    pp.by1 = nb + g->ny - R;
    pp.bz0 = nb + R;
    pp.bz1 = nb + g->nz - R;
    pp.box = pp.bx1 > pp.bx0 && pp.by1 > pp.by0 && pp.bz1 > pp.bz0;
    if (!pp.box) pp.bx0 = pp.bx1 = pp.by0 = pp.by1 = pp.bz0 = pp.bz1 = 0;
    if (pp.box) {
        pp.tiles_x = (pp.bx1 - pp.bx0 + TCfg::BX - 1) / TCfg::BX;
        pp.tiles_y = (pp.by1 - pp.by0 + TCfg::BY - 1) / TCfg::BY;
        // z-chunks: fewest waves x (chunk + the 8 planes of step-1 overhead),
        // chunks of at most 64 planes (neighbouring CTAs stay close in z)
        const int nzb = pp.bz1 - pp.bz0;
        const long long tiles = (long long)pp.tiles_x * pp.tiles_y, slots = ds.sms;
        double best = 1e300;
        pp.zc = nzb;
        for (int c = 1; c <= nzb; ++c) {
            const int zc = (nzb + c - 1) / c;
            if (zc > 64) continue;
            const long long units = tiles * ((nzb + zc - 1) / zc);
            const double cost = (double)((units + slots - 1) / slots) * (zc + 2 * R);
            if (cost < best * 0.999) {
                best = cost;
                pp.zc = zc;
            }
            if (zc <= 8) break;
        }
        pp.grid = (int)(tiles * ((nzb + pp.zc - 1) / pp.zc));
    }
    // shell: standard tiles; those inside B's x-y extent only need the z ranges
    // outside it; units sorted by z so that CTAs running together share planes
    pp.shell.clear();
    const int zs = 32;
    for (int y = 0; y < L.Ny; y += Cfg::BY)
        for (int x = 0; x < L.Nx; x += Cfg::BX) {
            const int xe = std::min(x + Cfg::BX, L.Nx), ye = std::min(y + Cfg::BY, L.Ny);
            const bool inside = pp.box && x >= pp.bx0 && xe <= pp.bx1 && y >= pp.by0 && ye <= pp.by1;
            int ranges[2][2] = {{0, inside ? pp.bz0 : L.Nz}, {inside ? pp.bz1 : L.Nz, L.Nz}};
            for (auto &r : ranges) {
                const int len = r[1] - r[0];
                if (len <= 0) continue;
                const int nch = (len + zs - 1) / zs, zc = (len + nch - 1) / nch;
                for (int z = r[0]; z < r[1]; z += zc) pp.shell.push_back(make_int4(x, y, z, std::min(z + zc, r[1])));
            }
        }
    std::stable_sort(pp.shell.begin(), pp.shell.end(), [](const int4 &a, const int4 &b) {
        return a.z != b.z ? a.z < b.z : (a.y != b.y ? a.y < b.y : a.x < b.x);
    });
}

// Tensor maps of one pair: (u^{n-1}, u^n) -> (u^{n+1}, u^{n+2}).
struct PairMaps {
    CUtensorMap two_u, two_up, two_m;  // the two-step kernel's u^n box, u^{n-1} and m tiles
    StepMaps shell0, shell1;           // shell launches of steps n and n+1
};

int encode_pair_maps(PairMaps &pm, const float *a_prev, const float *b_cur, const float *c_next,
                     const float *m, const float *phi, const sgb_layout_info &L)
{
    int rc;
    if ((rc = encode_map<float>(&pm.two_u, b_cur, L, TCfg::UW, TCfg::UH, SGB_L2PROMO))) return rc;
    if ((rc = encode_map<float>(&pm.two_up, a_prev, L, TCfg::EX, TCfg::EY))) return rc;
    if ((rc = encode_map<float>(&pm.two_m, m, L, TCfg::EX, TCfg::EY))) return rc;
    if ((rc = encode_step_maps<float>(pm.shell0, b_cur, a_prev, m, phi, L))) return rc;
    if ((rc = encode_step_maps<float>(pm.shell1, c_next, b_cur, m, phi, L))) return rc;
    return SGB_OK;
}

// Enqueue the three launches of one pair.  base: the step constants with phi,
// error word, source, receivers (sampled by the shell launches from their
// u^n, rows n-1 and n).  Steps n = *step_ptr + step_add and n + 1.
int launch_pair(const sgb_grid *g, const PairPlan &pp, const PairMaps &pm, const int4 *d_units,
                const StepArgs &base, float *c_next, float *d_next2, const float *b_cur,
                const int *step_ptr, int step_add, cudaStream_t st)
{
    if (pp.box) {
        TwoStepArgs t;
        memset(&t, 0, sizeof t);
        t.out1 = c_next;
        t.out2 = d_next2;
        t.Nx = base.Nx;
        t.Ny = base.Ny;
        t.Nz = base.Nz;
        t.sx = base.sx;
        t.sxy = base.sxy;
        t.origin = base.origin;
        t.c0 = base.c0;
        for (int q = 0; q < 4; ++q) {
            t.cx[q] = base.cx[q];
            t.cy[q] = base.cy[q];
            t.cz[q] = base.cz[q];
        }
        t.bx0 = pp.bx0;
        t.bx1 = pp.bx1;
        t.by0 = pp.by0;
        t.by1 = pp.by1;
        t.bz0 = pp.bz0;
        t.bz1 = pp.bz1;
        t.tiles_x = pp.tiles_x;
        t.tiles_y = pp.tiles_y;
        t.zc = pp.zc;
        t.si = base.si;
        t.sj = base.sj;
        t.sk = base.sk;
        t.wavelet = base.wavelet;
        t.inv_vol = base.inv_vol;
        t.step_ptr = step_ptr;
        t.step_add = step_add;
        t.err = base.err;
        two_step_kernel<TCfg><<<pp.grid, TCfg::BLOCK, TCfg::SMEM_BYTES, st>>>(t, pm.two_u, pm.two_up,
                                                                              pm.two_m);
        CUDA_TRY(cudaGetLastError());
        ++t_launches;
    }
    const int nunits = (int)pp.shell.size();
    if (nunits == 0) return SGB_OK;
    for (int h = 0; h < 2; ++h) {
        StepArgs a = base;
        a.units = d_units;
        a.bx0 = pp.bx0;
        a.bx1 = pp.bx1;
        a.by0 = pp.by0;
        a.by1 = pp.by1;
        a.bz0 = pp.bz0;
        a.bz1 = pp.bz1;
        a.u_cur = h == 0 ? b_cur : c_next;
        a.u_out = h == 0 ? c_next : d_next2;
        a.step_ptr = step_ptr;
        a.step_add = step_add + h;
        const StepMaps &mp = h == 0 ? pm.shell0 : pm.shell1;
        CUDA_TRY(launch_dependent(shell_step_kernel<Cfg>, nunits, Cfg::BLOCK,
                                  Stage<Cfg, float>::SMEM_BYTES, st, a, mp.ucur, mp.ucur_in,
                                  mp.uprev, mp.m, mp.phi));
        ++t_launches;
    }
    (void)g;
    return SGB_OK;
}

// The time-loop schedule run_shot uses for grid g.
int resolve_schedule(const sgb_grid *g)
{
    if (g->schedule != SGB_SCHED_AUTO) return g->schedule;
    return SGB_SCHED_STEP;
}

// Resident CTAs of the dataflow kernel for storage T (its shared memory and
// launch bounds are those of the one-step kernel plus two item slots).
template <class T>
int prepare_flow(int *occ)
{
    const size_t smem = Stage<Cfg, T>::SMEM_BYTES + FLOW_SMEM_EXTRA;
    CUDA_TRY(cudaFuncSetAttribute(flow_step_kernel<Cfg, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, flow_step_kernel<Cfg, T>, Cfg::BLOCK,
                                                           smem));
    if (*occ < 1) return fail(SGB_ERR_CUDA, "dataflow kernel does not fit on an SM");
    return SGB_OK;
}

// Steps 0 .. nt-1 of a shot in one persistent dataflow launch.  base: the step
// constants with phi, error word, source and receivers; maps[p], buf: the
// tensor maps and buffers of steps of parity p (step n writes buf[n & 1]).
template <class T>
int run_flow(const sgb_layout_info &L, DevState *ds, cudaStream_t st, Scratch &sc,
             const StepArgs &base, const StepMaps (&maps)[2], void *const (&buf)[2], int n_begin,
             int n_end, const int32_t *rec_ijk, int nrec)
{
    int rc, occ = 0;
    if ((rc = prepare_flow<T>(&occ))) return rc;
    const int ctas = ds->sms * occ;
    StepArgs fa = base;
    fa.tiles_x = (L.Nx + Cfg::BX - 1) / Cfg::BX;
    fa.tiles_y = (L.Ny + Cfg::BY - 1) / Cfg::BY;
    const int tiles = fa.tiles_x * fa.tiles_y;
    // z-chunks: the longest (fewest priming planes) that still gives two items
    // per resident CTA and step; every chunk but the last has >= 8 planes, so a
    // unit's radius-4 planes lie in its own and the adjacent chunks
    fa.zc = L.Nz;
    for (int zc : {32, 24, 16, 12, 8}) {
        fa.zc = std::min(zc, L.Nz);
        if ((long long)tiles * ((L.Nz + fa.zc - 1) / fa.zc) >= 2LL * ctas) break;
    }
    const int chunks = (L.Nz + fa.zc - 1) / fa.zc, units = tiles * chunks;
    // receivers grouped by the unit that computes them
    std::vector<int> rs(units + 1, 0), rl(std::max(nrec, 1));
    auto unit_of = [&](int r) {
        const int i = rec_ijk[3 * r], j = rec_ijk[3 * r + 1], k = rec_ijk[3 * r + 2];
        return (k / fa.zc) * tiles + (j / Cfg::BY) * fa.tiles_x + i / Cfg::BX;
    };
    for (int r = 0; r < nrec; ++r) ++rs[unit_of(r) + 1];
    for (int u = 0; u < units; ++u) rs[u + 1] += rs[u];
    {
        std::vector<int> pos(rs.begin(), rs.end() - 1);
        for (int r = 0; r < nrec; ++r) rl[pos[unit_of(r)]++] = r;
    }
    int *d_done, *d_counter, *d_rs, *d_rl;
    if ((rc = sc.get((void **)&d_done, (size_t)units * 4)) || (rc = sc.get((void **)&d_counter, 16)) ||
        (rc = sc.get((void **)&d_rs, rs.size() * 4)) || (rc = sc.get((void **)&d_rl, rl.size() * 4)))
        return rc;
    {  // every unit has completed n_begin steps when the launch starts
        std::vector<int> d0(units, n_begin);
        CUDA_TRY(cudaMemcpyAsync(d_done, d0.data(), (size_t)units * 4, cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaStreamSynchronize(st));  // d0 is a pageable temporary
    }
    CUDA_TRY(cudaMemsetAsync(d_counter, 0, 4, st));
    CUDA_TRY(cudaMemcpyAsync(d_rs, rs.data(), rs.size() * 4, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(d_rl, rl.data(), rl.size() * 4, cudaMemcpyHostToDevice, st));
    StepArgs a0 = fa;
    a0.u_out = nullptr;  // per step: f.buf
    a0.u_cur = nullptr;
    a0.step_ptr = nullptr;
    FlowArgs f;
    f.buf[0] = buf[0];
    f.buf[1] = buf[1];
    f.units = units;
    f.tiles_x = fa.tiles_x;
    f.tiles_y = fa.tiles_y;
    f.n_begin = n_begin;
    f.n_end = n_end;
    f.counter = d_counter;
    f.done = d_done;
    f.rec_start = d_rs;
    f.rec_list = d_rl;
    const StepMaps &p0 = maps[0], &p1 = maps[1];
    flow_step_kernel<Cfg, T><<<ctas, Cfg::BLOCK, Stage<Cfg, T>::SMEM_BYTES + FLOW_SMEM_EXTRA, st>>>(
        a0, f, p0.ucur, p0.ucur_in, p0.uprev, p0.m, p0.phi, p1.ucur, p1.ucur_in, p1.uprev,
        p1.m, p1.phi);
    CUDA_TRY(cudaGetLastError());
    ++t_launches;
    // the pageable copies above are staged before they return; the scratch is
    // released stream-ordered after the launch
    return SGB_OK;
}

// Shot time loop and outputs for wavefield storage T (run_shot after its
// argument checks and the CFL check).
template <class T, bool DIFF = false>
// Steps n_begin .. n_end-1; state: null (start from zero fields) or three
// device compact fp32 arrays (u^n, u^{n-1}, phi^n) read at n_begin and
// overwritten with the state at n_end.  Traces rows are steps n_begin ...
int run_shot_t(const sgb_grid *g, const sgb_layout_info &L, DevState *ds, cudaStream_t st,
               Scratch &sc, const float *d_vel, const float *d_wav, int n_begin, int n_end,
               const int32_t *src_ijk, const int32_t *rec_ijk, int nrec, const long long *d_off,
               float *d_tr, float *final_u, float *const *state, int *d_err)
{
    int rc;
    const int nt = n_end, nsteps = n_end - n_begin;
    const long long ncomp = (long long)L.Nx * L.Ny * L.Nz;
    const size_t ubytes = (size_t)L.elems * sizeof(T), fbytes = (size_t)L.elems * 4;
    void *u0, *u1;
    float *phi, *m;
    ScaleState *ss = nullptr;
    int *d_step;
    void *dfield = nullptr;  // difference form: d^n = u^n - u^{n-1}, updated in place
    if ((rc = sc.get(&u0, ubytes)) || (rc = sc.get(&u1, ubytes)) ||
        (rc = sc.get((void **)&phi, fbytes)) || (rc = sc.get((void **)&m, fbytes)) ||
        (rc = sc.get((void **)&d_step, sizeof(int))))
        return rc;
    if (DIFF) {
        if ((rc = sc.get(&dfield, ubytes))) return rc;
        CUDA_TRY(cudaMemsetAsync(dfield, 0, ubytes, st));
    }
    CUDA_TRY(cudaMemcpyAsync(d_step, &n_begin, sizeof(int), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemsetAsync(m, 0, fbytes, st));
    if (!state) {
        CUDA_TRY(cudaMemsetAsync(u0, 0, ubytes, st));
        CUDA_TRY(cudaMemsetAsync(u1, 0, ubytes, st));
        CUDA_TRY(cudaMemsetAsync(phi, 0, fbytes, st));
    } else {  // u^n into buf[(n+1)&1], u^{n-1} into buf[n&1] (n = n_begin), phi^n
        void *bb[2] = {u0, u1};
        const int eg = ew_grid(L.elems, *ds);
        pack_t_kernel<T><<<eg, 256, 0, st>>>(pad_geom(L), state[0], static_cast<T *>(bb[(n_begin + 1) & 1]),
                                             L.elems);
        pack_t_kernel<T><<<eg, 256, 0, st>>>(pad_geom(L), state[1], static_cast<T *>(bb[n_begin & 1]),
                                             L.elems);
        pack_kernel<<<eg, 256, 0, st>>>(pad_geom(L), state[2], phi, L.elems);
        CUDA_TRY(cudaGetLastError());
        t_launches += 3;
    }
    ScaleState *ssd = nullptr;  // difference form: the scales of d
    if (Elem<T>::SCALED) {
        static const ScaleState init = {{1.0f, 1.0f, 1.0f, 1.0f}, {0.0f, 0.0f, 0.0f, 0.0f}};
        if ((rc = sc.get((void **)&ss, sizeof(ScaleState)))) return rc;
        CUDA_TRY(cudaMemcpyAsync(ss, &init, sizeof init, cudaMemcpyHostToDevice, st));
        if (DIFF) {
            if ((rc = sc.get((void **)&ssd, sizeof(ScaleState)))) return rc;
            CUDA_TRY(cudaMemcpyAsync(ssd, &init, sizeof init, cudaMemcpyHostToDevice, st));
        }
    }
    make_m_kernel<<<ew_grid(ncomp, *ds), 256, 0, st>>>(pad_geom(L), d_vel, g->dt, m);
    CUDA_TRY(cudaGetLastError());
    ++t_launches;

    // buf[0] holds u^{-1}, buf[1] holds u^0; step n reads buf[(n+1)&1] and
    // overwrites buf[n&1] with u^{n+1}.
    void *buf[2] = {u0, u1};
    StepArgs base;
    fill_step_constants(g, L, base);
    base.phi = phi;
    base.err = d_err;
    base.scale = ss;
    base.scale_d = ssd;
    if (src_ijk) {
        base.si = src_ijk[0];
        base.sj = src_ijk[1];
        base.sk = src_ijk[2];
        base.wavelet = d_wav;
        base.m_src = m + L.origin + (long long)src_ijk[2] * L.stride_z +
                     (long long)src_ijk[1] * L.sx + src_ijk[0];
    }
    base.nrec = nrec;
    base.rec_off = d_off;
    base.traces = d_tr;
    base.rec_n0 = n_begin;
    base.d_io = dfield;
    const int occ = DIFF ? (std::is_same<T, float>::value    ? ds->occ_df
                            : std::is_same<T, __half>::value ? ds->occ_dh
                                                             : ds->occ_db)
                    : std::is_same<T, float>::value ? ds->occ
                    : std::is_same<T, __half>::value ? ds->occ_h : ds->occ_b;
    int grid = 0;
    choose_decomposition(L.Nx, L.Ny, L.Nz, ds->sms, occ, base, &grid);
    StepMaps maps[2];  // [parity of n]; the difference form reads d^n through the u^{n-1} map
    for (int p = 0; p < 2; ++p)
        if ((rc = encode_step_maps<T>(maps[p], buf[(p + 1) & 1], DIFF ? dfield : buf[p & 1], m, phi,
                                      L)))
            return rc;

    auto args_for = [&](int parity, const int *step_ptr, int step_add) {
        StepArgs a = base;
        a.u_out = buf[parity & 1];
        a.u_cur = buf[(parity + 1) & 1];
        a.step_ptr = step_ptr;
        a.step_add = step_add;
        return a;
    };

    bool looped = false;
    if constexpr (!Elem<T>::SCALED && !DIFF) {
        if (resolve_schedule(g) == SGB_SCHED_FLOW && nsteps > 0) {
            if ((rc = run_flow<T>(L, ds, st, sc, base, maps, buf, n_begin, n_end, rec_ijk, nrec)))
                return rc;
            looped = true;
        }
    }
    const int GS = 32;  // steps per graph replay (even: the buffer parity repeats)
    const int replays = looped ? 0 : nsteps / GS;
    if (replays > 0) {
        cudaStream_t cs;
        CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        int crc = SGB_OK;
        cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (ce == cudaSuccess) {
            for (int i = 0; i < GS && crc == SGB_OK; ++i)
                crc = launch_step<T, DIFF>(args_for(n_begin + i, d_step, i), maps[(n_begin + i) & 1],
                                           grid, cs);
            if (crc == SGB_OK) {
                advance_kernel<<<1, 32, 0, cs>>>(d_step, GS);
                ce = cudaGetLastError();
            }
            cudaError_t ee = cudaStreamEndCapture(cs, &graph);
            if (ce == cudaSuccess) ce = ee;
        }
        t_launches -= GS;  // captured launches are counted at replay
        if (ce == cudaSuccess && crc == SGB_OK) ce = cudaGraphInstantiate(&exec, graph, 0);
        if (ce == cudaSuccess && crc == SGB_OK) {
            for (int r = 0; r < replays && ce == cudaSuccess; ++r) {
                ce = cudaGraphLaunch(exec, st);
                t_launches += GS + 1;
            }
        }
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cs);
        if (crc) return crc;
        CUDA_TRY(ce);
    }
    for (int n = looped ? n_end : n_begin + replays * GS; n < n_end; ++n)
        if ((rc = launch_step<T, DIFF>(args_for(n, nullptr, n), maps[n & 1], grid, st))) return rc;

    // u^k lives in buf[(k+1)&1] (written by step k-1): u^{nt} in buf[(nt+1)&1]
    const void *u_final_dev = buf[(nt + 1) & 1];
    const float *s_final = ss ? &ss->s[nt & 3] : nullptr;
    if (nrec > 0 && nsteps > 0 && !looped) {  // the dataflow launch sampled every row itself
        gather_t_kernel<T><<<(nrec + 255) / 256, 256, 0, st>>>(
            static_cast<const T *>(u_final_dev), d_off, nrec, s_final,
            d_tr + (size_t)(nsteps - 1) * nrec, d_err);
        CUDA_TRY(cudaGetLastError());
        ++t_launches;
    }
    if (state) {  // the state at n_end: u^{nt}, u^{nt-1}, phi^{nt}
        unpack_t_kernel<T><<<ew_grid(ncomp, *ds), 256, 0, st>>>(pad_geom(L),
            static_cast<const T *>(u_final_dev), s_final, state[0]);
        unpack_t_kernel<T><<<ew_grid(ncomp, *ds), 256, 0, st>>>(pad_geom(L),
            static_cast<const T *>(buf[nt & 1]), nullptr, state[1]);
        unpack_kernel<<<ew_grid(ncomp, *ds), 256, 0, st>>>(pad_geom(L), phi, state[2]);
        CUDA_TRY(cudaGetLastError());
        t_launches += 3;
    }
    if (final_u) {
        const bool host_u = !is_device_ptr(final_u);
        float *dst = final_u;
        if (host_u && (rc = sc.get((void **)&dst, (size_t)ncomp * 4))) return rc;
        unpack_t_kernel<T><<<ew_grid(ncomp, *ds), 256, 0, st>>>(
            pad_geom(L), static_cast<const T *>(u_final_dev), s_final, dst);
        CUDA_TRY(cudaGetLastError());
        ++t_launches;
        if (host_u)
            CUDA_TRY(cudaMemcpyAsync(final_u, dst, (size_t)ncomp * 4, cudaMemcpyDeviceToHost, st));
    }
    return SGB_OK;
}

// run_shot with SGB_SCHED_PAIRS (fp32): steps in temporally blocked pairs, an
// odd last step as one ordinary fused step.  Four wavefield buffers: a pair
// reads (u^{n-1}, u^n) from one two and writes (u^{n+1}, u^{n+2}) to the other.
int run_shot_pairs(const sgb_grid *g, const sgb_layout_info &L, DevState *ds, cudaStream_t st,
                   Scratch &sc, const float *d_vel, const float *d_wav, int nt,
                   const int32_t *src_ijk, int nrec, const long long *d_off, float *d_tr,
                   float *final_u, int *d_err)
{
    int rc;
    if ((rc = prepare_two_step())) return rc;
    const long long ncomp = (long long)L.Nx * L.Ny * L.Nz;
    const size_t fbytes = (size_t)L.elems * 4;
    float *u[4], *phi, *m;
    int *d_step;
    for (int q = 0; q < 4; ++q)
        if ((rc = sc.get((void **)&u[q], fbytes))) return rc;
    if ((rc = sc.get((void **)&phi, fbytes)) || (rc = sc.get((void **)&m, fbytes)) ||
        (rc = sc.get((void **)&d_step, sizeof(int))))
        return rc;
    CUDA_TRY(cudaMemsetAsync(d_step, 0, sizeof(int), st));
    for (int q = 0; q < 2; ++q) CUDA_TRY(cudaMemsetAsync(u[q], 0, fbytes, st));
    CUDA_TRY(cudaMemsetAsync(phi, 0, fbytes, st));
    CUDA_TRY(cudaMemsetAsync(m, 0, fbytes, st));
    make_m_kernel<<<ew_grid(ncomp, *ds), 256, 0, st>>>(pad_geom(L), d_vel, g->dt, m);
    CUDA_TRY(cudaGetLastError());
    ++t_launches;

    StepArgs base;
    fill_step_constants(g, L, base);
    base.phi = phi;
    base.err = d_err;
    if (src_ijk) {
        base.si = src_ijk[0];
        base.sj = src_ijk[1];
        base.sk = src_ijk[2];
        base.wavelet = d_wav;
    }
    base.nrec = nrec;
    base.rec_off = d_off;
    base.traces = d_tr;
    PairPlan pp;
    plan_pair(g, L, *ds, pp);
    int4 *d_units = nullptr;
    if (!pp.shell.empty()) {
        if ((rc = sc.get((void **)&d_units, pp.shell.size() * sizeof(int4)))) return rc;
        CUDA_TRY(cudaMemcpyAsync(d_units, pp.shell.data(), pp.shell.size() * sizeof(int4),
                                 cudaMemcpyHostToDevice, st));
    }
    // pair parity p: reads (u[2p], u[2p+1]) = (u^{n-1}, u^n), writes u[2(1-p)],
    // u[2(1-p)+1]
    PairMaps pm[2];
    for (int p = 0; p < 2; ++p)
        if ((rc = encode_pair_maps(pm[p], u[2 * p], u[2 * p + 1], u[2 * (1 - p)], m, phi, L)))
            return rc;
    auto pair = [&](int parity, const int *step_ptr, int step_add, cudaStream_t s2) {
        return launch_pair(g, pp, pm[parity], d_units, base, u[2 * (1 - parity)],
                           u[2 * (1 - parity) + 1], u[2 * parity + 1], step_ptr, step_add, s2);
    };

    const int GS = 32;  // steps per graph replay: 16 pairs (even: the parity repeats)
    const int replays = nt / GS;
    if (replays > 0) {
        cudaStream_t cs;
        CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        int crc = SGB_OK;
        const int64_t before = t_launches;
        cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (ce == cudaSuccess) {
            for (int j = 0; j < GS / 2 && crc == SGB_OK; ++j) crc = pair(j & 1, d_step, 2 * j, cs);
            if (crc == SGB_OK) {
                advance_kernel<<<1, 32, 0, cs>>>(d_step, GS);
                ce = cudaGetLastError();
            }
            cudaError_t ee = cudaStreamEndCapture(cs, &graph);
            if (ce == cudaSuccess) ce = ee;
        }
        const int64_t per_replay = t_launches - before + 1;
        t_launches = before;  // captured launches are counted at replay
        if (ce == cudaSuccess && crc == SGB_OK) ce = cudaGraphInstantiate(&exec, graph, 0);
        if (ce == cudaSuccess && crc == SGB_OK) {
            for (int r = 0; r < replays && ce == cudaSuccess; ++r) {
                ce = cudaGraphLaunch(exec, st);
                t_launches += per_replay;
            }
        }
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cs);
        if (crc) return crc;
        CUDA_TRY(ce);
    }
    int n = replays * GS;
    for (; n + 1 < nt; n += 2)
        if ((rc = pair((n / 2) & 1, nullptr, n, st))) return rc;
    // (u^{n-1}, u^n) now live in u[2p], u[2p+1], p = (n / 2) & 1
    const int par = (n / 2) & 1;
    float *u_final_dev = u[2 * par + 1];
    if (n < nt) {  // odd step count: one ordinary fused step, in place over u^{n-1}
        StepArgs a = base;
        a.u_out = u[2 * par];
        a.u_cur = u[2 * par + 1];
        a.step_add = n;
        int grid = 0;
        choose_decomposition(L.Nx, L.Ny, L.Nz, ds->sms, ds->occ, a, &grid);
        StepMaps mp;
        if ((rc = encode_step_maps<float>(mp, a.u_cur, a.u_out, m, phi, L))) return rc;
        if ((rc = launch_step<float>(a, mp, grid, st))) return rc;
        u_final_dev = u[2 * par];
    }
    if (nrec > 0 && nt > 0) {
        gather_t_kernel<float><<<(nrec + 255) / 256, 256, 0, st>>>(
            u_final_dev, d_off, nrec, nullptr, d_tr + (size_t)(nt - 1) * nrec, d_err);
        CUDA_TRY(cudaGetLastError());
        ++t_launches;
    }
    if (final_u) {
        const bool host_u = !is_device_ptr(final_u);
        float *dst = final_u;
        if (host_u && (rc = sc.get((void **)&dst, (size_t)ncomp * 4))) return rc;
        unpack_kernel<<<ew_grid(ncomp, *ds), 256, 0, st>>>(pad_geom(L), u_final_dev, dst);
        CUDA_TRY(cudaGetLastError());
        ++t_launches;
        if (host_u)
            CUDA_TRY(cudaMemcpyAsync(final_u, dst, (size_t)ncomp * 4, cudaMemcpyDeviceToHost, st));
    }
    return SGB_OK;
}

}  // namespace

extern "C" int stencil_step2(const sgb_grid *g, const float *u_prev, const float *u_cur,
                             float *u_next, float *u_next2, const float *m, float *phi,
                             int32_t step, const sgb_source *src, void *stream)
{
    sgb_layout_info L;
    int rc = check_grid(g, &L);
    if (rc) return rc;
    if (g->storage != SGB_FP32) return fail(SGB_ERR_INVALID_ARG, "stencil_step2: SGB_FP32 storage only");
    const float *f[4] = {u_prev, u_cur, u_next, u_next2};
    for (int q = 0; q < 4; ++q) {
        if (!f[q]) return fail(SGB_ERR_INVALID_ARG, "NULL field pointer");
        if (!aligned16(f[q])) return fail(SGB_ERR_INVALID_ARG, "field pointers must be 16-byte aligned");
    }
    if (!m || !aligned16(m) || (phi && !aligned16(phi)))
        return fail(SGB_ERR_INVALID_ARG, "m (and phi) must be non-NULL and 16-byte aligned");
    if (g->nb > 0 && !phi) return fail(SGB_ERR_INVALID_ARG, "phi is required when nb > 0");
    {
        const size_t fb = (size_t)L.elems * 4;
        const Span ins[] = {{u_prev, fb, "u_prev"}, {u_cur, fb, "u_cur"}, {m, fb, "m"}};
        const Span outs[] = {{u_next, fb, "u_next"}, {u_next2, fb, "u_next2"}, {phi, fb, "phi"}};
        if ((rc = check_no_overlap(outs, 3, ins, 3))) return rc;
        if (spans_overlap(ins[0], ins[1])) return fail(SGB_ERR_INVALID_ARG, "u_prev overlaps u_cur");
    }
    if (step < 0) return fail(SGB_ERR_INVALID_ARG, "step must be >= 0");
    if (src) {
        if (!in_inner(g, src->i, src->j, src->k))
            return fail(SGB_ERR_INVALID_ARG, "source (%d,%d,%d) outside the inner region", src->i,
                        src->j, src->k);
        if (!src->wavelet) return fail(SGB_ERR_INVALID_ARG, "source wavelet is NULL");
    }
    if ((double)g->dt > cfl_limit(g, g->vmax))
        return fail(SGB_ERR_UNSTABLE_DT, "dt %g above the CFL limit %g for vmax %g", (double)g->dt,
                    cfl_limit(g, g->vmax), (double)g->vmax);
    DevState *ds;
    if ((rc = device_state(&ds))) return rc;
    if ((rc = prepare_two_step())) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    StepArgs base;
    fill_step_constants(g, L, base);
    base.phi = phi;
    base.err = ds->err;
    if (src) {
        base.si = src->i;
        base.sj = src->j;
        base.sk = src->k;
        base.wavelet = src->wavelet;
    }
    PairPlan pp;
    plan_pair(g, L, *ds, pp);
    Scratch sc{st, ds->pool, {}};
    int4 *d_units = nullptr;
    if (!pp.shell.empty()) {
        if ((rc = sc.get((void **)&d_units, pp.shell.size() * sizeof(int4)))) return rc;
        CUDA_TRY(cudaMemcpyAsync(d_units, pp.shell.data(), pp.shell.size() * sizeof(int4),
                                 cudaMemcpyHostToDevice, st));
    }
    PairMaps pm;
    if ((rc = encode_pair_maps(pm, u_prev, u_cur, u_next, m, phi ? phi : m, L))) return rc;
    // the unit table's pageable copy is staged before cudaMemcpyAsync returns;
    // the scratch is released stream-ordered after the launches
    return launch_pair(g, pp, pm, d_units, base, u_next, u_next2, u_cur, nullptr, step, st);
}

namespace {

// run_shot and run_shot_segment: steps n_begin .. n_end-1; state (u^n,
// u^{n-1}, phi^n compact fp32, host or device) or null for zero fields and no
// state out.
int run_shot_common(const sgb_grid *g, const float *velocity, const float *wavelet, int n_begin,
                    int n_end, const int32_t *src_ijk, const int32_t *rec_ijk, int32_t nrec,
                    float *traces, float *final_u, float *const *state, void *stream)
{
    sgb_layout_info L;
    int rc = check_grid(g, &L);
    if (rc) return rc;
    const int nt = n_end, nsteps = n_end - n_begin;
    if (!velocity) return fail(SGB_ERR_INVALID_ARG, "velocity is NULL");
    if (n_begin < 0 || nsteps < 0) return fail(SGB_ERR_INVALID_ARG, "steps must satisfy 0 <= n_begin <= n_end");
    if (nsteps > 0 && src_ijk && !wavelet) return fail(SGB_ERR_INVALID_ARG, "wavelet is NULL");
    if (nrec < 0) return fail(SGB_ERR_INVALID_ARG, "nrec < 0");
    if (nrec > 0 && (!rec_ijk || (nsteps > 0 && !traces)))
        return fail(SGB_ERR_INVALID_ARG, "receiver arrays NULL");
    if (state && g->storage != SGB_FP32 && g->storage != SGB_BF16)
        return fail(SGB_ERR_INVALID_ARG, "shot segments need SGB_FP32 or SGB_BF16 storage");
    if (src_ijk && !in_inner(g, src_ijk[0], src_ijk[1], src_ijk[2]))
        return fail(SGB_ERR_INVALID_ARG, "source (%d,%d,%d) outside the inner region", src_ijk[0],
                    src_ijk[1], src_ijk[2]);
    std::vector<long long> off(nrec > 0 ? nrec : 0);
    for (int r = 0; r < nrec; ++r) {
        const int i = rec_ijk[3 * r], j = rec_ijk[3 * r + 1], k = rec_ijk[3 * r + 2];
        if (!in_inner(g, i, j, k))
            return fail(SGB_ERR_INVALID_ARG, "receiver %d (%d,%d,%d) outside the inner region", r,
                        i, j, k);
        off[r] = L.origin + (long long)k * L.stride_z + (long long)j * L.sx + i;
    }
    const long long ncomp = (long long)L.Nx * L.Ny * L.Nz;
    const size_t cb = (size_t)ncomp * 4;
    {
        const Span ins[] = {{velocity, cb, "velocity"},
                            {src_ijk ? wavelet : nullptr, (size_t)nt * 4, "wavelet"}};
        const Span outs[] = {{nrec > 0 ? traces : nullptr, (size_t)nsteps * nrec * 4, "traces"},
                             {final_u, cb, "final_u"},
                             {state ? state[0] : nullptr, cb, "state u^n"},
                             {state ? state[1] : nullptr, cb, "state u^{n-1}"},
                             {state ? state[2] : nullptr, cb, "state phi^n"}};
        if ((rc = check_no_overlap(outs, 5, ins, 2))) return rc;
    }
    DevState *ds;
    if ((rc = device_state(&ds))) return rc;
    cudaStream_t st = (cudaStream_t)stream;

    Scratch sc{st, ds->pool, {}};
    int *d_err = nullptr;  // this call's own device error word
    if ((rc = sc.get((void **)&d_err, sizeof(int)))) return rc;
    CUDA_TRY(cudaMemsetAsync(d_err, 0, sizeof(int), st));
    const float *d_vel = velocity;
    if (!is_device_ptr(velocity)) {
        float *t;
        if ((rc = sc.get((void **)&t, cb))) return rc;
        CUDA_TRY(cudaMemcpyAsync(t, velocity, cb, cudaMemcpyHostToDevice, st));
        d_vel = t;
    }
    // velocity range -> CFL check against the model's actual maximum
    int *d_range;
    if ((rc = sc.get((void **)&d_range, 4 * sizeof(int)))) return rc;
    int init[4] = {0, 0x7f7fffff, 0, 0};
    CUDA_TRY(cudaMemcpyAsync(d_range, init, sizeof init, cudaMemcpyHostToDevice, st));
    vel_range_kernel<<<ew_grid(ncomp, *ds), 256, 0, st>>>(d_vel, ncomp, d_range);
    CUDA_TRY(cudaGetLastError());
    ++t_launches;
    int range[4];
    CUDA_TRY(cudaMemcpyAsync(range, d_range, sizeof range, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (range[2] != 0) return fail(SGB_ERR_INVALID_ARG, "velocity has non-positive or non-finite values");
    float vmax_model;
    memcpy(&vmax_model, &range[0], 4);
    if ((double)g->dt > cfl_limit(g, vmax_model))
        return fail(SGB_ERR_UNSTABLE_DT, "dt %g above the CFL limit %g of the model (vmax %g)",
                    (double)g->dt, cfl_limit(g, vmax_model), (double)vmax_model);

    const float *d_wav = wavelet;
    if (wavelet && nt > 0 && !is_device_ptr(wavelet)) {
        float *t;
        if ((rc = sc.get((void **)&t, (size_t)nt * 4))) return rc;
        CUDA_TRY(cudaMemcpyAsync(t, wavelet, (size_t)nt * 4, cudaMemcpyHostToDevice, st));
        d_wav = t;
    }
    float *d_tr = traces;
    const bool host_traces = nrec > 0 && !is_device_ptr(traces);
    if (host_traces && nsteps > 0) {
        if ((rc = sc.get((void **)&d_tr, (size_t)nsteps * nrec * 4))) return rc;
    }
    long long *d_off = nullptr;
    if (nrec > 0) {
        if ((rc = sc.get((void **)&d_off, (size_t)nrec * 8))) return rc;
        CUDA_TRY(cudaMemcpyAsync(d_off, off.data(), (size_t)nrec * 8, cudaMemcpyHostToDevice, st));
    }
    // the state on the device (host arrays are staged through scratch)
    float *d_state[3] = {nullptr, nullptr, nullptr};
    bool host_state[3] = {false, false, false};
    if (state) {
        for (int q = 0; q < 3; ++q) {
            d_state[q] = state[q];
            if (!is_device_ptr(state[q])) {
                host_state[q] = true;
                if ((rc = sc.get((void **)&d_state[q], cb))) return rc;
                CUDA_TRY(cudaMemcpyAsync(d_state[q], state[q], cb, cudaMemcpyHostToDevice, st));
            }
        }
    }
    float *const *dst = state ? d_state : nullptr;
    switch (g->storage) {
    case SGB_FP16_SCALED:
        rc = run_shot_t<__half>(g, L, ds, st, sc, d_vel, d_wav, n_begin, n_end, src_ijk, rec_ijk,
                                nrec, d_off, d_tr, final_u, dst, d_err);
        break;
    case SGB_BF16:
        rc = run_shot_t<__nv_bfloat16>(g, L, ds, st, sc, d_vel, d_wav, n_begin, n_end, src_ijk,
                                       rec_ijk, nrec, d_off, d_tr, final_u, dst, d_err);
        break;
    case SGB_FP32_DIFF:
        rc = run_shot_t<float, true>(g, L, ds, st, sc, d_vel, d_wav, n_begin, n_end, src_ijk,
                                     rec_ijk, nrec, d_off, d_tr, final_u, dst, d_err);
        break;
    case SGB_BF16_DIFF:
        rc = run_shot_t<__nv_bfloat16, true>(g, L, ds, st, sc, d_vel, d_wav, n_begin, n_end,
                                             src_ijk, rec_ijk, nrec, d_off, d_tr, final_u, dst,
                                             d_err);
        break;
    case SGB_FP16_DIFF:
        rc = run_shot_t<__half, true>(g, L, ds, st, sc, d_vel, d_wav, n_begin, n_end, src_ijk,
                                      rec_ijk, nrec, d_off, d_tr, final_u, dst, d_err);
        break;
    default:
        // temporal blocking covers whole shots; a segment takes one step per launch
        if (g->schedule == SGB_SCHED_PAIRS && !state && n_begin == 0)
            rc = run_shot_pairs(g, L, ds, st, sc, d_vel, d_wav, nt, src_ijk, nrec, d_off, d_tr,
                                final_u, d_err);
        else
            rc = run_shot_t<float>(g, L, ds, st, sc, d_vel, d_wav, n_begin, n_end, src_ijk, rec_ijk,
                                   nrec, d_off, d_tr, final_u, dst, d_err);
    }
    if (rc) return rc;
    if (host_traces && nsteps > 0)
        CUDA_TRY(cudaMemcpyAsync(traces, d_tr, (size_t)nsteps * nrec * 4, cudaMemcpyDeviceToHost, st));
    for (int q = 0; q < 3; ++q)
        if (host_state[q]) CUDA_TRY(cudaMemcpyAsync(state[q], d_state[q], cb, cudaMemcpyDeviceToHost, st));
    int dev_err = 0;
    CUDA_TRY(cudaMemcpyAsync(&dev_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return dev_err_status(dev_err);
}

}  // namespace

extern "C" int run_shot(const sgb_grid *g, const float *velocity, const float *wavelet, int32_t nt,
                        const int32_t *src_ijk, const int32_t *rec_ijk, int32_t nrec,
                        float *traces, float *final_u, void *stream)
{
    return run_shot_common(g, velocity, wavelet, 0, nt, src_ijk, rec_ijk, nrec, traces, final_u,
                           nullptr, stream);
}

extern "C" int run_shot_segment(const sgb_grid *g, const float *velocity, const float *wavelet,
                                int32_t n_begin, int32_t n_end, const int32_t *src_ijk,
                                const int32_t *rec_ijk, int32_t nrec, float *traces, float *u_cur,
                                float *u_prev, float *phi, void *stream)
{
    if (!u_cur || !u_prev || !phi) return fail(SGB_ERR_INVALID_ARG, "state arrays NULL");
    float *const state[3] = {u_cur, u_prev, phi};
    return run_shot_common(g, velocity, wavelet, n_begin, n_end, src_ijk, rec_ijk, nrec, traces,
                           nullptr, state, stream);
}

// ---------------------------------------------------------------------------
// Allocation-free shot.  Some callers cannot allocate device memory once they
// are running: a serving process whose device memory is all held by another
// allocator's pool, or a real-time loop that forbids cudaMalloc/cudaFree (and
// the device-wide synchronisation they can imply) after start-up.  For them,
// run_shot_noalloc takes its scratch from a fixed file-scope device array
// instead of the library's pool.
// ---------------------------------------------------------------------------
#define SGB_NOALLOC_SCRATCH_BYTES (32u << 20)

// Scratch of run_shot_noalloc: two wavefields, phi, m, receiver tables.  Every
// GPU that loads this library holds it until the process exits.  In host code
// this name is only a stand-in: kernels get the device address obtained with
// cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SGB_NOALLOC_SCRATCH_BYTES];

namespace {

struct NoAllocState {
    bool ready = false;
    unsigned char *scratch = nullptr;  // device address of g_noalloc_scratch
    int sms = 0, occ = 0;
};
NoAllocState g_noalloc[64];

// Once per device, with that device current: resolve the device address of
// the scratch array and the step kernel's launch limits.
int noalloc_setup(NoAllocState **out)
{
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(SGB_ERR_CUDA, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    NoAllocState &s = g_noalloc[dev];
    if (!s.ready) {
        CUDA_TRY(cudaGetSymbolAddress((void **)&s.scratch, g_noalloc_scratch));
        CUDA_TRY(cudaDeviceGetAttribute(&s.sms, cudaDevAttrMultiProcessorCount, dev));
        int rc0;
        if ((rc0 = prepare_step_kernel<float>(&s.occ))) return rc0;
        if (!g_encode) {
            cudaDriverEntryPointQueryResult q;
            void *fn = nullptr;
            CUDA_TRY(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                      cudaEnableDefault, &q));
            if (q != cudaDriverEntryPointSuccess || !fn)
                return fail(SGB_ERR_CUDA, "cuTensorMapEncodeTiled not available");
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        }
        s.ready = true;
    }
    *out = &s;
    return SGB_OK;
}

__global__ void rec_offsets_kernel(const int32_t *ijk, int nrec, long long sx, long long sxy,
                                   long long origin, long long *off)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < nrec)
        off[r] = origin + (long long)ijk[3 * r + 2] * sxy + (long long)ijk[3 * r + 1] * sx +
                 ijk[3 * r];
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

extern "C" int run_shot_noalloc(const sgb_grid *g, const float *velocity, const float *wavelet,
                                int32_t nt, const int32_t *src_ijk, const int32_t *rec_ijk,
                                int32_t nrec, float *traces, float *final_u, void *stream)
{
    sgb_layout_info L;
    int rc = check_grid(g, &L);
    if (rc) return rc;
    if (g->storage != SGB_FP32)
        return fail(SGB_ERR_INVALID_ARG, "run_shot_noalloc: only SGB_FP32 storage");
    if (!velocity) return fail(SGB_ERR_INVALID_ARG, "velocity is NULL");
    if (nt < 0) return fail(SGB_ERR_INVALID_ARG, "nt must be >= 0");
    if (nt > 0 && src_ijk && !wavelet) return fail(SGB_ERR_INVALID_ARG, "wavelet is NULL");
    if (nrec < 0) return fail(SGB_ERR_INVALID_ARG, "nrec < 0");
    if (nrec > 0 && (!rec_ijk || !traces)) return fail(SGB_ERR_INVALID_ARG, "receiver arrays NULL");
    if (src_ijk && !in_inner(g, src_ijk[0], src_ijk[1], src_ijk[2]))
        return fail(SGB_ERR_INVALID_ARG, "source (%d,%d,%d) outside the inner region", src_ijk[0],
                    src_ijk[1], src_ijk[2]);
    for (int r = 0; r < nrec; ++r)
        if (!in_inner(g, rec_ijk[3 * r], rec_ijk[3 * r + 1], rec_ijk[3 * r + 2]))
            return fail(SGB_ERR_INVALID_ARG, "receiver %d outside the inner region", r);
    const long long ncomp = (long long)L.Nx * L.Ny * L.Nz;
    {
        const Span ins[] = {{velocity, (size_t)ncomp * 4, "velocity"},
                            {src_ijk ? wavelet : nullptr, (size_t)nt * 4, "wavelet"}};
        const Span outs[] = {{nrec > 0 ? traces : nullptr, (size_t)nt * nrec * 4, "traces"},
                             {final_u, (size_t)ncomp * 4, "final_u"}};
        if ((rc = check_no_overlap(outs, 2, ins, 2))) return rc;
    }
    // scratch layout inside the fixed array
    const size_t fbytes = align256((size_t)L.elems * 4);
    const size_t off_u0 = 0, off_u1 = fbytes, off_phi = 2 * fbytes, off_m = 3 * fbytes;
    const size_t off_ijk = 4 * fbytes;
    const size_t off_rec = off_ijk + align256((size_t)nrec * 12);
    const size_t off_range = off_rec + align256((size_t)nrec * 8);  // range[4], then error word
    const size_t need = off_range + 256;
    if (need > SGB_NOALLOC_SCRATCH_BYTES)
        return fail(SGB_ERR_INVALID_ARG,
                    "run_shot_noalloc: this grid and receiver set need %zu bytes of scratch, above "
                    "the fixed %u bytes (about 2M padded points per field); use run_shot",
                    need, (unsigned)SGB_NOALLOC_SCRATCH_BYTES);
    const bool dev_ok = is_device_ptr(velocity) && (!src_ijk || nt == 0 || is_device_ptr(wavelet)) &&
                        (nrec == 0 || is_device_ptr(traces)) && (!final_u || is_device_ptr(final_u));
    if (!dev_ok)
        return fail(SGB_ERR_INVALID_ARG,
                    "run_shot_noalloc: velocity, wavelet, traces and final_u must be device pointers");
    NoAllocState *ns;
    if ((rc = noalloc_setup(&ns))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *base = ns->scratch;
    float *u0 = (float *)(base + off_u0), *u1 = (float *)(base + off_u1);
    float *phi = (float *)(base + off_phi), *m = (float *)(base + off_m);
    int32_t *d_ijk = (int32_t *)(base + off_ijk);
    long long *d_off = (long long *)(base + off_rec);
    int *d_range = (int *)(base + off_range);
    int *d_err = d_range + 4;  // this entry point's own error word
    const int ewg = (int)std::min<long long>((ncomp + 255) / 256, (long long)ns->sms * 8);

    // the array keeps the previous call's contents: clear what must start at zero
    CUDA_TRY(cudaMemsetAsync(base, 0, off_ijk, st));  // u0, u1, phi, m
    int init[8] = {0, 0x7f7fffff, 0, 0, 0, 0, 0, 0};  // velocity range; error word = 0
    CUDA_TRY(cudaMemcpyAsync(d_range, init, sizeof init, cudaMemcpyHostToDevice, st));
    vel_range_kernel<<<ewg, 256, 0, st>>>(velocity, ncomp, d_range);
    CUDA_TRY(cudaGetLastError());
    ++t_launches;
    int range[4];
    CUDA_TRY(cudaMemcpyAsync(range, d_range, sizeof range, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (range[2] != 0) return fail(SGB_ERR_INVALID_ARG, "velocity has non-positive or non-finite values");
    float vmax_model;
    memcpy(&vmax_model, &range[0], 4);
    if ((double)g->dt > cfl_limit(g, vmax_model))
        return fail(SGB_ERR_UNSTABLE_DT, "dt %g above the CFL limit %g of the model (vmax %g)",
                    (double)g->dt, cfl_limit(g, vmax_model), (double)vmax_model);
    make_m_kernel<<<ewg, 256, 0, st>>>(pad_geom(L), velocity, g->dt, m);
    CUDA_TRY(cudaGetLastError());
    ++t_launches;
    if (nrec > 0) {
        CUDA_TRY(cudaMemcpyAsync(d_ijk, rec_ijk, (size_t)nrec * 12, cudaMemcpyHostToDevice, st));
        rec_offsets_kernel<<<(nrec + 255) / 256, 256, 0, st>>>(d_ijk, nrec, L.sx, L.stride_z,
                                                               L.origin, d_off);
        CUDA_TRY(cudaGetLastError());
        ++t_launches;
    }

    float *buf[2] = {u0, u1};  // buf[0] = u^{-1}, buf[1] = u^0
    StepArgs base_args;
    fill_step_constants(g, L, base_args);
    base_args.phi = phi;
    base_args.err = d_err;
    if (src_ijk) {
        base_args.si = src_ijk[0];
        base_args.sj = src_ijk[1];
        base_args.sk = src_ijk[2];
        base_args.wavelet = wavelet;
    }
    base_args.nrec = nrec;
    base_args.rec_off = d_off;
    base_args.traces = traces;
    int grid = 0;
    choose_decomposition(L.Nx, L.Ny, L.Nz, ns->sms, ns->occ, base_args, &grid);
    StepMaps maps[2];
    for (int p = 0; p < 2; ++p)
        if ((rc = encode_step_maps<float>(maps[p], buf[(p + 1) & 1], buf[p & 1], m, phi, L))) return rc;
    for (int n = 0; n < nt; ++n) {
        StepArgs a = base_args;
        a.u_out = buf[n & 1];
        a.u_cur = buf[(n + 1) & 1];
        a.step_ptr = nullptr;
        a.step_add = n;
        if ((rc = launch_step<float>(a, maps[n & 1], grid, st))) return rc;
    }
    float *u_last = nt > 0 ? buf[(nt - 1) & 1] : buf[1];
    if (nrec > 0 && nt > 0) {
        gather_kernel<<<(nrec + 255) / 256, 256, 0, st>>>(u_last, d_off, nrec,
                                                          traces + (size_t)(nt - 1) * nrec, d_err);
        CUDA_TRY(cudaGetLastError());
        ++t_launches;
    }
    if (final_u) {
        unpack_kernel<<<ewg, 256, 0, st>>>(pad_geom(L), u_last, final_u);
        CUDA_TRY(cudaGetLastError());
        ++t_launches;
    }
    int dev_err = 0;
    CUDA_TRY(cudaMemcpyAsync(&dev_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return dev_err_status(dev_err);
}

#include "serve_impl.cuh"
#include "adjoint.cuh"
