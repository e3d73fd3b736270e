// C-ABI host side of seisgb: validation, padded layout, TMA tensor maps,
// launch configuration, CUDA-graph time loop (run_shot).
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
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

extern "C" const char *sgb_last_error(void) { return t_last_error.c_str(); }

extern "C" int64_t sgb_launch_count(int reset)
{
    int64_t v = t_launches;
    if (reset) t_launches = 0;
    return v;
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
    int *err = nullptr;
    cudaMemPool_t pool = nullptr;
};

std::mutex g_mu;
DevState g_dev[64];
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

// Allow the step kernel for storage T its dynamic shared memory; report how
// many of its CTAs fit on one SM.
template <class T>
int prepare_step_kernel(int *occ)
{
    using G = Stage<Cfg, T>;
    CUDA_TRY(cudaFuncSetAttribute(fused_step_kernel<Cfg, T>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)G::SMEM_BYTES));
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, fused_step_kernel<Cfg, T>,
                                                           Cfg::BLOCK, G::SMEM_BYTES));
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
    if (g->storage != SGB_FP32 && g->storage != SGB_FP16_SCALED && g->storage != SGB_BF16)
        return fail(SGB_ERR_INVALID_ARG, "unknown storage format %d", g->storage);
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

template <class T>
int launch_step(const StepArgs &a, const StepMaps &mp, int grid, cudaStream_t st)
{
    fused_step_kernel<Cfg, T><<<grid, Cfg::BLOCK, Stage<Cfg, T>::SMEM_BYTES, st>>>(
        a, mp.ucur, mp.ucur_in, mp.uprev, mp.m, mp.phi);
    CUDA_TRY(cudaGetLastError());
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

extern "C" int sgb_device_status(void *stream)
{
    DevState *ds;
    int rc = device_state(&ds);
    if (rc) return rc;
    int v = 0;
    if ((rc = read_and_clear_dev_err(ds->err, *ds, (cudaStream_t)stream, &v))) return rc;
    return dev_err_status(v);
}

extern "C" int stencil_step(const sgb_grid *g, const void *u_cur, void *u_prev_to_next,
                            const float *m, float *phi, int32_t step, const sgb_source *src,
                            const sgb_receivers *rec, void *stream)
{
    sgb_layout_info L;
    int rc = check_grid(g, &L);
    if (rc) return rc;
    if (g->storage != SGB_FP32)
        return fail(SGB_ERR_INVALID_ARG, "stencil_step: only SGB_FP32 storage here");
    if (!u_cur || !u_prev_to_next || !m) return fail(SGB_ERR_INVALID_ARG, "NULL field pointer");
    if (g->nb > 0 && !phi) return fail(SGB_ERR_INVALID_ARG, "phi is required when nb > 0");
    if (!aligned16(u_cur) || !aligned16(u_prev_to_next) || !aligned16(m) || (phi && !aligned16(phi)))
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

    StepArgs a;
    fill_step_constants(g, L, a);
    a.u_out = u_prev_to_next;
    a.u_cur = u_cur;
    a.phi = phi;
    a.err = ds->err;
    a.step_add = step;
    if (src) {
        a.si = src->i;
        a.sj = src->j;
        a.sk = src->k;
        a.wavelet = src->wavelet;
    }
    int grid = 0;
    choose_decomposition(L.Nx, L.Ny, L.Nz, ds->sms, ds->occ, a, &grid);
    StepMaps mp;
    if ((rc = encode_step_maps<float>(mp, a.u_cur, a.u_out, m, phi, L))) return rc;
    if ((rc = launch_step<float>(a, mp, grid, st))) return rc;
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
        gather_kernel<<<(rec->nrec + 255) / 256, 256, 0, st>>>(
            static_cast<const float *>(u_prev_to_next), static_cast<const long long *>(d_off),
            rec->nrec, rec->traces, ds->err);
        CUDA_TRY(cudaGetLastError());
        ++t_launches;
        // the pageable copy above is staged before cudaMemcpyAsync returns; the
        // scratch is released stream-ordered after the gather
    }
    return SGB_OK;
}

namespace {

// Shot time loop and outputs for wavefield storage T (run_shot after its
// argument checks and the CFL check).
template <class T>
int run_shot_t(const sgb_grid *g, const sgb_layout_info &L, DevState *ds, cudaStream_t st,
               Scratch &sc, const float *d_vel, const float *d_wav, int nt,
               const int32_t *src_ijk, int nrec, const long long *d_off, float *d_tr,
               float *final_u, int *d_err)
{
    int rc;
    const long long ncomp = (long long)L.Nx * L.Ny * L.Nz;
    const size_t ubytes = (size_t)L.elems * sizeof(T), fbytes = (size_t)L.elems * 4;
    void *u0, *u1;
    float *phi, *m;
    ScaleState *ss = nullptr;
    int *d_step;
    if ((rc = sc.get(&u0, ubytes)) || (rc = sc.get(&u1, ubytes)) ||
        (rc = sc.get((void **)&phi, fbytes)) || (rc = sc.get((void **)&m, fbytes)) ||
        (rc = sc.get((void **)&d_step, sizeof(int))))
        return rc;
    CUDA_TRY(cudaMemsetAsync(d_step, 0, sizeof(int), st));
    CUDA_TRY(cudaMemsetAsync(u0, 0, ubytes, st));
    CUDA_TRY(cudaMemsetAsync(u1, 0, ubytes, st));
    CUDA_TRY(cudaMemsetAsync(phi, 0, fbytes, st));
    CUDA_TRY(cudaMemsetAsync(m, 0, fbytes, st));
    if (Elem<T>::SCALED) {
        if ((rc = sc.get((void **)&ss, sizeof(ScaleState)))) return rc;
        static const ScaleState init = {{1.0f, 1.0f, 1.0f, 1.0f}, {0.0f, 0.0f, 0.0f, 0.0f}};
        CUDA_TRY(cudaMemcpyAsync(ss, &init, sizeof init, cudaMemcpyHostToDevice, st));
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
    const int occ = std::is_same<T, float>::value ? ds->occ
                    : std::is_same<T, __half>::value ? ds->occ_h : ds->occ_b;
    int grid = 0;
    choose_decomposition(L.Nx, L.Ny, L.Nz, ds->sms, occ, base, &grid);
    StepMaps maps[2];  // [parity of n]
    for (int p = 0; p < 2; ++p)
        if ((rc = encode_step_maps<T>(maps[p], buf[(p + 1) & 1], buf[p & 1], m, phi, L))) return rc;

    auto args_for = [&](int parity, const int *step_ptr, int step_add) {
        StepArgs a = base;
        a.u_out = buf[parity & 1];
        a.u_cur = buf[(parity + 1) & 1];
        a.step_ptr = step_ptr;
        a.step_add = step_add;
        return a;
    };

    const int GS = 32;  // steps per graph replay (even: the buffer parity repeats)
    const int replays = nt / GS;
    if (replays > 0) {
        cudaStream_t cs;
        CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        int crc = SGB_OK;
        cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (ce == cudaSuccess) {
            for (int i = 0; i < GS && crc == SGB_OK; ++i)
                crc = launch_step<T>(args_for(i, d_step, i), maps[i & 1], grid, cs);
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
    for (int n = replays * GS; n < nt; ++n)
        if ((rc = launch_step<T>(args_for(n, nullptr, n), maps[n & 1], grid, st))) return rc;

    // u^{nt}: written by step nt-1 into buf[(nt-1)&1] (u^0 = buf[1] when nt = 0)
    const void *u_final_dev = nt > 0 ? buf[(nt - 1) & 1] : buf[1];
    const float *s_final = ss ? &ss->s[nt & 3] : nullptr;
    if (nrec > 0 && nt > 0) {
        gather_t_kernel<T><<<(nrec + 255) / 256, 256, 0, st>>>(
            static_cast<const T *>(u_final_dev), d_off, nrec, s_final,
            d_tr + (size_t)(nt - 1) * nrec, d_err);
        CUDA_TRY(cudaGetLastError());
        ++t_launches;
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

}  // namespace

extern "C" int run_shot(const sgb_grid *g, const float *velocity, const float *wavelet, int32_t nt,
                        const int32_t *src_ijk, const int32_t *rec_ijk, int32_t nrec,
                        float *traces, float *final_u, void *stream)
{
    sgb_layout_info L;
    int rc = check_grid(g, &L);
    if (rc) return rc;
    if (!velocity) return fail(SGB_ERR_INVALID_ARG, "velocity is NULL");
    if (nt < 0) return fail(SGB_ERR_INVALID_ARG, "nt must be >= 0");
    if (nt > 0 && src_ijk && !wavelet) return fail(SGB_ERR_INVALID_ARG, "wavelet is NULL");
    if (nrec < 0) return fail(SGB_ERR_INVALID_ARG, "nrec < 0");
    if (nrec > 0 && (!rec_ijk || !traces)) return fail(SGB_ERR_INVALID_ARG, "receiver arrays NULL");
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
    {
        const Span ins[] = {{velocity, (size_t)ncomp * 4, "velocity"},
                            {src_ijk ? wavelet : nullptr, (size_t)nt * 4, "wavelet"}};
        const Span outs[] = {{nrec > 0 ? traces : nullptr, (size_t)nt * nrec * 4, "traces"},
                             {final_u, (size_t)ncomp * 4, "final_u"}};
        if ((rc = check_no_overlap(outs, 2, ins, 2))) return rc;
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
        if ((rc = sc.get((void **)&t, (size_t)ncomp * 4))) return rc;
        CUDA_TRY(cudaMemcpyAsync(t, velocity, (size_t)ncomp * 4, cudaMemcpyHostToDevice, st));
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
    if (host_traces && nt > 0) {
        if ((rc = sc.get((void **)&d_tr, (size_t)nt * nrec * 4))) return rc;
    }
    long long *d_off = nullptr;
    if (nrec > 0) {
        if ((rc = sc.get((void **)&d_off, (size_t)nrec * 8))) return rc;
        CUDA_TRY(cudaMemcpyAsync(d_off, off.data(), (size_t)nrec * 8, cudaMemcpyHostToDevice, st));
    }
    switch (g->storage) {
    case SGB_FP16_SCALED:
        rc = run_shot_t<__half>(g, L, ds, st, sc, d_vel, d_wav, nt, src_ijk, nrec, d_off, d_tr, final_u, d_err);
        break;
    case SGB_BF16:
        rc = run_shot_t<__nv_bfloat16>(g, L, ds, st, sc, d_vel, d_wav, nt, src_ijk, nrec, d_off, d_tr,
                                       final_u, d_err);
        break;
    default:
        rc = run_shot_t<float>(g, L, ds, st, sc, d_vel, d_wav, nt, src_ijk, nrec, d_off, d_tr, final_u, d_err);
    }
    if (rc) return rc;
    if (host_traces && nt > 0)
        CUDA_TRY(cudaMemcpyAsync(traces, d_tr, (size_t)nt * nrec * 4, cudaMemcpyDeviceToHost, st));
    int dev_err = 0;
    CUDA_TRY(cudaMemcpyAsync(&dev_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return dev_err_status(dev_err);
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
