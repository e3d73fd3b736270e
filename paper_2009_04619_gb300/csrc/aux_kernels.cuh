// Small helper kernels around the fused step: layout conversion, m = v^2 dt^2,
// velocity range, receiver gathers and the graph step counter.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace sgb {

struct PadGeom {
    int Nx, Ny, Nz;
    long long sx, sxy, origin;
};

// compact (Nz, Ny, Nx) -> padded; halo and row padding receive zeros.
// Padded coordinates (ii, jj, kk) map to computed (ii - 8, jj - 4, kk - 4).
__global__ void pack_kernel(PadGeom g, const float *__restrict__ src, float *__restrict__ dst,
                            long long elems)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < elems; p += stride) {
        const long long kk = p / g.sxy, rem = p - kk * g.sxy;
        const long long jj = rem / g.sx, ii = rem - jj * g.sx;
        const long long i = ii - 8, j = jj - 4, k = kk - 4;
        float v = 0.0f;
        if (i >= 0 && i < g.Nx && j >= 0 && j < g.Ny && k >= 0 && k < g.Nz)
            v = src[(k * g.Ny + j) * g.Nx + i];
        dst[p] = v;
    }
}

// compact fp32 (Nz, Ny, Nx) -> padded field of storage T (rounded to nearest);
// halo and row padding receive zeros.
template <class T>
__global__ void pack_t_kernel(PadGeom g, const float *__restrict__ src, T *__restrict__ dst,
                              long long elems)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < elems; p += stride) {
        const long long kk = p / g.sxy, rem = p - kk * g.sxy;
        const long long jj = rem / g.sx, ii = rem - jj * g.sx;
        const long long i = ii - 8, j = jj - 4, k = kk - 4;
        float v = 0.0f;
        if (i >= 0 && i < g.Nx && j >= 0 && j < g.Ny && k >= 0 && k < g.Nz)
            v = src[(k * g.Ny + j) * g.Nx + i];
        dst[p] = T(v);
    }
}

// padded -> compact
__global__ void unpack_kernel(PadGeom g, const float *__restrict__ src, float *__restrict__ dst)
{
    const long long n = (long long)g.Nx * g.Ny * g.Nz;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) {
        const long long i = c % g.Nx, t = c / g.Nx;
        const long long j = t % g.Ny, k = t / g.Ny;
        dst[c] = src[g.origin + k * g.sxy + j * g.sx + i];
    }
}

// m = v^2 dt^2 at computed points of a zeroed padded array.
__global__ void make_m_kernel(PadGeom g, const float *__restrict__ vel, float dt,
                              float *__restrict__ m)
{
    const long long n = (long long)g.Nx * g.Ny * g.Nz;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) {
        const long long i = c % g.Nx, t = c / g.Nx;
        const long long j = t % g.Ny, k = t / g.Ny;
        const float v = vel[c] * dt;
        m[g.origin + k * g.sxy + j * g.sx + i] = v * v;
    }
}

// out[0] = max(v), out[1] = min(v) as float bit patterns (positive floats order
// like integers); out[2] counts non-finite values.
__global__ void vel_range_kernel(const float *__restrict__ vel, long long n, int *out)
{
    float mx = 0.0f, mn = 3.0e38f;
    int bad = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) {
        const float v = vel[c];
        if (!isfinite(v) || v <= 0.0f) {
            bad = 1;
            continue;
        }
        mx = fmaxf(mx, v);
        mn = fminf(mn, v);
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(out, __float_as_int(mx));
        atomicMin(out + 1, __float_as_int(mn));
        if (bad) atomicAdd(out + 2, 1);
    }
}

// row[r] = u[off[r]]; flags non-finite samples.
__global__ void gather_kernel(const float *__restrict__ u, const long long *__restrict__ off,
                              int nrec, float *__restrict__ row, int *err)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < nrec) {
        const float v = u[off[r]];
        row[r] = v;
        if (!isfinite(v)) atomicOr(err, 2);
    }
}

// 16-bit (or fp32) field -> fp32 compact, times the field's scale (null: 1).
template <class T>
__global__ void unpack_t_kernel(PadGeom g, const T *__restrict__ src, const float *scale,
                                float *__restrict__ dst)
{
    const float s = scale ? *scale : 1.0f;
    const long long n = (long long)g.Nx * g.Ny * g.Nz;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) {
        const long long i = c % g.Nx, t = c / g.Nx;
        const long long j = t % g.Ny, k = t / g.Ny;
        dst[c] = (float)src[g.origin + k * g.sxy + j * g.sx + i] * s;
    }
}

template <class T>
__global__ void gather_t_kernel(const T *__restrict__ u, const long long *__restrict__ off, int nrec,
                                const float *scale, float *__restrict__ row, int *err)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < nrec) {
        const float v = (float)u[off[r]] * (scale ? *scale : 1.0f);
        row[r] = v;
        if (!isfinite(v)) atomicOr(err, 2);
    }
}

__global__ void advance_kernel(int *counter, int by)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *counter += by;
}

}  // namespace sgb
