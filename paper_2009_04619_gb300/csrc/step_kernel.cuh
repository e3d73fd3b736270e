// Fused 25-point wave step with in-launch PML, FP32 storage (sm_103a).
//
// What it computes (arXiv 2009.04619, section III-A): one leapfrog step of
// Eq. 2, u^{n+1} = 2u^n - u^{n-1} + m L u^n with m = V^2 dt^2 and L the
// 25-point star Laplacian of Eq. 3, at every computed point of the inner
// region; a PML update at the points outside it (the paper names a PML and a
// 7-point stencil on an eta array but prints no formulas; the reading used
// is the single-stretch PML
//     u^{n+1} (1 + e) = (2 - e^2) u^n - (1 - e) u^{n-1} + m (L u^n + phi^n)
//     phi^{n+1} (1 + e) = phi^n - dt grad(eta) . grad(u^n)
// with e = eta dt, eta = eta_x(i) + eta_y(j) + eta_z(k), eta_a = eta_max
// (d_a / nb)^2 and 2nd-order central differences for both gradients); the
// point source of Eq. 2's right-hand side (Algorithm 1).
//
// How (a GB300 design; the paper's 2.5D register-streaming kernels of
// section IV are the starting idea, not the blueprint):
//  - one CTA owns a BX x BY tile of the x-y plane and streams a chunk of z
//    (2.5D blocking);
//  - planes of u^n arrive by TMA, with their radius-4 x-y halo, into an
//    NU-stage shared-memory ring; u^{n-1}, m and (PML planes only) phi tiles
//    into an NP-stage ring; one elected thread issues the copies, mbarriers
//    carry completion, so several planes are always in flight;
//  - each thread owns 4 consecutive x points (128-bit accesses) in TY rows;
//    the z-neighbours of its points sit in a 9-deep register queue whose
//    rotation is resolved at compile time by unrolling the z loop 9 times
//    (the fixed-register idea of the paper's st_reg_fixed kernels);
//  - whether a plane takes the PML path depends only on the tile and k, so
//    the branch is uniform across the CTA; inside a PML-path plane, inner
//    points select the Eq. 2 result computed by the same instructions as the
//    inner path, bit for bit;
//  - eta and its central differences are evaluated in closed form from the
//    integer depth into the layer: no eta array is read;
//  - every mbarrier wait is bounded (2 s); on timeout the CTA records
//    DEV_ERR_TIMEOUT, drains its own copies (bounded) and exits.
#pragma once
#include "ptx.cuh"

namespace sgb {

constexpr int R = 4;          // stencil radius (half the spatial order)
constexpr int HALO_LO_X = 8;  // zero points before computed x = 0 (16-byte aligned origin)
constexpr int HALO = 4;       // zero points before y = 0, z = 0 and after every axis

enum : int { DEV_ERR_TIMEOUT = 1, DEV_ERR_NONFINITE = 2, DEV_ERR_RANGE = 4 };

struct StepArgs {
    float *u_out;          // padded base: holds u^{n-1} on entry, u^{n+1} on exit
    const float *u_cur;    // padded base of u^n (receiver pre-sampling only)
    float *phi;            // padded base of phi (PML auxiliary field)
    int Nx, Ny, Nz;        // computed extents
    int nb, nx, ny, nz;    // PML width, inner extents
    long long sx, sxy;     // element strides of y and z
    long long origin;      // element offset of computed (0, 0, 0)
    float c0;              // centre coefficient of Eq. 3
    float cx[4], cy[4], cz[4];
    float ax, ay, az;      // eta_a dt = a * d^2
    float kx, ky, kz;      // dt d(eta)/da d(u)/da = k (d(+1)^2 - d(-1)^2) (u(+1) - u(-1))
    int si, sj, sk;        // source point (sk < 0: none)
    const float *wavelet;  // w(n dt) samples
    float inv_vol;         // 1 / (dx dy dz)
    const int *step_ptr;   // device step counter (graph replays) or null
    int step_add;          // n = *step_ptr + step_add
    int nrec;              // receivers sampled from u^n into row n - 1 (n >= 1)
    const long long *rec_off;
    float *traces;
    int *err;              // device error word
    int tiles_x, tiles_y, zc;
};

template <int TXT_, int TYT_, int TY_, int NU_, int NP_, int MINB_>
struct TileCfg {
    static constexpr int TXT = TXT_, TYT = TYT_, TY = TY_, NU = NU_, NP = NP_, MINB = MINB_;
    static constexpr int THREADS = TXT * TYT;
    static constexpr int BX = 4 * TXT, BY = TY * TYT;
    static constexpr int HX = 4;  // x margin of the u^n box: 16 bytes keeps TMA x aligned
    static constexpr int SW = BX + 2 * HX;
    static constexpr int SH = BY + 2 * R;
    static constexpr int U_STAGE = SW * SH;
    static constexpr int P_TILE = BX * BY;
    static constexpr int P_STAGE = 3 * P_TILE;
    static constexpr size_t SMEM_BYTES =
        size_t(NU * U_STAGE + NP * P_STAGE) * 4 + size_t(NU + NP) * 8 + size_t(NU + NP + 1) * 4;
    static_assert(NU >= 8, "the u ring must hold the 8 planes that prime the register queue");
    static_assert((U_STAGE * 4) % 128 == 0 && (P_TILE * 4) % 128 == 0, "stage alignment");
    static_assert(SW <= 256 && SH <= 256 && BX <= 256 && BY <= 256, "TMA box limits");
};

// Depth (points) of index i into the PML along one axis; 0 in the inner range.
__device__ __forceinline__ int pml_depth(int n_inner, int nb, int i)
{
    return max(max(nb - i, i - (nb + n_inner - 1)), 0);
}

__device__ __forceinline__ float interior_update(float c, float up, float mm, float L)
{
    return fmaf(mm, L, fmaf(2.0f, c, -up));
}

__device__ __forceinline__ float f4get(const float4 &v, int e)
{
    return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w;
}
__device__ __forceinline__ void f4set(float4 &v, int e, float s)
{
    if (e == 0) v.x = s;
    else if (e == 1) v.y = s;
    else if (e == 2) v.z = s;
    else v.w = s;
}
__device__ __forceinline__ void f4fma(float4 &acc, float c, const float4 &v)
{
    acc.x = fmaf(c, v.x, acc.x);
    acc.y = fmaf(c, v.y, acc.y);
    acc.z = fmaf(c, v.z, acc.z);
    acc.w = fmaf(c, v.w, acc.w);
}

template <class C>
__global__ void __launch_bounds__(C::THREADS, C::MINB)
    fused_step_kernel(const StepArgs a, const __grid_constant__ CUtensorMap tm_ucur,
                      const __grid_constant__ CUtensorMap tm_uprev,
                      const __grid_constant__ CUtensorMap tm_m,
                      const __grid_constant__ CUtensorMap tm_phi)
{
    constexpr int TXT = C::TXT, TY = C::TY, NU = C::NU, NP = C::NP, THREADS = C::THREADS;
    constexpr int BX = C::BX, BY = C::BY, HX = C::HX, SW = C::SW;
    constexpr int U_STAGE = C::U_STAGE, P_TILE = C::P_TILE, P_STAGE = C::P_STAGE;
    constexpr uint64_t WAIT_NS = 2000000000ull;

    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *su = reinterpret_cast<float *>(smem_raw);
    float *sp = su + NU * U_STAGE;
    uint64_t *bar_u = reinterpret_cast<uint64_t *>(sp + NP * P_STAGE);
    uint64_t *bar_p = bar_u + NU;
    int *lastf_u = reinterpret_cast<int *>(bar_p + NP);
    int *lastf_p = lastf_u + NU;
    int &s_abort = lastf_p[NP];  // kept in the dynamic region: no static shared memory,
                                 // so the TMA destinations start at the aligned base

    const int tid = threadIdx.x;
    const int txi = tid % TXT, tyi = tid / TXT;

    // Work unit: chunk-major so that CTAs running together share z and their
    // x-y halos meet in L2.
    const int per_chunk = a.tiles_x * a.tiles_y;
    const int chunk = blockIdx.x / per_chunk;
    const int trem = blockIdx.x - chunk * per_chunk;
    const int tyl = trem / a.tiles_x, txl = trem - tyl * a.tiles_x;
    const int x0 = txl * BX, y0 = tyl * BY;
    const int z0 = chunk * a.zc;
    const int z1 = min(z0 + a.zc, a.Nz);
    const int nit = z1 - z0;
    const int n = (a.step_ptr ? *a.step_ptr : 0) + a.step_add;

    // Receivers of the previous step: u^n is read-only in this launch.
    if (a.nrec > 0 && n >= 1) {
        for (int r = blockIdx.x * THREADS + tid; r < a.nrec; r += gridDim.x * THREADS) {
            const float v = a.u_cur[a.rec_off[r]];
            a.traces[(long long)(n - 1) * a.nrec + r] = v;
            if (!isfinite(v)) atomicOr(a.err, DEV_ERR_NONFINITE);
        }
    }

    const int xe = min(x0 + BX, a.Nx), ye = min(y0 + BY, a.Ny);
    const bool xy_inner = x0 >= a.nb && xe <= a.nb + a.nx && y0 >= a.nb && ye <= a.nb + a.ny;

    if (tid == 0) {
        s_abort = 0;
        for (int i = 0; i < NU; ++i) {
            mbar_init(bar_u + i, 1);
            lastf_u[i] = -1;
        }
        for (int i = 0; i < NP; ++i) {
            mbar_init(bar_p + i, 1);
            lastf_p[i] = -1;
        }
        fence_barrier_init();
    }
    __syncthreads();
    if (nit <= 0) return;

    auto plane_pml = [&](int k) { return !xy_inner || k < a.nb || k >= a.nb + a.nz; };
    auto issue_u = [&](int p) {
        const int rel = p - z0 + 4;
        const int s = rel % NU;
        lastf_u[s] = rel / NU;
        mbar_arrive_expect_tx(bar_u + s, U_STAGE * 4);
        tma_load_3d(su + s * U_STAGE, &tm_ucur, bar_u + s, x0 - HX, y0 - R, p);
    };
    auto issue_p = [&](int k) {
        const int rel = k - z0;
        const int s = rel % NP;
        lastf_p[s] = rel / NP;
        const bool pml = plane_pml(k);
        const uint64_t pol = policy_evict_first();
        mbar_arrive_expect_tx(bar_p + s, (pml ? 3 : 2) * P_TILE * 4);
        float *d = sp + s * P_STAGE;
        tma_load_3d_hint(d, &tm_uprev, bar_p + s, x0, y0, k, pol);
        tma_load_3d_hint(d + P_TILE, &tm_m, bar_p + s, x0, y0, k, pol);
        if (pml) tma_load_3d_hint(d + 2 * P_TILE, &tm_phi, bar_p + s, x0, y0, k, pol);
    };

    if (tid == 0) {
        for (int p = z0 - 4; p < z0 - 4 + NU && p < z1 + 4; ++p) issue_u(p);
        for (int k = z0; k < z0 + NP && k < z1; ++k) issue_p(k);
    }

    const int row0 = R + TY * tyi;  // first own row inside a u stage
    const int colu = HX + 4 * txi;  // own column inside a u stage
    const int gi = x0 + 4 * txi;    // first own x
    const int gj0 = y0 + TY * tyi;  // first own y

    // Prime the register queue with planes z0-4 .. z0+3.
    float4 q[TY][9];
    bool ok = true;
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        ok &= mbar_wait_bounded(bar_u + s, 0, WAIT_NS);
#pragma unroll
        for (int r = 0; r < TY; ++r) q[r][s] = lds128(su + s * U_STAGE + (row0 + r) * SW + colu);
    }
    if (!ok) {
        s_abort = 1;
        atomicOr(a.err, DEV_ERR_TIMEOUT);
    }
    __syncthreads();
    if (tid == 0 && !s_abort)
        for (int p = z0 - 4; p < z0; ++p)
            if (p + NU < z1 + 4) issue_u(p + NU);

    bool aborted = s_abort != 0;
    for (int it0 = 0; it0 < nit && !aborted; it0 += 9) {
#pragma unroll
        for (int rr = 0; rr < 9; ++rr) {
            const int it = it0 + rr;
            if (it >= nit) break;
            const int k = z0 + it;
            // Front plane k + 4 enters the queue.
            {
                const int rel = it + 8;
                const int s = rel % NU;
                if (!mbar_wait_bounded(bar_u + s, (rel / NU) & 1, WAIT_NS)) {
                    s_abort = 1;
                    atomicOr(a.err, DEV_ERR_TIMEOUT);
                }
#pragma unroll
                for (int r = 0; r < TY; ++r)
                    q[r][(rr + 8) % 9] = lds128(su + s * U_STAGE + (row0 + r) * SW + colu);
            }
            const int sq = it % NP;
            if (!mbar_wait_bounded(bar_p + sq, (it / NP) & 1, WAIT_NS)) {
                s_abort = 1;
                atomicOr(a.err, DEV_ERR_TIMEOUT);
            }
            const float *cu = su + ((it + 4) % NU) * U_STAGE;
            const float *pu = sp + sq * P_STAGE;
            const bool pml = plane_pml(k);

            // 25-point Laplacian (Eq. 3) of the TY x 4 own points.
            float4 L[TY], gy[TY];
#pragma unroll
            for (int r = 0; r < TY; ++r) {
                const float4 c = q[r][(rr + 4) % 9];
                L[r] = make_float4(a.c0 * c.x, a.c0 * c.y, a.c0 * c.z, a.c0 * c.w);
                gy[r] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int m = 1; m <= R; ++m) {
                    f4fma(L[r], a.cz[m - 1], q[r][(rr + 4 - m + 9) % 9]);
                    f4fma(L[r], a.cz[m - 1], q[r][(rr + 4 + m) % 9]);
                }
            }
            // y neighbours: rows -4 .. TY+3 relative to the first own row.
#pragma unroll
            for (int d = -R; d < TY + R; ++d) {
                float4 v;
                if (d >= 0 && d < TY) v = q[d][(rr + 4) % 9];
                else v = lds128(cu + (row0 + d) * SW + colu);
#pragma unroll
                for (int r = 0; r < TY; ++r) {
                    const int m = d > r ? d - r : r - d;
                    if (m >= 1 && m <= R) f4fma(L[r], a.cy[m - 1], v);
                    if (d == r + 1) {
                        gy[r].x += v.x;
                        gy[r].y += v.y;
                        gy[r].z += v.z;
                        gy[r].w += v.w;
                    }
                    if (d == r - 1) {
                        gy[r].x -= v.x;
                        gy[r].y -= v.y;
                        gy[r].z -= v.z;
                        gy[r].w -= v.w;
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < TY; ++r) {
                const float *rowp = cu + (row0 + r) * SW + colu;
                const float4 c = q[r][(rr + 4) % 9];
                const float4 lf = lds128(rowp - 4), rt = lds128(rowp + 4);
                const float w[12] = {lf.x, lf.y, lf.z, lf.w, c.x, c.y, c.z, c.w,
                                     rt.x, rt.y, rt.z, rt.w};
                float4 Lr = L[r];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    float s = f4get(Lr, e);
#pragma unroll
                    for (int m = 1; m <= R; ++m) {
                        s = fmaf(a.cx[m - 1], w[4 + e - m], s);
                        s = fmaf(a.cx[m - 1], w[4 + e + m], s);
                    }
                    f4set(Lr, e, s);
                }
                const int prow = (TY * tyi + r) * BX + 4 * txi;
                const float4 up = lds128(pu + prow);
                const float4 mm = lds128(pu + P_TILE + prow);
                float4 un;
                un.x = interior_update(c.x, up.x, mm.x, Lr.x);
                un.y = interior_update(c.y, up.y, mm.y, Lr.y);
                un.z = interior_update(c.z, up.z, mm.z, Lr.z);
                un.w = interior_update(c.w, up.w, mm.w, Lr.w);
                const int j = gj0 + r;
                float4 phn;
                bool any_pml = false;
                if (pml) {
                    const float4 ph = lds128(pu + 2 * P_TILE + prow);
                    phn = ph;
                    const int dyj = pml_depth(a.ny, a.nb, j);
                    const int dyp = pml_depth(a.ny, a.nb, j + 1), dym = pml_depth(a.ny, a.nb, j - 1);
                    const int dzk = pml_depth(a.nz, a.nb, k);
                    const int dzp = pml_depth(a.nz, a.nb, k + 1), dzm = pml_depth(a.nz, a.nb, k - 1);
                    const float ey = a.ay * float(dyj * dyj) + a.az * float(dzk * dzk);
                    const float gyc = a.ky * float(dyp * dyp - dym * dym);
                    const float gzc = a.kz * float(dzp * dzp - dzm * dzm);
                    const float4 zp = q[r][(rr + 5) % 9], zm = q[r][(rr + 3) % 9];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int i = gi + e;
                        const int dxi = pml_depth(a.nx, a.nb, i);
                        const int dxp = pml_depth(a.nx, a.nb, i + 1), dxm = pml_depth(a.nx, a.nb, i - 1);
                        const bool pt = (dxi | dyj | dzk) != 0;
                        any_pml |= pt;
                        const float edt = fmaf(a.ax, float(dxi * dxi), ey);
                        const float G = a.kx * float(dxp * dxp - dxm * dxm) * (w[5 + e] - w[3 + e]) +
                                        gyc * f4get(gy[r], e) +
                                        gzc * (f4get(zp, e) - f4get(zm, e));
                        const float inv = 1.0f / (1.0f + edt);
                        const float cc = f4get(c, e), pe = f4get(ph, e);
                        const float upml =
                            ((2.0f - edt * edt) * cc - (1.0f - edt) * f4get(up, e) +
                             f4get(mm, e) * (f4get(Lr, e) + pe)) * inv;
                        const float ppml = (pe - G) * inv;
                        if (pt) {
                            f4set(un, e, upml);
                            f4set(phn, e, ppml);
                        }
                    }
                }
                // Point source (Eq. 2 right-hand side), added by the owning thread.
                if (k == a.sk && j == a.sj && a.si >= gi && a.si < gi + 4) {
                    const int e = a.si - gi;
                    f4set(un, e, f4get(un, e) + f4get(mm, e) * a.wavelet[n] * a.inv_vol);
                }
                if (j < a.Ny && gi < a.Nx) {
                    const long long off = a.origin + (long long)k * a.sxy + (long long)j * a.sx + gi;
                    if (gi + 3 < a.Nx) {
                        stg128(a.u_out + off, un);
                        if (any_pml) stg128(a.phi + off, phn);
                    } else {
                        for (int e = 0; e < 4 && gi + e < a.Nx; ++e) {
                            a.u_out[off + e] = f4get(un, e);
                            if (any_pml) a.phi[off + e] = f4get(phn, e);
                        }
                    }
                }
            }
            __syncthreads();
            aborted = s_abort != 0;
            if (aborted) break;
            if (tid == 0) {
                if (k + NU < z1 + 4) issue_u(k + NU);
                if (k + NP < z1) issue_p(k + NP);
            }
        }
    }
    if (aborted && tid == 0) {
        // Drain this CTA's own copies still in flight (bounded) before exiting.
        for (int s = 0; s < NU; ++s)
            if (lastf_u[s] >= 0) mbar_wait_bounded(bar_u + s, lastf_u[s] & 1, WAIT_NS);
        for (int s = 0; s < NP; ++s)
            if (lastf_p[s] >= 0) mbar_wait_bounded(bar_p + s, lastf_p[s] & 1, WAIT_NS);
    }
}

}  // namespace sgb
