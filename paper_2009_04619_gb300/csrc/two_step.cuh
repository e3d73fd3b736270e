// Two time steps per HBM pass on the PML-free interior (temporal blocking).
//
// The paper names reintegrating the boundary with the inner region, so that
// time steps can be blocked (3.5D blocking, section II), as future work
// (section VI).  This kernel does the blocking on the part of the grid where
// no PML arithmetic is needed: a box B inside the inner region, shrunk by the
// stencil radius on every side, so that the first step can be evaluated on the
// box plus a radius-4 halo with Eq. 2 alone.  One work unit = a BX x BY tile of
// B's x-y extent x a z-chunk of B:
//
//   step 1: u^{n+1} = 2 u^n - u^{n-1} + m L u^n on the tile plus a 4-point x-y
//           halo (EX x EY points) and on 4 planes below and above the chunk,
//           from u^n with an 8-point halo (TMA boxes) and u^{n-1}, m on the
//           extended tile;
//   step 2: u^{n+2} = 2 u^{n+1} - u^n + m L u^{n+1} on the tile: z-neighbours
//           of u^{n+1} from a register queue filled by the thread's own step-1
//           results, x-y neighbours from a shared-memory ring of u^{n+1} planes,
//           u^n from the step-1 queue, m from the step-1 tile ring.
//
// Both outputs go to fresh buffers (u^{n+1} and u^{n+2} on the tile): writing
// them over u^{n-1} or u^n would race with neighbouring tiles that read those
// fields in their halos.  Points of the grid outside B (the PML and an inner
// band next to it) take two ordinary fused steps (shell launches of the
// single-step kernel), after which all of u^{n+1} and u^{n+2} are complete.
//
// The per-point arithmetic is the interior path of the single-step kernel,
// operation for operation (same coefficient order, packed FMAs split the same
// way, explicit roundings), so a temporally blocked shot reproduces the
// single-step shot bit for bit.
#pragma once
#include "step_kernel.cuh"

namespace sgb {

struct TwoStepArgs {
    float *out1;           // padded base of u^{n+1}
    float *out2;           // padded base of u^{n+2}
    int Nx, Ny, Nz;        // computed extents
    long long sx, sxy;     // element strides of y and z
    long long origin;      // element offset of computed (0, 0, 0)
    float c0;              // centre coefficient of Eq. 3
    float cx[4], cy[4], cz[4];
    int bx0, bx1, by0, by1, bz0, bz1;  // the box B (computed coordinates)
    int tiles_x, tiles_y, zc;
    int si, sj, sk;        // source point (sk < 0: none)
    const float *wavelet;
    float inv_vol;
    const int *step_ptr;   // device step counter (graph replays) or null
    int step_add;          // n = *step_ptr + step_add: the pair's first step
    int *err;              // device error word
};

template <int BX_, int BY_, int NU_, int NP_, int NW_>
struct TwoCfg {
    static constexpr int BX = BX_, BY = BY_;          // output tile
    static constexpr int EX = BX + 2 * R, EY = BY + 2 * R;  // step-1 region
    static constexpr int TXT = EX / 4, TYT = EY;      // one quad per consumer thread
    static constexpr int THREADS = TXT * TYT, WARPS = THREADS / 32, BLOCK = THREADS + 32;
    static constexpr int UW = EX + 2 * R, UH = EY + 2 * R;  // u^n box (8-point halo)
    static constexpr int NU = NU_, NP = NP_, NW = NW_;
    static constexpr int U_BYTES = UW * UH * 4;
    static constexpr int E_BYTES = EX * EY * 4;       // one extended fp32 tile
    static constexpr int P_BYTES = 2 * E_BYTES;       // u^{n-1}, m
    static constexpr int W_BYTES = E_BYTES;           // one u^{n+1} plane
    static constexpr size_t SMEM_BYTES = size_t(NU) * U_BYTES + size_t(NP) * P_BYTES +
                                         size_t(NW) * W_BYTES +
                                         size_t(2 * (NU + NP + NW)) * 8 + size_t(NU + NP + 1) * 4;
    // step-2 warps: those whose rows lie in the tile (rows R .. R + BY - 1)
    static constexpr int W2_FIRST = R * TXT / 32, W2_COUNT = BY * TXT / 32;
    static_assert(EX % 4 == 0 && TXT == 16, "a warp covers two rows of 16 quads");
    static_assert((R * TXT) % 32 == 0 && (BY * TXT) % 32 == 0, "step-2 rows are whole warps");
    static_assert(U_BYTES % 128 == 0 && E_BYTES % 128 == 0, "stage alignment");
    static_assert(UW <= 256 && UH <= 256, "TMA box limits");
    static_assert(NU >= 8 && NP >= 6 && NW >= 5, "ring depths");
};

template <class C>
struct TwoStepCta {
    static constexpr uint64_t WAIT_NS = 2000000000ull;
    const TwoStepArgs *pa;
    unsigned char *su, *sp, *sw;
    uint64_t *full_u, *empty_u, *full_p, *empty_p, *full_w, *empty_w;
    int *lastf_u, *lastf_p, *s_abort;
    int x0, y0, z0, z1;
    bool aborted;

    // Bounded wait that also gives up as soon as another warp of the CTA has.
    __device__ __forceinline__ void wait(uint64_t *bar, uint32_t parity)
    {
        if (mbar_try_wait(bar, parity)) return;
        const uint64_t t0 = global_timer_ns();
        for (;;) {
#pragma unroll 1
            for (int i = 0; i < 32; ++i)
                if (mbar_try_wait(bar, parity)) return;
            if (*reinterpret_cast<volatile int *>(s_abort) ||
                global_timer_ns() - t0 > WAIT_NS) {
                *reinterpret_cast<volatile int *>(s_abort) = 1;
                atomicOr(pa->err, DEV_ERR_TIMEOUT);
                return;
            }
        }
    }

    // Producer lane: u^n planes z0-8 .. z1+7 (8-point halo boxes) and (u^{n-1},
    // m) planes z0-4 .. z1+3 (extended tiles), in the order the consumers need
    // them; every refill first waits for its slot to be released; then waits for
    // its own copies, so none is in flight when the CTA exits.
    __device__ __forceinline__ void produce(const CUtensorMap *tm_u, const CUtensorMap *tm_up,
                                            const CUtensorMap *tm_m)
    {
        int nu = z0 - 2 * R, np = z0 - R;
        while ((nu < z1 + 2 * R || np < z1 + R) && !aborted) {
            // u plane nu is first needed at iteration nu - z0 (as the front
            // plane), (u^{n-1}, m) plane np at iteration np - z0 + 4
            const bool do_u = nu < z1 + 2 * R && (np >= z1 + R || nu <= np + R);
            if (do_u) {
                const int rel = nu - (z0 - 2 * R), s = rel % C::NU, f = rel / C::NU;
                if (f > 0) wait(empty_u + s, (f - 1) & 1);
                lastf_u[s] = f;
                mbar_arrive_expect_tx(full_u + s, C::U_BYTES);
                tma_load_3d(su + s * C::U_BYTES, tm_u, full_u + s, x0 - 2 * R, y0 - 2 * R, nu);
                ++nu;
            } else {
                const int rel = np - (z0 - R), s = rel % C::NP, f = rel / C::NP;
                if (f > 0) wait(empty_p + s, (f - 1) & 1);
                lastf_p[s] = f;
                mbar_arrive_expect_tx(full_p + s, C::P_BYTES);
                unsigned char *d = sp + s * C::P_BYTES;
                tma_load_3d(d, tm_up, full_p + s, x0 - R, y0 - R, np);
                tma_load_3d(d + C::E_BYTES, tm_m, full_p + s, x0 - R, y0 - R, np);
                ++np;
            }
            aborted = *reinterpret_cast<volatile int *>(s_abort) != 0;
        }
        for (int s = 0; s < C::NU; ++s)
            if (lastf_u[s] >= 0) mbar_wait_bounded(full_u + s, lastf_u[s] & 1, WAIT_NS);
        for (int s = 0; s < C::NP; ++s)
            if (lastf_p[s] >= 0) mbar_wait_bounded(full_p + s, lastf_p[s] & 1, WAIT_NS);
    }
};

// 25-point Laplacian of one quad in the interior path's operation order:
// centre, z pairs (m = 1..4), y terms (m = 4..1 below, then 1..4 above), then
// per point the x pairs.  q: z-queue with the centre at q[4]; rows(d): the quad
// d rows away in the same plane (d = -4 .. 4, d != 0); lf, rt: the quads left
// and right of the centre quad.
template <class RowFn>
__device__ __forceinline__ float4 lap_quad(const TwoStepArgs &a, const float4 (&q)[9], RowFn rows,
                                           const float4 &lf, const float4 &rt)
{
    float4 L = f4mul(a.c0, q[4]);
#pragma unroll
    for (int m = 1; m <= R; ++m) {
        f4fma(L, a.cz[m - 1], q[4 - m]);
        f4fma(L, a.cz[m - 1], q[4 + m]);
    }
#pragma unroll
    for (int d = -R; d <= R; ++d) {
        if (d == 0) continue;
        const int m = d > 0 ? d : -d;
        f4fma(L, a.cy[m - 1], rows(d));
    }
    const float4 c = q[4];
    const float w[12] = {lf.x, lf.y, lf.z, lf.w, c.x, c.y, c.z, c.w, rt.x, rt.y, rt.z, rt.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        float s = f4get(L, e);
#pragma unroll
        for (int m = 1; m <= R; ++m) {
            s = fmaf(a.cx[m - 1], w[4 + e - m], s);
            s = fmaf(a.cx[m - 1], w[4 + e + m], s);
        }
        f4set(L, e, s);
    }
    return L;
}

template <class C>
__global__ void __launch_bounds__(C::BLOCK, 1)
    two_step_kernel(const __grid_constant__ TwoStepArgs a, const __grid_constant__ CUtensorMap tm_u,
                    const __grid_constant__ CUtensorMap tm_up, const __grid_constant__ CUtensorMap tm_m)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TwoStepCta<C> st;
    st.pa = &a;
    st.su = smem_raw;
    st.sp = st.su + C::NU * C::U_BYTES;
    st.sw = st.sp + C::NP * C::P_BYTES;
    st.full_u = reinterpret_cast<uint64_t *>(st.sw + C::NW * C::W_BYTES);
    st.empty_u = st.full_u + C::NU;
    st.full_p = st.empty_u + C::NU;
    st.empty_p = st.full_p + C::NP;
    st.full_w = st.empty_p + C::NP;
    st.empty_w = st.full_w + C::NW;
    st.lastf_u = reinterpret_cast<int *>(st.empty_w + C::NW);
    st.lastf_p = st.lastf_u + C::NU;
    st.s_abort = st.lastf_p + C::NP;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per_chunk = a.tiles_x * a.tiles_y;
    const int chunk = blockIdx.x / per_chunk;
    const int trem = blockIdx.x - chunk * per_chunk;
    const int tyl = trem / a.tiles_x, txl = trem - tyl * a.tiles_x;
    st.x0 = a.bx0 + txl * C::BX;
    st.y0 = a.by0 + tyl * C::BY;
    st.z0 = a.bz0 + chunk * a.zc;
    st.z1 = min(st.z0 + a.zc, a.bz1);
    st.aborted = false;
    const int n = (a.step_ptr ? *a.step_ptr : 0) + a.step_add;

    if (tid == C::THREADS) {
        *st.s_abort = (*reinterpret_cast<volatile int *>(a.err) & DEV_ERR_TIMEOUT) ? 1 : 0;
        for (int i = 0; i < C::NU; ++i) {
            mbar_init(st.full_u + i, 1);
            mbar_init(st.empty_u + i, C::WARPS);
            st.lastf_u[i] = -1;
        }
        for (int i = 0; i < C::NP; ++i) {
            mbar_init(st.full_p + i, 1);
            mbar_init(st.empty_p + i, C::WARPS);
            st.lastf_p[i] = -1;
        }
        for (int i = 0; i < C::NW; ++i) {
            mbar_init(st.full_w + i, C::WARPS);
            mbar_init(st.empty_w + i, C::W2_COUNT);
        }
        fence_barrier_init();
    }
    __syncthreads();
    st.aborted = *reinterpret_cast<volatile int *>(st.s_abort) != 0;
    if (st.z1 <= st.z0 || st.aborted) return;

    if (tid >= C::THREADS) {  // producer warp: one lane issues every copy
        if (tid == C::THREADS) st.produce(&tm_u, &tm_up, &tm_m);
        return;
    }

    const int txi = tid % C::TXT, tyi = tid / C::TXT;
    const bool w2 = warp >= C::W2_FIRST && warp < C::W2_FIRST + C::W2_COUNT;  // step-2 warp
    const int gx = st.x0 - R + 4 * txi, gy = st.y0 - R + tyi;  // this thread's quad
    // step-2 outputs: tile quads inside B
    const bool own2 = w2 && txi >= 1 && txi < C::TXT - 1 && gx < a.bx1 && gy < a.by1;
    const int ucol = R + 4 * txi, urow = R + tyi;      // quad in the u^n box
    const int eoff = tyi * C::EX + 4 * txi;             // quad in an extended tile
    const long long goff0 = a.origin + (long long)gy * a.sx + gx;
    const bool src_here = a.sk >= 0 && gy == a.sj && a.si >= gx && a.si < gx + 4;
    const int src_e = a.si - gx;
    const float f1 = src_here ? a.wavelet[n] * a.inv_vol : 0.0f;
    const float f2 = src_here ? a.wavelet[n + 1] * a.inv_vol : 0.0f;

    auto ubox = [&](int s) { return reinterpret_cast<const float *>(st.su + s * C::U_BYTES); };

    // prime the step-1 queue with u^n planes z0-8 .. z0-1 (slots 0..7)
    float4 q1[9], q2[9];
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        st.wait(st.full_u + s, 0);
        q1[s] = lds128(ubox(s) + urow * C::UW + ucol);
    }
    // planes z0-8 .. z0-5 only prime the queue
    __syncwarp();
    if (lane == 0)
        for (int s = 0; s < 4; ++s) mbar_arrive(st.empty_u + s);
#pragma unroll
    for (int s = 0; s < 9; ++s) q2[s] = make_float4(0.f, 0.f, 0.f, 0.f);

    const int nit = st.z1 - st.z0 + 2 * R;
    for (int it = 0; it < nit && !st.aborted; ++it) {
        const int p = st.z0 - R + it;  // step-1 plane
        // front plane p + 4 of u^n into the queue
        const int sf = (it + 8) % C::NU;
        st.wait(st.full_u + sf, ((it + 8) / C::NU) & 1);
        q1[8] = lds128(ubox(sf) + urow * C::UW + ucol);
        const int sq = it % C::NP;  // (u^{n-1}, m) of plane p
        st.wait(st.full_p + sq, (it / C::NP) & 1);
        const float *cu = ubox((it + 4) % C::NU);
        const float *pe = reinterpret_cast<const float *>(st.sp + sq * C::P_BYTES);

        // step 1 at (quad, p)
        float4 un;
        {
            const float *rowp = cu + urow * C::UW + ucol;
            const float4 L = lap_quad(a, q1, [&](int d) { return lds128(rowp + d * C::UW); },
                                      lds128(rowp - 4), lds128(rowp + 4));
            const float4 c = q1[4], up = lds128(pe + eoff), mm = lds128(pe + C::E_BYTES / 4 + eoff);
            un.x = fmaf(mm.x, L.x, fmaf(2.0f, c.x, -up.x));
            un.y = fmaf(mm.y, L.y, fmaf(2.0f, c.y, -up.y));
            un.z = fmaf(mm.z, L.z, fmaf(2.0f, c.z, -up.z));
            un.w = fmaf(mm.w, L.w, fmaf(2.0f, c.w, -up.w));
            if (src_here && p == a.sk) f4set(un, src_e, fmaf(f4get(mm, src_e), f1, f4get(un, src_e)));
        }
        const bool in_chunk = p >= st.z0 && p < st.z1;
        if (in_chunk) {
            // u^{n+1} plane p into the ring (x-y neighbours of step 2) and, on
            // the tile, to global memory
            const int wr = p - st.z0, ws = wr % C::NW;
            if (wr >= C::NW) st.wait(st.empty_w + ws, ((wr / C::NW) - 1) & 1);
            *reinterpret_cast<float4 *>(st.sw + ws * C::W_BYTES + eoff * 4) = un;
            if (own2) stg128(a.out1 + goff0 + (long long)p * a.sxy, un);
            __syncwarp();
            if (lane == 0) mbar_arrive(st.full_w + ws);
        }
        q2[8] = un;
        // release the centre u^n plane; the (u^{n-1}, m) slot waits for step 2
        // where step 2 will use its m
        __syncwarp();
        if (lane == 0) {
            mbar_arrive(st.empty_u + (it + 4) % C::NU);
            if (!(w2 && in_chunk)) mbar_arrive(st.empty_p + sq);
        }

        // step 2 at (quad, q = p - 4)
        if (w2 && it >= 2 * R) {
            const int q = p - R, wr = q - st.z0, ws = wr % C::NW;
            st.wait(st.full_w + ws, (wr / C::NW) & 1);
            const float *wp = reinterpret_cast<const float *>(st.sw + ws * C::W_BYTES) + eoff;
            const float4 L = lap_quad(a, q2, [&](int d) { return lds128(wp + d * C::EX); },
                                      lds128(wp - 4), lds128(wp + 4));
            const int sq2 = (it - R) % C::NP;
            const float4 c = q2[4], up = q1[0];
            const float4 mm = lds128(reinterpret_cast<const float *>(st.sp + sq2 * C::P_BYTES) +
                                     C::E_BYTES / 4 + eoff);
            float4 u2;
            u2.x = fmaf(mm.x, L.x, fmaf(2.0f, c.x, -up.x));
            u2.y = fmaf(mm.y, L.y, fmaf(2.0f, c.y, -up.y));
            u2.z = fmaf(mm.z, L.z, fmaf(2.0f, c.z, -up.z));
            u2.w = fmaf(mm.w, L.w, fmaf(2.0f, c.w, -up.w));
            if (src_here && q == a.sk) f4set(u2, src_e, fmaf(f4get(mm, src_e), f2, f4get(u2, src_e)));
            if (own2) stg128(a.out2 + goff0 + (long long)q * a.sxy, u2);
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(st.empty_w + ws);
                mbar_arrive(st.empty_p + sq2);
            }
        }
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            q1[s] = q1[s + 1];
            q2[s] = q2[s + 1];
        }
        st.aborted = *reinterpret_cast<volatile int *>(st.s_abort) != 0;
    }
}

}  // namespace sgb
