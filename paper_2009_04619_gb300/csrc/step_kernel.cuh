// Fused 25-point wave step with in-launch PML (sm_103a), templated on the
// wavefield storage type: fp32, fp16 with a per-field power-of-two scale, or
// bf16; the arithmetic is fp32 in every case.
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
//    NU-stage shared-memory ring (the 4 planes below and above a z-chunk are
//    only needed for the z-neighbours of the chunk's own points, so they come
//    without the halo, with an L2 evict-last hint for the neighbouring chunk
//    that reads them again); u^{n-1}, m and (PML planes only) phi tiles
//    into an NP-stage ring, with no evict-first hint because u^{n-1} and phi
//    are rewritten in place a few planes later; phi comes in 32-column blocks,
//    and a tile that touches only the x-PML loads only the blocks holding PML
//    columns outside the z-PML; one lane of a dedicated producer warp issues the
//    copies in the order the consumers need them, as far ahead as the rings
//    allow; "full" mbarriers carry copy completion to the consumer warps and
//    "empty" mbarriers (one arrival per consumer warp) carry slot release back
//    to the producer, so there is no block-wide barrier in the z loop;
//  - each thread owns 4 consecutive x points (128-bit accesses) in TY rows;
//    the z-neighbours of its points sit in a register queue (the paper's
//    register-streaming idea, section IV); the z loop is unrolled U times with
//    compile-time queue offsets and the queue shifts by U once per group, so
//    there are 8 register moves per U planes.  Full 9-fold unrolling (the
//    paper's st_reg_fixed form, no moves at all) measured slower on GB300:
//    its code no longer fits the instruction cache;
//  - whether a plane takes the PML path depends only on the tile and k, so
//    the branch is uniform across the CTA: the z range of a tile splits into
//    segments of three plane kinds (interior; PML path outside the z-PML, where
//    1/(1+e) and 1-e come from per-thread tables; z-PML), each a separately
//    compiled loop, which keeps the hot interior loop small enough for the
//    instruction cache; inside a PML-path plane, inner points select the Eq. 2
//    result computed by the same instructions as the interior path, bit for bit;
//  - eta and its central differences are evaluated in closed form from the
//    integer depth into the layer: no eta array is read;
//  - every mbarrier wait is bounded (2 s); on timeout the CTA records
//    DEV_ERR_TIMEOUT, drains its own copies (bounded) and exits;
//  - 16-bit storage keeps only the two wavefields in 16 bits (m and phi stay
//    fp32).  The Laplacian is accumulated on the stored values and multiplied
//    by the field's scale once.  The fp16 scale of u^{n+1} is a power of two
//    chosen in the kernel from max|u^n|, max|u^{n-1}| and the injected
//    amplitude, so that |u^{n+1}| / scale < 2^14 (fp16 max 65504); every CTA
//    also contributes max|u^{n+1}| (warp max + atomicMax) for the next step.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ptx.cuh"

namespace sgb {

constexpr int R = 4;          // stencil radius (half the spatial order)
constexpr int HALO_LO_X = 8;  // zero points before computed x = 0 (16-byte aligned origin)
constexpr int HALO = 4;       // zero points before y = 0, z = 0 and after every axis

enum : int { DEV_ERR_TIMEOUT = 1, DEV_ERR_NONFINITE = 2, DEV_ERR_RANGE = 4 };

// Kernel modes: the forward step; the forward step that also stores its
// acceleration term g^n = L u^n + phi^n + f^n (recomputation for the adjoint);
// the adjoint step (see adjoint notes below).
// MODE_DIFF: the forward step in difference form. The state is (u^n, d^n) with
// d^n = u^n - u^{n-1} instead of (u^n, u^{n-1}): the same scheme in exact
// arithmetic, but a rounding error stored in u no longer also enters the time
// difference, so stored 16-bit values lose far less (each field keeps its own
// relative precision). d is read through the u^{n-1} tile map and updated in
// place through d_io; u^{n+1} goes to u_out.
enum : int { MODE_FWD = 0, MODE_FWD_ACC = 1, MODE_ADJ = 2, MODE_DIFF = 3 };

// Plane kinds of a work unit (compile-time paths of the plane body).
enum : int { PLANE_INTERIOR = 0, PLANE_XY = 1, PLANE_Z = 2 };

// Scale state of a 16-bit wavefield pair (device memory): s[k & 3] is the
// scale of u^k (stored value = u^k / s), mx[k & 3] is max |u^k|.
struct ScaleState {
    float s[4];
    float mx[4];
};

struct StepArgs {
    void *u_out;           // padded base: holds u^{n-1} on entry, u^{n+1} on exit
    void *d_io;            // MODE_DIFF: padded base of d^n on entry, d^{n+1} on exit
    const void *u_cur;     // padded base of u^n (receiver pre-sampling only)
    float *phi;            // padded base of phi (PML auxiliary field, fp32)
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
    const float *m_src;    // m at the source point (fp16 scale bound)
    float inv_vol;         // 1 / (dx dy dz)
    const int *step_ptr;   // device step counter (graph replays) or null
    int step_add;          // n = *step_ptr + step_add
    int nrec;              // receivers sampled from u^n into row n - 1 - rec_n0 (n > rec_n0)
    int rec_n0;            // first step of the traces buffer (a shot segment's first step)
    const long long *rec_off;
    float *traces;
    ScaleState *scale;     // fp16 storage only
    ScaleState *scale_d;   // fp16 storage in MODE_DIFF: scales and maxima of d
    float *acc_out;        // MODE_FWD_ACC: g = L u^n + phi^n + f^n (padded fp32)
    float *gsum;           // MODE_ADJ: fp32 partial sum of w^k g^{k-1} (padded)
    const float *mu_in;    // MODE_ADJ: mu^{k+1} (padded); phi is mu^k
    int *err;              // device error word
    int tiles_x, tiles_y, zc;
    // shell launches of a temporally blocked pair: work units (x0, y0, z0, z1)
    // from a table, and no store inside the box [bx0,bx1) x [by0,by1) x
    // [bz0,bz1), which the two-step kernel writes
    const int4 *units;
    int bx0, bx1, by0, by1, bz0, bz1;
};

// Counter-based hash (Murmur3 finaliser) of a point index and a step: the random
// bits of stochastic rounding, reproducible run to run.  One hash is drawn per
// thread and plane; the other 32-bit words that thread needs for the plane come
// from it by an odd multiply (a bijection of 2^32, so each word is uniform when
// the hash is, and its low half is a permutation of the hash's low half): see
// next_bits and Elem<T>::st.
__device__ __forceinline__ uint32_t hash_bits(uint32_t a, uint32_t b)
{
    uint32_t h = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u);
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

// Next random word of the same thread and plane (another row's quad).
__device__ __forceinline__ uint32_t next_bits(uint32_t h)
{
    return (h ^ (h >> 16)) * 0x45D9F3Bu;
}

// Stochastic rounding of an fp32 pair to 16 bits in the conversion itself
// (the cvt.rs form of sm_100-family GPUs, fed 32 random bits): each value
// rounds up with probability equal to its distance from the lower neighbour.
// With round-to-nearest, the rounding errors of a smooth field repeat from
// step to step and add up coherently over a run; stochastic rounding makes
// them uncorrelated (zero mean), so they grow like a random walk instead.
// The first source operand of the pair conversion lands in the upper half.
__device__ __forceinline__ uint32_t cvt_rs_f16x2(float lo, float hi, uint32_t rnd)
{
    uint32_t d;
    asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rnd));
    return d;
}

__device__ __forceinline__ uint32_t cvt_rs_bf16x2(float lo, float hi, uint32_t rnd)
{
    uint32_t d;
    asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rnd));
    return d;
}

// Storage traits: TMA x margin (16 bytes), 4-wide loads from shared memory and
// stores to global memory (rnd: random bits for stochastic rounding), scalar
// access.
template <class T>
struct Elem;

template <>
struct Elem<float> {
    static constexpr int HX = 4;
    static constexpr bool SCALED = false;
    __device__ static __forceinline__ float4 ld(const float *p) { return lds128(p); }
    __device__ static __forceinline__ void st(float *p, float4 v, uint32_t) { stg128(p, v); }
    __device__ static __forceinline__ float get(const float *p) { return *p; }
    __device__ static __forceinline__ void put(float *p, float v, uint32_t) { *p = v; }
};

template <>
struct Elem<__half> {
    static constexpr int HX = 8;
    static constexpr bool SCALED = true;
    __device__ static __forceinline__ float4 ld(const __half *p)
    {
        const uint2 r = *reinterpret_cast<const uint2 *>(p);
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&r.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&r.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
    __device__ static __forceinline__ __half2 pack(float x, float y, uint32_t rnd)
    {
#ifdef SGB_16BIT_RN
        (void)rnd;
        return __floats2half2_rn(x, y);
#else
        const uint32_t d = cvt_rs_f16x2(x, y, rnd);
        return *reinterpret_cast<const __half2 *>(&d);
#endif
    }
    __device__ static __forceinline__ void st(__half *p, float4 v, uint32_t rnd)
    {
        // the second pair's word: an odd multiple of the first (cheap, uniform)
        __half2 a = pack(v.x, v.y, rnd), b = pack(v.z, v.w, rnd * 0x9E3779B1u);
        uint2 r;
        r.x = *reinterpret_cast<uint32_t *>(&a);
        r.y = *reinterpret_cast<uint32_t *>(&b);
        *reinterpret_cast<uint2 *>(p) = r;
    }
    __device__ static __forceinline__ float get(const __half *p) { return __half2float(*p); }
    __device__ static __forceinline__ void put(__half *p, float v, uint32_t rnd)
    {
        *p = pack(v, v, rnd).x;
    }
};

template <>
struct Elem<__nv_bfloat16> {
    static constexpr int HX = 8;
    static constexpr bool SCALED = false;
    __device__ static __forceinline__ float4 ld(const __nv_bfloat16 *p)
    {
        const uint2 r = *reinterpret_cast<const uint2 *>(p);
        const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&r.x));
        const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&r.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
    __device__ static __forceinline__ __nv_bfloat162 pack(float x, float y, uint32_t rnd)
    {
#ifdef SGB_16BIT_RN
        (void)rnd;
        return __floats2bfloat162_rn(x, y);
#else
        const uint32_t d = cvt_rs_bf16x2(x, y, rnd);
        return *reinterpret_cast<const __nv_bfloat162 *>(&d);
#endif
    }
    __device__ static __forceinline__ void st(__nv_bfloat16 *p, float4 v, uint32_t rnd)
    {
        // the second pair's word: an odd multiple of the first (cheap, uniform)
        __nv_bfloat162 a = pack(v.x, v.y, rnd), b = pack(v.z, v.w, rnd * 0x9E3779B1u);
        uint2 r;
        r.x = *reinterpret_cast<uint32_t *>(&a);
        r.y = *reinterpret_cast<uint32_t *>(&b);
        *reinterpret_cast<uint2 *>(p) = r;
    }
    __device__ static __forceinline__ float get(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    __device__ static __forceinline__ void put(__nv_bfloat16 *p, float v, uint32_t rnd)
    {
        *p = pack(v, v, rnd).x;
    }
};

constexpr int align128(int b) { return (b + 127) / 128 * 128; }

template <int TXT_, int TYT_, int TY_, int NU_, int NP_, int MINB_, int U_>
struct TileCfg {
    static constexpr int TXT = TXT_, TYT = TYT_, TY = TY_, NU = NU_, NP = NP_, MINB = MINB_;
    static constexpr int U = U_;       // z-loop unroll factor
    static constexpr int QN = 8 + U_;  // register-queue length
    static constexpr int THREADS = TXT * TYT;   // consumer (compute) threads
    static constexpr int BLOCK = THREADS + 32;  // plus one producer warp
    static constexpr int BX = 4 * TXT, BY = TY * TYT;
    static constexpr int SH = BY + 2 * R;
    static constexpr int P_TILE = BX * BY;
    static constexpr int WARPS = THREADS / 32;
    // phi (or mu) tiles travel as PHI_BW-column blocks, stored block after
    // block in shared memory, so that a tile touching only the x-PML can load
    // just the blocks that hold PML columns
    static constexpr int PHI_BW = 32, PHI_NB = BX / PHI_BW;
    static_assert(NU >= 8, "the u ring must hold the 8 planes that prime the register queue");
    static_assert(BX % PHI_BW == 0 && PHI_NB <= 8, "phi blocks");
    static_assert(U_ >= 1 && U_ <= 9, "unroll factor");
    static_assert(NP >= 2 && THREADS % 32 == 0, "ring sizes");
    static_assert(SH <= 256 && BX <= 240 && BY <= 256, "TMA box limits");
};

// Shared-memory geometry of a configuration for storage type T (bytes).
template <class C, class T, int MODE = MODE_FWD>
struct Stage {
    static constexpr int HX = Elem<T>::HX;         // x margin of the u^n box
    static constexpr int SW = C::BX + 2 * HX;      // u^n box width (elements)
    static constexpr int U_BYTES = align128(SW * C::SH * (int)sizeof(T));
    static constexpr int UP_BYTES = align128(C::P_TILE * (int)sizeof(T));
    static constexpr int F_BYTES = C::P_TILE * 4;  // one fp32 tile (m, phi, g, S)
    // the adjoint's mu^{k+1} tile carries its x-y neighbours: a (BX + 8) x (BY + 2)
    // box (x halo 4 for the TMA's 16-byte alignment, y halo 1)
    static constexpr int MBW = C::BX + 8, MBH = C::BY + 2;
    static constexpr int MU_BYTES = align128(MBW * MBH * 4);
    static constexpr int PH_BYTES = MODE == MODE_ADJ ? MU_BYTES : F_BYTES;  // phi or mu slot
    static constexpr int P_BYTES = UP_BYTES + F_BYTES + PH_BYTES + (MODE == MODE_ADJ ? 2 : 0) * F_BYTES;
    // MODE_ADJ: mu^{k+1} one plane below each thread's points, kept from plane to
    // plane in shared memory (registers are at their limit)
    static constexpr int MZ_BYTES = MODE == MODE_ADJ ? C::THREADS * C::TY * 16 : 0;
    // ring depths: 16-bit storage halves the stages' bytes, so its rings run deeper
    // (12 u^n planes and 6 tile stages in ~108 KB, still two CTAs per SM)
#ifndef SGB_NU16
#define SGB_NU16 12
#endif
#ifndef SGB_NP16
#define SGB_NP16 6
#endif
    static constexpr int NU = sizeof(T) == 2 ? SGB_NU16 : C::NU;
    static constexpr int NP = sizeof(T) == 2 ? SGB_NP16 : C::NP;
    static constexpr size_t SMEM_BYTES = size_t(NU) * U_BYTES + size_t(NP) * P_BYTES +
                                         size_t(MZ_BYTES) + size_t(NU + NP) * 16 +
                                         size_t(NU + NP + 1) * 4;
    static_assert(U_BYTES % 128 == 0 && F_BYTES % 128 == 0, "stage alignment");
    static_assert(SW <= 256, "TMA box limit");
};

// Depth (points) of index i into the PML along one axis; 0 in the inner range.
__device__ __forceinline__ int pml_depth(int n_inner, int nb, int i)
{
    return max(max(nb - i, i - (nb + n_inner - 1)), 0);
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
#ifdef SGB_SCALAR_FMA
__device__ __forceinline__ void f4fma(float4 &acc, float c, const float4 &v)
{
    acc.x = fmaf(c, v.x, acc.x);
    acc.y = fmaf(c, v.y, acc.y);
    acc.z = fmaf(c, v.z, acc.z);
    acc.w = fmaf(c, v.w, acc.w);
}
__device__ __forceinline__ float4 f4mul(float c, const float4 &v)
{
    return make_float4(c * v.x, c * v.y, c * v.z, c * v.w);
}
#else
// acc += c * v on a float4 as two packed f32x2 FMAs.
__device__ __forceinline__ void f4fma(float4 &acc, float c, const float4 &v)
{
    const float2 cc = make_float2(c, c);
    float2 lo = __ffma2_rn(cc, make_float2(v.x, v.y), make_float2(acc.x, acc.y));
    float2 hi = __ffma2_rn(cc, make_float2(v.z, v.w), make_float2(acc.z, acc.w));
    acc = make_float4(lo.x, lo.y, hi.x, hi.y);
}

__device__ __forceinline__ float4 f4mul(float c, const float4 &v)
{
    const float2 cc = make_float2(c, c);
    float2 lo = __fmul2_rn(cc, make_float2(v.x, v.y));
    float2 hi = __fmul2_rn(cc, make_float2(v.z, v.w));
    return make_float4(lo.x, lo.y, hi.x, hi.y);
}
#endif

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Launch variants of the step: one launch per step over the standard units;
// the shell launches of a temporally blocked pair (units from a table, no store
// inside the two-step kernel's box); the persistent dataflow launch (CTAs take
// (step, unit) items in turn, ring slots counted across units); one launch per
// step whose output buffer is chosen on the device by the parity of the step
// (CUDA-graph replays that do not repeat with the buffer parity).
enum : int { VAR_PLAIN = 0, VAR_SHELL = 1, VAR_FLOW = 2, VAR_PARITY = 3 };

// Per-thread state of one fused-step work unit (a tile x a z-chunk).
template <class C, class T, int MODE = MODE_FWD, int VAR = VAR_PLAIN>
struct StepCta {
    static constexpr bool SHELL = VAR == VAR_SHELL, FLOW = VAR == VAR_FLOW;
    static constexpr bool OUTV = VAR == VAR_FLOW || VAR == VAR_PARITY;  // output via u_out_v
    using E = Elem<T>;
    using G = Stage<C, T, MODE>;
    // the adjoint's PML-path band is one point wider: inner points next to the
    // PML receive psi from their PML neighbours
    static constexpr int BAND = MODE == MODE_ADJ ? 1 : 0;
    static constexpr bool SCALED = E::SCALED;
    static constexpr int TXT = C::TXT, TY = C::TY, NU = Stage<C, T, MODE>::NU, NP = Stage<C, T, MODE>::NP;
    static constexpr int THREADS = C::THREADS, QN = C::QN, U = C::U, WARPS = C::WARPS;
    static constexpr int BX = C::BX, BY = C::BY, HX = G::HX, SW = G::SW;
    static constexpr int P_TILE = C::P_TILE;
    static constexpr uint64_t WAIT_NS = 2000000000ull;

    const StepArgs *pa;  // the kernel argument, in the constant parameter space
    const CUtensorMap *tm_ucur, *tm_ucur_in, *tm_uprev, *tm_m, *tm_phi, *tm_acc, *tm_gs;
    unsigned char *su, *sp;  // u ring, (u^{n-1}, m, phi) ring
    uint64_t *full_u, *empty_u, *full_p, *empty_p;
    int *lastf_u, *lastf_p, *s_abort;
    long long base_off;  // element offset of (gi, gj0, k = 0)
    int tid, lane, x0, y0, z0, z1, n, row0, colu, gi, gj0, prow;
    bool xy_inner, aborted, store_ok;
    int phi_xmask;  // phi blocks holding x-PML columns, when the tile touches only the
                    // x-PML (planes outside the z-PML load only these); 0 otherwise
    int phoff;      // offset of this thread's row-0 quad in the blocked phi tile
    int mbox;           // MODE_ADJ: offset of this thread's row-0 quad in the mu box

    // MODE_ADJ: mu^{k+1} at this thread's row-r points one plane below, kept from
    // plane to plane in shared memory (registers are at their limit)
    __device__ __forceinline__ float4 *mz_prev(int r) const
    {
        return reinterpret_cast<float4 *>(sp + NP * G::P_BYTES) + r * THREADS + tid;
    }
    int useq, pseq;  // FLOW: u and (u^{n-1}, m, phi) planes of earlier units of this CTA
    void *u_out_v;   // FLOW, PARITY: the output buffer of the current step
    float s_cur, s_prev, inv_s_next;  // fp16 scales (1 otherwise)
    float sd_cur, inv_sd_next;        // fp16 MODE_DIFF: scales of d^n and d^{n+1}
    float vmax, vmax_d;               // running max |u^{n+1}|, |d^{n+1}| of this thread
    // PML terms of the thread's fixed columns i = gi + e and rows j = gj0 + r:
    // eta dt = a d(i)^2, the gradient factor k (d(i+1)^2 - d(i-1)^2), the
    // adjoint's k G(i +- 1) with G(y) = d(y+1)^2 - d(y-1)^2, and PML masks
    float pex[4], pgx[4], phxp[4], phxm[4];
    float pey[TY], pgy[TY], phyp[TY], phym[TY];
    int pmx, pmy;
    // 1 / (1 + e) and 1 - e of the thread's points in planes outside the z-PML
    // (e = eta dt depends on x and y only there)
    float pinv[TY][4], pome[TY][4];

    __device__ __forceinline__ void pml_axis(int n_in, int i, float ca, float ck, float &e, float &gk,
                                             float &hp, float &hm, bool &in_pml) const
    {
        const int nb = pa->nb;
        const int d = pml_depth(n_in, nb, i), dp = pml_depth(n_in, nb, i + 1);
        const int dm = pml_depth(n_in, nb, i - 1);
        const int d2p = pml_depth(n_in, nb, i + 2), d2m = pml_depth(n_in, nb, i - 2);
        e = __fmul_rn(ca, float(d * d));
        gk = __fmul_rn(ck, float(dp * dp - dm * dm));
        hp = __fmul_rn(ck, float(d2p * d2p - d * d));
        hm = __fmul_rn(ck, float(d * d - d2m * d2m));
        in_pml = d > 0;
    }

    // Every PML-path operation below has an explicit rounding (fmaf, __fmul_rn,
    // __fadd_rn): implicit contraction may differ between the kernels that
    // inline this code, and the serving kernel must reproduce run_shot to the bit.
    __device__ __forceinline__ void pml_tables()
    {
        const StepArgs &a = *pa;
        pmx = pmy = 0;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            bool in;
            pml_axis(a.nx, gi + e, a.ax, a.kx, pex[e], pgx[e], phxp[e], phxm[e], in);
            pmx |= int(in) << e;
        }
#pragma unroll
        for (int r = 0; r < TY; ++r) {
            bool in;
            pml_axis(a.ny, gj0 + r, a.ay, a.ky, pey[r], pgy[r], phyp[r], phym[r], in);
            pmy |= int(in) << r;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float exy = __fadd_rn(pex[e], pey[r]);
                pinv[r][e] = rcp_approx(__fadd_rn(1.0f, exy));
                pome[r][e] = __fsub_rn(1.0f, exy);
            }
        }
    }

    __device__ __forceinline__ bool plane_pml(int k) const
    {
        return !xy_inner || k < pa->nb + BAND || k >= pa->nb + pa->nz - BAND;
    }

    __device__ __forceinline__ void wait(uint64_t *bar, uint32_t parity)
    {
        if (!mbar_wait_bounded(bar, parity, WAIT_NS)) {
            *reinterpret_cast<volatile int *>(s_abort) = 1;
            atomicOr(pa->err, DEV_ERR_TIMEOUT);
        }
    }

    __device__ __forceinline__ const T *ustage(int s) const
    {
        return reinterpret_cast<const T *>(su + s * G::U_BYTES);
    }

    // Planes outside the chunk feed only the z-queue: no x-y halo needed.
    __device__ __forceinline__ bool front_only(int p) const { return p < z0 || p >= z1; }

    // Offset, inside a u stage holding plane p, of this thread's row-r quad.
    __device__ __forceinline__ int own_off(int p, int r) const
    {
        return front_only(p) ? prow + r * BX : (row0 + r) * SW + colu;
    }

    __device__ __forceinline__ void issue_u(int p)
    {
        const int rel = p - z0 + 4 + (FLOW ? useq : 0);
        const int s = rel % NU, f = rel / NU;
        if (f > 0) wait(empty_u + s, (f - 1) & 1);  // previous plane of the slot released
        lastf_u[s] = f;
        if (front_only(p)) {
            mbar_arrive_expect_tx(full_u + s, P_TILE * (int)sizeof(T));
            // a neighbouring z-chunk's plane: kept in L2 for that chunk's own read
            tma_load_3d_hint(su + s * G::U_BYTES, tm_ucur_in, full_u + s, x0, y0, p,
                             policy_evict_last());
        } else {
            mbar_arrive_expect_tx(full_u + s, SW * C::SH * (int)sizeof(T));
            tma_load_3d(su + s * G::U_BYTES, tm_ucur, full_u + s, x0 - HX, y0 - R, p);
        }
    }

    __device__ __forceinline__ void issue_p(int k)
    {
        const int rel = k - z0 + (FLOW ? pseq : 0);
        const int s = rel % NP, f = rel / NP;
        if (f > 0) wait(empty_p + s, (f - 1) & 1);
        lastf_p[s] = f;
        const bool pml = plane_pml(k);
        const bool zpml = k < pa->nb || k >= pa->nb + pa->nz;
        const int phmask = !pml ? 0 : (phi_xmask && !zpml) ? phi_xmask : (1 << C::PHI_NB) - 1;
        const int ntiles = 1 + (MODE == MODE_ADJ ? 2 : 0);
        constexpr int PHB_BYTES = C::PHI_BW * C::BY * 4;
        const int ph_bytes = MODE == MODE_ADJ ? (pml ? G::MBW * G::MBH * 4 : 0)
                                              : __popc(phmask) * PHB_BYTES;
        mbar_arrive_expect_tx(full_p + s, P_TILE * (int)sizeof(T) + ntiles * G::F_BYTES + ph_bytes);
        unsigned char *d = sp + s * G::P_BYTES;
        // No evict-first hint: u^{n-1} and phi are overwritten in place (u^{n+1},
        // phi^{n+1}) a few planes later, and marking their lines first-to-go cost
        // 8% of the step at 512^3 (118 MB more DRAM read per launch).
        tma_load_3d(d, tm_uprev, full_p + s, x0, y0, k);
        tma_load_3d(d + G::UP_BYTES, tm_m, full_p + s, x0, y0, k);
        if constexpr (MODE == MODE_ADJ) {
            // mu^{k+1} with its x-y halo; g^{k-1} of the recomputation; partial sum S
            if (pml) tma_load_3d(d + G::UP_BYTES + G::F_BYTES, tm_phi, full_p + s, x0 - 4, y0 - 1, k);
            tma_load_3d(d + G::UP_BYTES + G::F_BYTES + G::PH_BYTES, tm_acc, full_p + s, x0, y0, k);
            tma_load_3d(d + G::UP_BYTES + 2 * G::F_BYTES + G::PH_BYTES, tm_gs, full_p + s, x0, y0, k);
        } else {
#pragma unroll
            for (int b = 0; b < C::PHI_NB; ++b)
                if ((phmask >> b) & 1)
                    tma_load_3d(d + G::UP_BYTES + G::F_BYTES + b * PHB_BYTES, tm_phi, full_p + s,
                                x0 + b * C::PHI_BW, y0, k);
        }
    }

    // Producer lane: every plane of u^n (z0-4 .. z1+3) and every (u^{n-1}, m,
    // phi) plane (z0 .. z1-1), in the order the consumers need them; each
    // refill first waits for its slot to be released.  Then waits for its own
    // copies to land, so no copy is in flight when it exits.
    __device__ __forceinline__ void produce()
    {
        produce_unit();
        drain();
    }

    __device__ __forceinline__ void produce_unit()
    {
        int nu = z0 - 4, np = z0;
        while ((nu < z1 + 4 || np < z1) && !aborted) {
            // plane nu is first needed at iteration nu - z0 - 4 (as the front
            // plane), plane np at iteration np - z0
            const bool do_u = nu < z1 + 4 && (np >= z1 || nu - z0 - 4 <= np - z0);
            if (do_u) issue_u(nu++);
            else issue_p(np++);
            aborted = *reinterpret_cast<volatile int *>(s_abort) != 0;
        }
    }

    __device__ __forceinline__ void drain()
    {
        for (int s = 0; s < NU; ++s)
            if (lastf_u[s] >= 0) mbar_wait_bounded(full_u + s, lastf_u[s] & 1, WAIT_NS);
        for (int s = 0; s < NP; ++s)
            if (lastf_p[s] >= 0) mbar_wait_bounded(full_p + s, lastf_p[s] & 1, WAIT_NS);
    }

    // One z-plane: iteration it (plane k = z0 + it).  The queue holds planes
    // k-4 .. k+3 at q[O .. O+7]; the front plane k+4 is loaded into q[O+8].
    // Queue values are the stored (scaled) values; true u = stored * s_cur.
    // KIND: PLANE_INTERIOR (no PML point in the tile's plane), PLANE_XY (PML
    // path, plane outside the z-PML: e from the thread's tables), PLANE_Z (a
    // z-PML plane).
    template <int O, int KIND>
    __device__ __forceinline__ void plane(float4 (&q)[TY][QN], int it)
    {
        constexpr bool PML = KIND != PLANE_INTERIOR;
        constexpr bool ZP = KIND == PLANE_Z;
        const StepArgs &a = *pa;
        const int k = z0 + it;
        const int relf = it + 8 + (FLOW ? useq : 0);
        const int sf = relf % NU;
        wait(full_u + sf, (relf / NU) & 1);
#pragma unroll
        for (int r = 0; r < TY; ++r) q[r][O + 8] = E::ld(ustage(sf) + own_off(k + 4, r));
        const int itp = it + (FLOW ? pseq : 0);
        const int sq = itp % NP;
        wait(full_p + sq, (itp / NP) & 1);
        const int sc = (it + 4 + (FLOW ? useq : 0)) % NU;
        const T *cu = ustage(sc);
        const unsigned char *pu = sp + sq * G::P_BYTES;
        const T *pup = reinterpret_cast<const T *>(pu);
        const float *pm = reinterpret_cast<const float *>(pu + G::UP_BYTES);
        const float *pph = reinterpret_cast<const float *>(pu + G::UP_BYTES + G::F_BYTES);
        const float *pg = reinterpret_cast<const float *>(pu + G::UP_BYTES + G::F_BYTES + G::PH_BYTES);
        const float *pgs =
            reinterpret_cast<const float *>(pu + G::UP_BYTES + 2 * G::F_BYTES + G::PH_BYTES);

        // 25-point Laplacian (Eq. 3): centre and z part from the queue
        float4 L[TY], gy[TY];
#pragma unroll
        for (int r = 0; r < TY; ++r) {
            L[r] = f4mul(a.c0, q[r][O + 4]);
#pragma unroll
            for (int m = 1; m <= R; ++m) {
                f4fma(L[r], a.cz[m - 1], q[r][O + 4 - m]);
                f4fma(L[r], a.cz[m - 1], q[r][O + 4 + m]);
            }
        }
        // y part: rows -4 .. TY+3 around the thread's first row
#pragma unroll
        for (int d = -R; d < TY + R; ++d) {
            float4 v;
            if (d >= 0 && d < TY) v = q[d][O + 4];
            else v = E::ld(cu + (row0 + d) * SW + colu);
#pragma unroll
            for (int r = 0; r < TY; ++r) {
                const int m = d > r ? d - r : r - d;
                if (m >= 1 && m <= R) f4fma(L[r], a.cy[m - 1], v);
                // gy = u(j+1) - u(j-1); row r-1 is visited before row r+1
                if (PML && d == r - 1) gy[r] = make_float4(-v.x, -v.y, -v.z, -v.w);
                if (PML && d == r + 1) f4fma(gy[r], 1.0f, v);
            }
        }
        float ez = 0.f, gzk = 0.f, hzp = 0.f, hzm = 0.f;
        bool zin = false;
        if (PML) pml_axis(a.nz, k, a.az, a.kz, ez, gzk, hzp, hzm, zin);
        const long long off0 = base_off + (long long)k * a.sxy;
        // random bits of this thread's stores in this plane (16-bit storage)
        uint32_t rnd = 0;
        if constexpr (sizeof(T) == 2) rnd = hash_bits((uint32_t)off0, (uint32_t)n);
#pragma unroll
        for (int r = 0; r < TY; ++r) {
            const T *rowp = cu + (row0 + r) * SW + colu;
            float4 c = q[r][O + 4];
            const float4 lf = E::ld(rowp - 4), rt = E::ld(rowp + 4);
            const float w[12] = {lf.x, lf.y, lf.z, lf.w, c.x, c.y, c.z, c.w,
                                 rt.x, rt.y, rt.z, rt.w};
            float4 Lr = L[r];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                float sacc = f4get(Lr, e);
#pragma unroll
                for (int m = 1; m <= R; ++m) {
                    sacc = fmaf(a.cx[m - 1], w[4 + e - m], sacc);
                    sacc = fmaf(a.cx[m - 1], w[4 + e + m], sacc);
                }
                f4set(Lr, e, sacc);
            }
            const int pr = prow + r * BX;
            float4 up = E::ld(pup + pr);
            const float4 mm = lds128(pm + pr);
            if constexpr (SCALED) {  // stored values -> true values
                Lr = f4mul(s_cur, Lr);
                c = f4mul(s_cur, c);
                up = f4mul(MODE == MODE_DIFF ? sd_cur : s_prev, up);
            }
            float4 un;  // MODE_DIFF: d^{n+1} until the source is added
            if constexpr (MODE == MODE_DIFF) {  // up = d^n: d^{n+1} = d^n + m L u^n
                un.x = fmaf(mm.x, Lr.x, up.x);
                un.y = fmaf(mm.y, Lr.y, up.y);
                un.z = fmaf(mm.z, Lr.z, up.z);
                un.w = fmaf(mm.w, Lr.w, up.w);
            } else {
                un.x = fmaf(mm.x, Lr.x, fmaf(2.0f, c.x, -up.x));
                un.y = fmaf(mm.y, Lr.y, fmaf(2.0f, c.y, -up.y));
                un.z = fmaf(mm.z, Lr.z, fmaf(2.0f, c.z, -up.z));
                un.w = fmaf(mm.w, Lr.w, fmaf(2.0f, c.w, -up.w));
            }
            const int j = gj0 + r;
            float4 phn = make_float4(0.f, 0.f, 0.f, 0.f);
            bool any_pml = false;
            int ptmask = 0;
            float4 ph = make_float4(0.f, 0.f, 0.f, 0.f);
            if (PML) {
                if constexpr (MODE == MODE_ADJ) ph = lds128(pph + mbox + r * G::MBW);
                else ph = lds128(pph + phoff + r * C::PHI_BW);
                phn = ph;
                const float eyz = ZP ? __fadd_rn(pey[r], ez) : 0.0f;
                const float gyk = pgy[r];
                // bit e: point e of this row is a PML point
                const int rowmask = (ZP || zin || ((pmy >> r) & 1)) ? 0xF : pmx;
                const float4 zp = q[r][O + 5], zm = q[r][O + 3];
                // adjoint: psi = sum_a k_a [G_a mu](x + e_a) - [G_a mu](x - e_a) from the six
                // neighbours of mu^{k+1} (zero outside the PML and in the halo): x and y
                // from the haloed box, -z kept from the plane below, +z from global memory
                float4 myp = make_float4(0.f, 0.f, 0.f, 0.f), mym = myp, mzp = myp, mzm = myp;
                float mxl = 0.f, mxr = 0.f;
                if constexpr (MODE == MODE_ADJ) {
                    const float *mb = pph + mbox + r * G::MBW;
                    myp = lds128(mb + G::MBW);
                    mym = lds128(mb - G::MBW);
                    mxl = mb[-1];
                    mxr = mb[4];
                    mzm = *mz_prev(r);
                    if (store_ok && j < a.Ny) mzp = ldg128(a.mu_in + off0 + (long long)r * a.sx + a.sxy);
                    *mz_prev(r) = ph;
                }
                const float mux[6] = {mxl, ph.x, ph.y, ph.z, ph.w, mxr};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const bool pt = (rowmask >> e) & 1;
                    any_pml |= pt;
                    float Gd = fmaf(pgx[e], __fsub_rn(w[5 + e], w[3 + e]),
                                    fmaf(gyk, f4get(gy[r], e),
                                         __fmul_rn(gzk, __fsub_rn(f4get(zp, e), f4get(zm, e)))));
                    if constexpr (SCALED) Gd = __fmul_rn(Gd, s_cur);
                    float inv, ome;  // 1 / (1 + e), 1 - e
                    if constexpr (ZP) {
                        const float edt = __fadd_rn(pex[e], eyz);
                        inv = rcp_approx(__fadd_rn(1.0f, edt));
                        ome = __fsub_rn(1.0f, edt);
                    } else {
                        inv = pinv[r][e];
                        ome = pome[r][e];
                    }
                    const float cc = f4get(c, e), pe = f4get(ph, e);
                    float rhs = pe;  // phi^n (forward) or psi (adjoint)
                    if constexpr (MODE == MODE_ADJ) {
                        rhs = fmaf(phxp[e], mux[e + 2], __fmul_rn(-phxm[e], mux[e]));
                        rhs = fmaf(phyp[r], f4get(myp, e), rhs);
                        rhs = fmaf(-phym[r], f4get(mym, e), rhs);
                        rhs = fmaf(hzp, f4get(mzp, e), rhs);
                        rhs = fmaf(-hzm, f4get(mzm, e), rhs);
                    }
                    const float lr = __fadd_rn(f4get(Lr, e), rhs);
                    float upml;
                    if constexpr (MODE == MODE_DIFF) {
                        // d^{n+1} = u^{n+1} - c with u^{n-1} = c - d^n:
                        //   [(1 - e) d^n + m lr - e^2 c] / (1 + e)
                        const float ed = __fsub_rn(1.0f, ome);
                        upml = __fmul_rn(inv, fmaf(f4get(mm, e), lr,
                                                   fmaf(ome, f4get(up, e), -__fmul_rn(__fmul_rn(ed, ed), cc))));
                    } else {
                        // [(2 - e^2) c - (1 - e) u^{n-1} + m lr] / (1 + e)
                        //   = (1 - e) c + [c - (1 - e) u^{n-1} + m lr] / (1 + e)
                        upml = fmaf(inv, fmaf(f4get(mm, e), lr, fmaf(-ome, f4get(up, e), cc)),
                                    __fmul_rn(ome, cc));
                    }
                    const float ppml = __fmul_rn(__fsub_rn(pe, Gd), inv);
                    ptmask |= int(pt) << e;
                    if constexpr (MODE == MODE_ADJ) {
                        // psi also reaches the inner points next to the PML;
                        // mu^k = (mu^{k+1} + w^{k+1}) / (1 + e) on the PML
                        f4set(un, e, pt ? upml : fmaf(f4get(mm, e), lr, fmaf(2.0f, cc, -f4get(up, e))));
                        if (pt) f4set(phn, e, __fmul_rn(__fadd_rn(pe, cc), inv));
                    } else if (pt) {
                        f4set(un, e, upml);
                        f4set(phn, e, ppml);
                    }
                }
            }
            if constexpr (MODE == MODE_ADJ && !PML) *mz_prev(r) = make_float4(0.f, 0.f, 0.f, 0.f);
            float4 acc4 = Lr;  // MODE_FWD_ACC: g = L u^n + phi^n + f^n
            if constexpr (MODE == MODE_FWD_ACC) {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if ((ptmask >> e) & 1) f4set(acc4, e, f4get(acc4, e) + f4get(ph, e));
            }
            // point source (Eq. 2 right-hand side), added by the owning thread
            if (MODE != MODE_ADJ && k == a.sk && j == a.sj && a.si >= gi && a.si < gi + 4) {
                const int e = a.si - gi;
                const float f = a.wavelet[n] * a.inv_vol;
                f4set(un, e, fmaf(f4get(mm, e), f, f4get(un, e)));
                if constexpr (MODE == MODE_FWD_ACC) f4set(acc4, e, f4get(acc4, e) + f);
            }
            float4 dn;  // MODE_DIFF: d^{n+1}; u^{n+1} = u^n + d^{n+1}
            if constexpr (MODE == MODE_DIFF) {
                dn = un;
                un = make_float4(__fadd_rn(c.x, dn.x), __fadd_rn(c.y, dn.y), __fadd_rn(c.z, dn.z),
                                 __fadd_rn(c.w, dn.w));
            }
            // shell launches leave the box to the two-step kernel (its x bounds
            // are multiples of 4: a quad is wholly inside or outside)
            const bool boxed = SHELL && gi >= a.bx0 && gi < a.bx1 && j >= a.by0 && j < a.by1 &&
                               k >= a.bz0 && k < a.bz1;
            if (store_ok && j < a.Ny && !boxed) {
                const long long off = off0 + (long long)r * a.sx;
                if constexpr (SCALED) {
                    vmax = fmaxf(vmax, fmaxf(fmaxf(fabsf(un.x), fabsf(un.y)),
                                             fmaxf(fabsf(un.z), fabsf(un.w))));
                    un = f4mul(inv_s_next, un);
                    if constexpr (MODE == MODE_DIFF) {
                        vmax_d = fmaxf(vmax_d, fmaxf(fmaxf(fabsf(dn.x), fabsf(dn.y)),
                                                     fmaxf(fabsf(dn.z), fabsf(dn.w))));
                        dn = f4mul(inv_sd_next, dn);
                    }
                }
                T *uo = static_cast<T *>(OUTV ? u_out_v : a.u_out) + off;
                const bool wphi = PML && any_pml;  // phi^{n+1}, or mu^k in the adjoint
                // MODE_DIFF: d^{n+1} rounded with its own random word (an odd
                // multiple of u's, so uniform and distinct)
                T *dio = nullptr;
                if constexpr (MODE == MODE_DIFF) dio = static_cast<T *>(a.d_io) + off;
                const uint32_t rnd_d = rnd * 0x2C1B3C6Du;
                if (gi + 3 < a.Nx) {
                    E::st(uo, un, rnd);
                    if constexpr (MODE == MODE_DIFF) E::st(dio, dn, rnd_d);
                    if (wphi) stg128(a.phi + off, phn);
                    if constexpr (MODE == MODE_FWD_ACC) stg128(a.acc_out + off, acc4);
                } else {
                    for (int e = 0; e < 4 && gi + e < a.Nx; ++e) {
                        E::put(uo + e, f4get(un, e), hash_bits(rnd, (uint32_t)e));
                        if constexpr (MODE == MODE_DIFF)
                            E::put(dio + e, f4get(dn, e), hash_bits(rnd_d, (uint32_t)e));
                        if (wphi) a.phi[off + e] = f4get(phn, e);
                        if constexpr (MODE == MODE_FWD_ACC) a.acc_out[off + e] = f4get(acc4, e);
                    }
                }
                if constexpr (sizeof(T) == 2) rnd = next_bits(rnd);  // the next row's word
                if constexpr (MODE == MODE_ADJ) {
                    // S += w^k g^{k-1} (dJ/dm = sum_k w^k g^{k-1} / m; S is folded
                    // into the fp64 sum every few steps)
                    const float4 gk = lds128(pg + pr);
                    float4 s4 = lds128(pgs + pr);
                    s4.x = fmaf(un.x, gk.x, s4.x);
                    s4.y = fmaf(un.y, gk.y, s4.y);
                    s4.z = fmaf(un.z, gk.z, s4.z);
                    s4.w = fmaf(un.w, gk.w, s4.w);
                    if (gi + 3 < a.Nx) stg128(a.gsum + off, s4);
                    else
                        for (int e = 0; e < 4 && gi + e < a.Nx; ++e) a.gsum[off + e] = f4get(s4, e);
                }
            }
        }
        // release the current u plane and this p slot
        __syncwarp();
        if (lane == 0) {
            mbar_arrive(empty_u + sc);
            mbar_arrive(empty_p + sq);
        }
        aborted = *reinterpret_cast<volatile int *>(s_abort) != 0;
    }

    // Tile-level geometry of the unit (x0, y0, z0, z1 set): whether the tile
    // touches the x-y PML band, and which phi blocks its planes need.
    __device__ __forceinline__ void unit_geometry()
    {
        const StepArgs &a = *pa;
        const int xe = min(x0 + BX, a.Nx), ye = min(y0 + BY, a.Ny);
        xy_inner = x0 >= a.nb + BAND && xe <= a.nb + a.nx - BAND && y0 >= a.nb + BAND &&
                   ye <= a.nb + a.ny - BAND;
        phi_xmask = 0;
        if (MODE != MODE_ADJ && !xy_inner && y0 >= a.nb && ye <= a.nb + a.ny) {
            // rows all y-inner: only columns in the x-PML need phi outside the z-PML
            for (int b = 0; b < C::PHI_NB; ++b) {
                const int c0 = x0 + b * C::PHI_BW, c1 = min(c0 + C::PHI_BW, a.Nx);
                if (c0 < a.Nx && (c0 < a.nb || c1 > a.nb + a.nx)) phi_xmask |= 1 << b;
            }
        }
    }

    // This consumer thread's points in the unit and their PML tables.
    __device__ __forceinline__ void thread_geometry()
    {
        const StepArgs &a = *pa;
        const int txi = tid % C::TXT, tyi = tid / C::TXT;
        row0 = R + TY * tyi;
        colu = G::HX + 4 * txi;
        gi = x0 + 4 * txi;
        gj0 = y0 + TY * tyi;
        prow = (TY * tyi) * BX + 4 * txi;
        phoff = (4 * txi / C::PHI_BW) * C::PHI_BW * BY + (TY * tyi) * C::PHI_BW + (4 * txi) % C::PHI_BW;
        store_ok = gi < a.Nx;
        base_off = a.origin + (long long)gj0 * a.sx + gi;
        pml_tables();
        if constexpr (MODE == MODE_ADJ) mbox = (1 + TY * tyi) * G::MBW + 4 + 4 * txi;
    }

    // Prime the register queue with planes z0-4 .. z0+3 and run the unit's
    // planes: z-PML planes below the inner region, then the planes outside the
    // z-PML (interior path, or the PML path for tiles touching the x-y PML band
    // and for the adjoint's band planes next to the z-PML), then the z-PML
    // planes above it.
    __device__ __forceinline__ void consume_unit(float4 (&q)[TY][QN])
    {
        const StepArgs &a = *pa;
        const int nit = z1 - z0;
        const int u0 = FLOW ? useq : 0;
        if constexpr (MODE == MODE_ADJ) {  // mu^{k+1} one plane below the unit
#pragma unroll
            for (int r = 0; r < TY; ++r)
                *mz_prev(r) = store_ok && gj0 + r < a.Ny
                                 ? ldg128(a.mu_in + base_off + (long long)(z0 - 1) * a.sxy +
                                          (long long)r * a.sx)
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            wait(full_u + (u0 + s) % NU, ((u0 + s) / NU) & 1);
#pragma unroll
            for (int r = 0; r < TY; ++r) q[r][s] = E::ld(ustage((u0 + s) % NU) + own_off(z0 - 4 + s, r));
        }
        // planes z0-4 .. z0-1 are not needed again
        __syncwarp();
        if (lane == 0)
            for (int s = 0; s < 4; ++s) mbar_arrive(empty_u + (u0 + s) % NU);
        aborted = *reinterpret_cast<volatile int *>(s_abort) != 0;
        const int zlo = min(max(a.nb - z0, 0), nit);
        const int zhi = min(max(a.nb + a.nz - z0, zlo), nit);
        segment<PLANE_Z>(q, 0, zlo);
        if (!xy_inner) {
            segment<PLANE_XY>(q, zlo, zhi);
        } else {
            const int b0 = min(max(a.nb + BAND - z0, zlo), zhi);
            const int b1 = min(max(a.nb + a.nz - BAND - z0, b0), zhi);
            segment<PLANE_XY>(q, zlo, b0);
            segment<PLANE_INTERIOR>(q, b0, b1);
            segment<PLANE_XY>(q, b1, zhi);
        }
        segment<PLANE_Z>(q, zhi, nit);
    }

    template <int O>
    __device__ __forceinline__ void shift(float4 (&q)[TY][QN])
    {
#pragma unroll
        for (int r = 0; r < TY; ++r)
#pragma unroll
            for (int jq = 0; jq < 8; ++jq) q[r][jq] = q[r][jq + O];
    }

    template <int O, int KIND>
    __device__ __forceinline__ void group(float4 (&q)[TY][QN], int it)
    {
        if constexpr (O < U) {
            plane<O, KIND>(q, it + O);
            group<O + 1, KIND>(q, it);
        }
    }

    // Iterations [it, it_end) of one kind (PML or interior): groups of U
    // planes with compile-time queue offsets, then single planes.
    template <int KIND>
    __device__ __forceinline__ void segment(float4 (&q)[TY][QN], int it, int it_end)
    {
        if (U > 1) {
            for (; it + U <= it_end && !aborted; it += U) {
                group<0, KIND>(q, it);
                shift<U>(q);
            }
        }
        for (; it < it_end && !aborted; ++it) {
            plane<0, KIND>(q, it);
            shift<1>(q);
        }
    }
};

// Power-of-two fp16 scale for a field bounded by B: B / scale < 2^14.
__device__ __forceinline__ float pow2_scale_for(float B)
{
    if (!(B > 0.0f) || !isfinite(B)) return 1.0f;
    return ldexpf(1.0f, ilogbf(B) + 1 - 14);
}

// Resident CTAs per SM asked of the compiler: 16-bit storage halves the u
// ring's shared memory, leaving room for a third CTA if registers allow.
template <class C, class T>
constexpr int min_blocks()
{
#ifdef SGB_MINB16
    return sizeof(T) == 2 ? SGB_MINB16 : C::MINB;
#else
    return C::MINB;
#endif
}

// The five tensor maps of one step: u^n with halo, u^n interior, u^{n-1}, m, phi.
struct StepMapPtrs {
    const CUtensorMap *ucur, *ucur_in, *uprev, *m, *phi;
    const CUtensorMap *acc;  // MODE_ADJ: g^{k-1}
    const CUtensorMap *gs;   // MODE_ADJ: partial sum S
};

// One work unit (tile x z-chunk, index `unit` of `units`) of step n.  With
// sample_only, only the receivers of the previous step are sampled (the extra
// launch after a shot's last step).
template <class C, class T, int MODE = MODE_FWD, int VAR = VAR_PLAIN>
__device__ __forceinline__ void step_unit(const StepArgs &a, const StepMapPtrs &tm, int unit,
                                          int units, int n, bool sample_only,
                                          void *u_out_v = nullptr, const void *u_cur_v = nullptr)
{
    using S = StepCta<C, T, MODE, VAR>;
    constexpr bool SHELL = VAR == VAR_SHELL;
    using G = Stage<C, T, MODE>;
    static_assert(MODE == MODE_FWD || MODE == MODE_DIFF || sizeof(T) == 4,
                  "the adjoint runs in fp32");
    constexpr int TY = C::TY, NU = G::NU, NP = G::NP, THREADS = C::THREADS;
    constexpr int BX = C::BX, BY = C::BY;

    extern __shared__ __align__(128) unsigned char smem_raw[];
    S st;
    st.pa = &a;
    st.tm_ucur = tm.ucur;
    st.tm_ucur_in = tm.ucur_in;
    st.tm_uprev = tm.uprev;
    st.tm_m = tm.m;
    st.tm_phi = tm.phi;
    st.tm_acc = tm.acc;
    st.tm_gs = tm.gs;
    st.su = smem_raw;
    st.sp = smem_raw + NU * G::U_BYTES;
    st.full_u = reinterpret_cast<uint64_t *>(st.sp + NP * G::P_BYTES + G::MZ_BYTES);
    st.empty_u = st.full_u + NU;
    st.full_p = st.empty_u + NU;
    st.empty_p = st.full_p + NP;
    st.lastf_u = reinterpret_cast<int *>(st.empty_p + NP);
    st.lastf_p = st.lastf_u + NU;
    // kept in the dynamic region: no static shared memory, so the TMA
    // destinations start at the aligned base
    st.s_abort = st.lastf_p + NP;

    const int tid = threadIdx.x;
    st.tid = tid;
    st.lane = tid & 31;
    st.u_out_v = u_out_v;

    // Work unit: chunk-major so that CTAs running together share z and their
    // x-y halos meet in L2.
    if constexpr (SHELL) {
        const int4 u = a.units[unit];
        st.x0 = u.x;
        st.y0 = u.y;
        st.z0 = u.z;
        st.z1 = u.w;
    } else {
        const int per_chunk = a.tiles_x * a.tiles_y;
        const int chunk = unit / per_chunk;
        const int trem = unit - chunk * per_chunk;
        const int tyl = trem / a.tiles_x, txl = trem - tyl * a.tiles_x;
        st.x0 = txl * BX;
        st.y0 = tyl * BY;
        st.z0 = chunk * a.zc;
        st.z1 = min(st.z0 + a.zc, a.Nz);
    }
    const int nit = st.z1 - st.z0;
    st.n = n;
    st.aborted = false;
    st.s_cur = st.s_prev = st.inv_s_next = st.sd_cur = st.inv_sd_next = 1.0f;
    st.vmax = st.vmax_d = 0.0f;
    if constexpr (S::SCALED) {
        ScaleState *ss = a.scale;
        st.s_cur = ss->s[n & 3];
        st.s_prev = ss->s[(n - 1) & 3];
        const float inj = a.sk >= 0 ? fabsf(*a.m_src * a.wavelet[n] * a.inv_vol) : 0.0f;
        float B = 4.0f * fmaxf(ss->mx[n & 3], ss->mx[(n - 1) & 3]) + inj;
        if constexpr (MODE == MODE_DIFF) {
            // |m L u| <= 4 max|u| at a stable dt, so |d^{n+1}| <= 2 max|d^n| + 4 max|u^n|
            // + the injected amplitude (the factor 2 covers the PML terms), and
            // |u^{n+1}| <= max|u^n| + that
            ScaleState *sd = a.scale_d;
            st.sd_cur = sd->s[n & 3];
            const float Bd = 2.0f * sd->mx[n & 3] + 4.0f * ss->mx[n & 3] + inj;
            const float sd_next = pow2_scale_for(Bd);
            st.inv_sd_next = 1.0f / sd_next;  // exact: a power of two
            B = ss->mx[n & 3] + Bd;
            if (unit == 0 && tid == 0 && !sample_only) {
                sd->s[(n + 1) & 3] = sd_next;
                sd->mx[(n + 2) & 3] = 0.0f;
            }
        }
        const float s_next = pow2_scale_for(B);
        st.inv_s_next = 1.0f / s_next;  // exact: a power of two
        if (unit == 0 && tid == 0 && !sample_only) {
            ss->s[(n + 1) & 3] = s_next;
            ss->mx[(n + 2) & 3] = 0.0f;
        }
    }

    // Receivers of the previous step: u^n is read-only in this launch.
    if (a.nrec > 0 && n >= 1 + a.rec_n0) {
        const T *uc = static_cast<const T *>(S::OUTV ? u_cur_v : a.u_cur);
        for (int r = unit * C::BLOCK + tid; r < a.nrec; r += units * C::BLOCK) {
            const float v = Elem<T>::get(uc + a.rec_off[r]) * st.s_cur;
            a.traces[(long long)(n - 1 - a.rec_n0) * a.nrec + r] = v;
            if (!isfinite(v)) atomicOr(a.err, DEV_ERR_NONFINITE);
        }
    }

    if (sample_only) return;

    st.unit_geometry();

    if (tid == THREADS) {
        *st.s_abort = 0;
        for (int i = 0; i < NU; ++i) {
            mbar_init(st.full_u + i, 1);
            mbar_init(st.empty_u + i, C::WARPS);
            st.lastf_u[i] = -1;
        }
        for (int i = 0; i < NP; ++i) {
            mbar_init(st.full_p + i, 1);
            mbar_init(st.empty_p + i, C::WARPS);
            st.lastf_p[i] = -1;
        }
        fence_barrier_init();
    }
    __syncthreads();
    if (nit <= 0) return;

    if (tid >= THREADS) {  // producer warp: one lane issues every copy
        if (tid == THREADS) st.produce();
        return;
    }

    st.thread_geometry();
    float4 q[TY][C::QN];
    st.consume_unit(q);

    if constexpr (S::SCALED) {  // max |u^{n+1}| for the next step's scale
        float v = st.vmax;
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (st.lane == 0 && v > 0.0f) atomicMax(reinterpret_cast<int *>(&a.scale->mx[(n + 1) & 3]),
                                                 __float_as_int(v));
        if constexpr (MODE == MODE_DIFF) {  // and max |d^{n+1}|
            float vd = st.vmax_d;
            for (int o = 16; o > 0; o >>= 1) vd = fmaxf(vd, __shfl_xor_sync(0xffffffffu, vd, o));
            if (st.lane == 0 && vd > 0.0f)
                atomicMax(reinterpret_cast<int *>(&a.scale_d->mx[(n + 1) & 3]), __float_as_int(vd));
        }
    }
}

// One time step of one grid: one CTA per work unit.
template <class C, class T>
__global__ void __launch_bounds__(C::BLOCK, (min_blocks<C, T>()))
    fused_step_kernel(const __grid_constant__ StepArgs a,
                      const __grid_constant__ CUtensorMap tm_ucur,
                      const __grid_constant__ CUtensorMap tm_ucur_in,
                      const __grid_constant__ CUtensorMap tm_uprev,
                      const __grid_constant__ CUtensorMap tm_m,
                      const __grid_constant__ CUtensorMap tm_phi)
{
    grid_dependency_sync();
    const StepMapPtrs tm = {&tm_ucur, &tm_ucur_in, &tm_uprev, &tm_m, &tm_phi, nullptr, nullptr};
    const int n = (a.step_ptr ? *a.step_ptr : 0) + a.step_add;
    step_unit<C, T>(a, tm, blockIdx.x, gridDim.x, n, false);
}

// One time step in difference form (MODE_DIFF): one CTA per work unit.
template <class C, class T>
__global__ void __launch_bounds__(C::BLOCK, (min_blocks<C, T>()))
    diff_step_kernel(const __grid_constant__ StepArgs a,
                     const __grid_constant__ CUtensorMap tm_ucur,
                     const __grid_constant__ CUtensorMap tm_ucur_in,
                     const __grid_constant__ CUtensorMap tm_d,
                     const __grid_constant__ CUtensorMap tm_m,
                     const __grid_constant__ CUtensorMap tm_phi)
{
    grid_dependency_sync();
    const StepMapPtrs tm = {&tm_ucur, &tm_ucur_in, &tm_d, &tm_m, &tm_phi, nullptr, nullptr};
    const int n = (a.step_ptr ? *a.step_ptr : 0) + a.step_add;
    step_unit<C, T, MODE_DIFF>(a, tm, blockIdx.x, gridDim.x, n, false);
}

// One fused step on the work units of a table, storing nothing inside the
// two-step kernel's box (the shell of a temporally blocked pair, fp32).
template <class C>
__global__ void __launch_bounds__(C::BLOCK, C::MINB)
    shell_step_kernel(const __grid_constant__ StepArgs a, const __grid_constant__ CUtensorMap tm_ucur,
                      const __grid_constant__ CUtensorMap tm_ucur_in,
                      const __grid_constant__ CUtensorMap tm_uprev,
                      const __grid_constant__ CUtensorMap tm_m,
                      const __grid_constant__ CUtensorMap tm_phi)
{
    grid_dependency_sync();
    const StepMapPtrs tm = {&tm_ucur, &tm_ucur_in, &tm_uprev, &tm_m, &tm_phi, nullptr, nullptr};
    const int n = (a.step_ptr ? *a.step_ptr : 0) + a.step_add;
    step_unit<C, float, MODE_FWD, VAR_SHELL>(a, tm, blockIdx.x, gridDim.x, n, false);
}

// One step of one shot inside a CUDA-graph replay: the step n = *step_ptr +
// step_add comes from a device counter, the buffers and tensor maps of its
// parity are chosen here (so a replay of any length repeats), and launches past
// the shot's last step do nothing (n_end: the last launch, which only samples
// the receivers of step n_end - 1).
struct ShotRun {
    void *buf[2];         // step n reads buf[(n + 1) & 1] and writes buf[n & 1]
    const int *step_ptr;  // the shot's device step counter
    int step_add;
    int n_end;
};

template <class C>
__global__ void __launch_bounds__(C::BLOCK, C::MINB)
    shot_step_kernel(const __grid_constant__ StepArgs a, const __grid_constant__ ShotRun r,
                     const __grid_constant__ CUtensorMap m0_ucur,
                     const __grid_constant__ CUtensorMap m0_ucur_in,
                     const __grid_constant__ CUtensorMap m0_uprev,
                     const __grid_constant__ CUtensorMap m0_m,
                     const __grid_constant__ CUtensorMap m0_phi,
                     const __grid_constant__ CUtensorMap m1_ucur,
                     const __grid_constant__ CUtensorMap m1_ucur_in,
                     const __grid_constant__ CUtensorMap m1_uprev,
                     const __grid_constant__ CUtensorMap m1_m,
                     const __grid_constant__ CUtensorMap m1_phi)
{
    grid_dependency_sync();
    const int n = *r.step_ptr + r.step_add;
    if (n > r.n_end) return;  // finished: waits for retirement
    const bool odd = n & 1;
    const StepMapPtrs tm = odd ? StepMapPtrs{&m1_ucur, &m1_ucur_in, &m1_uprev, &m1_m, &m1_phi,
                                             nullptr, nullptr}
                               : StepMapPtrs{&m0_ucur, &m0_ucur_in, &m0_uprev, &m0_m, &m0_phi,
                                             nullptr, nullptr};
    step_unit<C, float, MODE_FWD, VAR_PARITY>(a, tm, blockIdx.x, gridDim.x, n, n == r.n_end,
                                              r.buf[n & 1], r.buf[(n + 1) & 1]);
}

// Forward step that also stores g^n = L u^n + phi^n + f^n (adjoint recomputation).
template <class C>
__global__ void __launch_bounds__(C::BLOCK, C::MINB)
    fwd_acc_kernel(const __grid_constant__ StepArgs a, const __grid_constant__ CUtensorMap tm_ucur,
                   const __grid_constant__ CUtensorMap tm_ucur_in,
                   const __grid_constant__ CUtensorMap tm_uprev,
                   const __grid_constant__ CUtensorMap tm_m,
                   const __grid_constant__ CUtensorMap tm_phi)
{
    grid_dependency_sync();
    const StepMapPtrs tm = {&tm_ucur, &tm_ucur_in, &tm_uprev, &tm_m, &tm_phi, nullptr, nullptr};
    step_unit<C, float, MODE_FWD_ACC>(a, tm, blockIdx.x, gridDim.x, a.step_add, false);
}

// Adjoint step k (see the adjoint notes in adjoint.cuh): reads w^{k+1} through
// the u^n maps, w^{k+2} through the u^{n-1} map (overwritten with w^k),
// mu^{k+1} through the phi map (mu^k is written to a.phi), g^{k-1} through the
// acc map and the partial gradient sum S through the gs map (updated in place).
template <class C>
__global__ void __launch_bounds__(C::BLOCK, C::MINB)
    adjoint_step_kernel(const __grid_constant__ StepArgs a,
                        const __grid_constant__ CUtensorMap tm_ucur,
                        const __grid_constant__ CUtensorMap tm_ucur_in,
                        const __grid_constant__ CUtensorMap tm_uprev,
                        const __grid_constant__ CUtensorMap tm_m,
                        const __grid_constant__ CUtensorMap tm_mu,
                        const __grid_constant__ CUtensorMap tm_acc,
                        const __grid_constant__ CUtensorMap tm_gs)
{
    grid_dependency_sync();
    const StepMapPtrs tm = {&tm_ucur, &tm_ucur_in, &tm_uprev, &tm_m, &tm_mu, &tm_acc, &tm_gs};
    step_unit<C, float, MODE_ADJ>(a, tm, blockIdx.x, gridDim.x, a.step_add, false);
}

}  // namespace sgb
