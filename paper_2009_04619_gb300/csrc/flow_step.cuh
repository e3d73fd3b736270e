// Persistent dataflow launch of the fused step (Algorithm 1's time loop in one
// launch).
//
// A launch of one-step-per-launch kernels ends each step with a tail (the last
// wave of work units leaves SMs idle) and starts the next with every CTA
// priming its pipeline at once; on grids of a few waves (256^3 and below) that
// costs a quarter of the step.  Here a grid of resident-size CTAs stays on the
// GPU for many steps.  The (step, work unit) items of the launch are numbered
// step-major and taken in turn from a global counter by each CTA's producer
// warp.  Before loading item (n, u) the producer waits until the 3 x 3 x 3
// neighbouring units of u (tiles +-1 in x and y, z-chunks +-1) have completed
// step n - 1:
//   - their u^n is then written (u's planes read u^n with a radius-4 halo,
//     tiles and chunks are at least 4 points wide);
//   - their step n - 1 has finished reading u^{n-1} around u, which step n
//     overwrites in place with u^{n+1} at u's points;
//   - phi^n at u's points was written by (n - 1, u) itself.
// A unit's completion is published after all its stores (and its receiver
// samples) by a release store of n + 1 into done[u]; waits use acquire loads
// and a proxy fence before the TMA copies.  Items are taken in increasing
// order and an item depends only on items of the previous step, which running
// CTAs took earlier, so the launch always makes progress whatever the number
// of resident CTAs.  Every wait is bounded; on timeout the error word gets
// DEV_ERR_TIMEOUT and every CTA leaves.
//
// Receivers are sampled by the unit that computes them, right after its last
// plane, from u^{n+1} (so no sampling launch follows the last step).  The
// per-point arithmetic is the plane body of the one-step kernel: results equal
// the one-launch-per-step path bit for bit.  fp16 with a per-field scale is not
// supported here (its scale needs all of step n before step n + 1 starts).
#pragma once
#include "step_kernel.cuh"

namespace sgb {

struct FlowArgs {
    int units;             // work units per step (chunk-major numbering)
    int tiles_x, tiles_y;  // tiles per chunk
    int n_begin, n_end;    // steps of this launch
    int *counter;          // item counter, zero when the launch starts
    int *done;             // done[u]: number of steps unit u has completed
    const int *rec_start;  // receivers in unit u: rec_list[rec_start[u] .. rec_start[u + 1])
    const int *rec_list;   // receiver indices, grouped by unit
    void *buf[2];          // step n reads u^n from buf[(n + 1) & 1] and writes u^{n+1}
                           // over u^{n-1} in buf[n & 1]
};

__device__ __forceinline__ int ld_acquire_gpu(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(int *p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Order this thread's later async-proxy (TMA) reads of global memory after its
// generic-proxy view, which acquired other CTAs' writes.
__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ void consumer_barrier(int threads)
{
    asm volatile("bar.sync 1, %0;" ::"r"(threads) : "memory");
}

// A stored wavefield value read through L2 (not L1), as fp32.
__device__ __forceinline__ float ld_cg_value(const float *p) { return __ldcg(p); }
__device__ __forceinline__ float ld_cg_value(const __nv_bfloat16 *p)
{
    const unsigned short b = __ldcg(reinterpret_cast<const unsigned short *>(p));
    return __uint_as_float((uint32_t)b << 16);
}

// Wait (the whole warp) until the units around `unit` have completed `need`
// steps.  False when the wait gave up or another CTA did.
__device__ __forceinline__ bool flow_wait_deps(const FlowArgs &f, int chunks, int unit, int need,
                                               int *err, int *s_abort)
{
    if (need <= 0) return true;
    const int lane = threadIdx.x & 31;
    const int per_chunk = f.tiles_x * f.tiles_y;
    const int c = unit / per_chunk, rem = unit - c * per_chunk;
    const int ty = rem / f.tiles_x, tx = rem - ty * f.tiles_x;
    int v = -1;
    if (lane < 27) {
        const int c2 = c + lane / 9 - 1, y2 = ty + (lane / 3) % 3 - 1, x2 = tx + lane % 3 - 1;
        if (c2 >= 0 && c2 < chunks && y2 >= 0 && y2 < f.tiles_y && x2 >= 0 && x2 < f.tiles_x)
            v = c2 * per_chunk + y2 * f.tiles_x + x2;
    }
    const uint64_t t0 = global_timer_ns();
    for (;;) {
        const bool ok = v < 0 || ld_acquire_gpu(f.done + v) >= need;
        if (__all_sync(0xffffffffu, ok)) return true;
        bool give_up = false;
        if (lane == 0)
            give_up = global_timer_ns() - t0 > 2000000000ull ||
                      (*reinterpret_cast<volatile int *>(err) & DEV_ERR_TIMEOUT) ||
                      *reinterpret_cast<volatile int *>(s_abort);
        if (__any_sync(0xffffffffu, give_up)) {
            if (lane == 0) {
                *reinterpret_cast<volatile int *>(s_abort) = 1;
                atomicOr(err, DEV_ERR_TIMEOUT);
            }
            return false;
        }
        __nanosleep(100);
    }
}

// Shared memory of the flow kernel beyond the step kernel's: two item slots
// and their full / empty barriers.
constexpr int FLOW_SMEM_EXTRA = 64;

template <class C, class T>
__global__ void __launch_bounds__(C::BLOCK, (min_blocks<C, T>()))
    flow_step_kernel(const __grid_constant__ StepArgs a0, const __grid_constant__ FlowArgs f,
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
    using S = StepCta<C, T, MODE_FWD, VAR_FLOW>;
    using G = Stage<C, T>;
    static_assert(!S::SCALED, "the dataflow launch has no per-step fp16 scale");
    constexpr int NU = S::NU, NP = S::NP, THREADS = C::THREADS, TY = C::TY;

    extern __shared__ __align__(128) unsigned char smem_raw[];
    S st;
    st.su = smem_raw;
    st.sp = smem_raw + NU * G::U_BYTES;
    st.full_u = reinterpret_cast<uint64_t *>(st.sp + NP * G::P_BYTES + G::MZ_BYTES);
    st.empty_u = st.full_u + NU;
    st.full_p = st.empty_u + NU;
    st.empty_p = st.full_p + NP;
    st.lastf_u = reinterpret_cast<int *>(st.empty_p + NP);
    st.lastf_p = st.lastf_u + NU;
    st.s_abort = st.lastf_p + NP;
    uint64_t *item_full = reinterpret_cast<uint64_t *>(smem_raw + (G::SMEM_BYTES + 7) / 8 * 8);
    uint64_t *item_empty = item_full + 2;
    int *item_buf = reinterpret_cast<int *>(item_empty + 2);

    const int tid = threadIdx.x;
    st.tid = tid;
    st.lane = tid & 31;
    st.aborted = false;
    st.s_cur = st.s_prev = st.inv_s_next = 1.0f;
    st.vmax = 0.0f;
    st.useq = st.pseq = 0;
    st.tm_acc = st.tm_gs = nullptr;
    st.pa = &a0;
    const int chunks = (a0.Nz + a0.zc - 1) / a0.zc;
    const int total = (f.n_end - f.n_begin) * f.units;

    if (tid == THREADS) {
        *st.s_abort = (*reinterpret_cast<volatile int *>(a0.err) & DEV_ERR_TIMEOUT) ? 1 : 0;
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
        for (int i = 0; i < 2; ++i) {
            mbar_init(item_full + i, 1);
            mbar_init(item_empty + i, C::WARPS);
        }
        fence_barrier_init();
    }
    __syncthreads();
    st.aborted = *reinterpret_cast<volatile int *>(st.s_abort) != 0;

    auto place = [&](int item, int &n, int &unit) {
        n = f.n_begin + item / f.units;
        unit = item - (item / f.units) * f.units;
        const int per_chunk = f.tiles_x * f.tiles_y;
        const int chunk = unit / per_chunk, rem = unit - chunk * per_chunk;
        const int tyl = rem / f.tiles_x, txl = rem - tyl * f.tiles_x;
        st.x0 = txl * C::BX;
        st.y0 = tyl * C::BY;
        st.z0 = chunk * a0.zc;
        st.z1 = min(st.z0 + a0.zc, a0.Nz);
        st.n = n;
        st.u_out_v = f.buf[n & 1];
    };

    if (tid >= THREADS) {  // producer warp: takes items, waits for them, issues copies
        const int lane = st.lane;
        for (int k = 0;; ++k) {
            int item = 0;
            if (lane == 0) item = atomicAdd(f.counter, 1);
            item = __shfl_sync(0xffffffffu, item, 0);
            const bool stop = item >= total || st.aborted;
            const int slot = k & 1;
            if (lane == 0) {
                if (k >= 2) st.wait(item_empty + slot, ((k >> 1) - 1) & 1);
                item_buf[slot] = stop ? -1 : item;
                mbar_arrive(item_full + slot);
            }
            __syncwarp();
            if (stop) break;
            int n, unit;
            place(item, n, unit);
            if (!flow_wait_deps(f, chunks, unit, n, a0.err, st.s_abort)) break;
            if (lane == 0) {
                __threadfence();
                fence_proxy_async_global();
                const bool odd = n & 1;
                st.tm_ucur = odd ? &m1_ucur : &m0_ucur;
                st.tm_ucur_in = odd ? &m1_ucur_in : &m0_ucur_in;
                st.tm_uprev = odd ? &m1_uprev : &m0_uprev;
                st.tm_m = odd ? &m1_m : &m0_m;
                st.tm_phi = odd ? &m1_phi : &m0_phi;
                st.unit_geometry();
                st.produce_unit();
            }
            st.useq += st.z1 - st.z0 + 8;
            st.pseq += st.z1 - st.z0;
            st.aborted = __shfl_sync(0xffffffffu, st.aborted ? 1 : 0, 0) != 0;
        }
        if (lane == 0) st.drain();
        return;
    }

    float4 q[TY][C::QN];
    for (int k = 0;; ++k) {
        const int slot = k & 1;
        st.wait(item_full + slot, (k >> 1) & 1);
        const int item = *reinterpret_cast<volatile int *>(item_buf + slot);
        __syncwarp();
        if (st.lane == 0) mbar_arrive(item_empty + slot);
        st.aborted = st.aborted || *reinterpret_cast<volatile int *>(st.s_abort) != 0;
        if (item < 0 || st.aborted) break;
        int n, unit;
        place(item, n, unit);
        st.unit_geometry();
        st.thread_geometry();
        st.consume_unit(q);
        const int nit = st.z1 - st.z0;
        // the unit's last four u planes only fed the queue: release their slots
        __syncwarp();
        if (st.lane == 0)
            for (int s = 0; s < 4; ++s) mbar_arrive(st.empty_u + (st.useq + nit + 4 + s) % NU);
        st.useq += nit + 8;
        st.pseq += nit;
        // unit complete: its receivers' samples of u^{n+1}, then the flag
        consumer_barrier(THREADS);
        const StepArgs &a = a0;
        if (a.nrec > 0) {
            const T *uo = static_cast<const T *>(st.u_out_v);
            for (int r = f.rec_start[unit] + tid; r < f.rec_start[unit + 1]; r += THREADS) {
                const int ri = f.rec_list[r];
                const float v = ld_cg_value(uo + a.rec_off[ri]);
                a.traces[(long long)(n - a.rec_n0) * a.nrec + ri] = v;
                if (!isfinite(v)) atomicOr(a.err, DEV_ERR_NONFINITE);
            }
        }
        consumer_barrier(THREADS);
        // after an abort the unit's results are incomplete: no flag, so that
        // the units waiting for it give up as well
        if (tid == 0 && !*reinterpret_cast<volatile int *>(st.s_abort)) {
            __threadfence();
            st_release_gpu(f.done + unit, n + 1);
        }
    }
}

}  // namespace sgb
