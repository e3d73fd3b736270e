/*
 * seisgb: GB300 (sm_103a) library for the 3D acoustic-isotropic wave equation
 * with an 8th-order, 25-point star Laplacian and a fused PML boundary
 * (Sai, Mellor-Crummey, Meng, Araya-Polo, Meng, "Accelerating High-Order
 * Stencils on GPUs", arXiv 2009.04619).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Coordinates (i, j, k) index the computed domain, x fastest, z = depth
 *    (section IV-A stores the grid as a flat array with X innermost).  The
 *    computed domain is the inner region (nx, ny, nz) plus a PML of nb points
 *    on each side (section III-B): Nx = nx + 2 nb, likewise Ny, Nz.
 *  - Fields passed to stencil_step live in the padded layout reported by
 *    sgb_layout: a zero halo around the computed domain (8 points on the low x
 *    side, at least 4 elsewhere), rows padded to a multiple of 32 elements.
 *    The halo must hold zeros and is never written.
 *  - Every call returns SGB_OK (0) or a negative SGB_ERR_* code.  Arguments
 *    are validated before any GPU work is enqueued, so a rejected call leaves
 *    no partial state.  sgb_last_error() gives a message for the calling
 *    thread's most recent failure.
 *  - Device pointers are owned by the caller; the library never frees them.
 *  - "stream" is a cudaStream_t passed as void* (NULL = legacy default).
 */
#ifndef SEISGB_H
#define SEISGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SGB_OK 0
#define SGB_PENDING 1
#define SGB_ERR_INVALID_ARG (-1)
#define SGB_ERR_OUT_OF_MEMORY (-2)
#define SGB_ERR_UNSTABLE_DT (-3)
#define SGB_ERR_CUDA (-4)
#define SGB_ERR_TIMEOUT (-5)
#define SGB_ERR_NONFINITE (-6)
#define SGB_ERR_REJECTED (-7)
#define SGB_ERR_CANCELLED (-8)

/* Wavefield storage formats (arithmetic is always fp32).  The _DIFF formats
 * keep the leapfrog state of Eq. 2 as (u^n, d^n = u^n - u^{n-1}) instead of
 * (u^n, u^{n-1}): the same scheme in exact arithmetic, but a rounding error
 * stored in u^n no longer also enters the time difference, so 16-bit storage
 * loses far less accuracy.  They take a third wavefield: run_shot (one launch
 * per step) and stencil_step_diff.  SGB_FP16_DIFF is the scaled fp16 form
 * (a power-of-two scale for u and one for d, kept by the library): run_shot
 * only. */
#define SGB_FP32 0
#define SGB_FP16_SCALED 1
#define SGB_BF16 2
#define SGB_FP32_DIFF 3
#define SGB_BF16_DIFF 4
#define SGB_FP16_DIFF 5

/* Problem statement (section III-B: inner-region size and PML width are
 * inputs; Eq. 2: spacing and dt). */
typedef struct {
    int32_t nx, ny, nz;  /* inner-region points, each >= 1 */
    int32_t nb;          /* PML width per side in points, >= 0 (0: zero walls) */
    float dx, dy, dz;    /* grid spacing, metres, > 0 */
    float dt;            /* time step, seconds, > 0 */
    float vmax;          /* velocity (m/s) that sets the PML damping strength
                            eta_max = -3 vmax ln(pml_r0) / (2 nb h); normally
                            the model's maximum velocity */
    float pml_r0;        /* PML target reflection coefficient in (0, 1];
                            1 switches the damping off */
    int32_t storage;     /* SGB_FP32, SGB_FP16_SCALED, SGB_BF16, SGB_FP32_DIFF,
                            SGB_BF16_DIFF (these two: run_shot and
                            stencil_step_diff) or SGB_FP16_DIFF (run_shot) */
    int32_t schedule;    /* how run_shot launches its time loop (SGB_SCHED_*);
                            every schedule gives the same bits.  Other entry
                            points ignore it. */
} sgb_grid;

/* run_shot time-loop schedules (the arithmetic per point is the same in all):
 *  SGB_SCHED_AUTO   the library's choice (SGB_SCHED_STEP, measured fastest);
 *  SGB_SCHED_STEP   one launch per step, replayed in CUDA graphs of 32 steps;
 *  SGB_SCHED_PAIRS  temporal blocking: two steps per pass over HBM on the
 *                   PML-free interior, see stencil_step2 (SGB_FP32 only);
 *  SGB_SCHED_FLOW   one persistent launch for the whole time loop: CTAs take
 *                   (step, tile) items in order and start an item as soon as
 *                   its neighbouring tiles have finished the previous step
 *                   (no per-step tail; SGB_FP32 and SGB_BF16). */
#define SGB_SCHED_AUTO 0
#define SGB_SCHED_STEP 1
#define SGB_SCHED_PAIRS 2
#define SGB_SCHED_FLOW 3

/* Padded device layout of one field (element counts; multiply by the element
 * size for bytes). */
typedef struct {
    int32_t Nx, Ny, Nz;   /* computed extents */
    int32_t halo_lo_x;    /* zero points before computed x = 0 (8) */
    int32_t halo;         /* zero points before y = 0 and z = 0 (4) */
    int64_t sx, sy, sz;   /* padded extents: row pitch, rows per plane, planes */
    int64_t stride_y;     /* = sx */
    int64_t stride_z;     /* = sx * sy */
    int64_t origin;       /* element offset of computed point (0, 0, 0) */
    int64_t elems;        /* elements per field = sx * sy * sz */
} sgb_layout_info;

/* Point source: f = w(t) delta(x - x_s), added into u^{n+1} as
 * m(x_s) w(n dt) / (dx dy dz) (Eq. 2 right-hand side, Algorithm 1). */
typedef struct {
    int32_t i, j, k;        /* computed coordinates, inside the inner region */
    const float *wavelet;   /* device array of w(n dt); element [step] is used */
} sgb_source;

/* Receivers sample u^{n+1} after source injection. */
typedef struct {
    int32_t nrec;
    const int32_t *ijk;     /* HOST array nrec x 3 of computed coordinates */
    float *traces;          /* device array of nrec floats receiving the samples */
} sgb_receivers;

/* Fill *out with the padded layout of g.  INVALID_ARG on bad extents. */
int sgb_layout(const sgb_grid *g, sgb_layout_info *out);

/* Largest stable dt for velocities up to vmax: the von Neumann limit of the
 * leapfrog step of Eq. 2 with the 25-point Laplacian,
 * 2 / (vmax sqrt((2048/315) (dx^-2 + dy^-2 + dz^-2))). */
int sgb_cfl_dt(const sgb_grid *g, float vmax, float *dt_max);

/* One time step (Eq. 2 in the inner region, the PML update outside it, one
 * launch).  Reads u_cur = u^n and u_prev_to_next = u^{n-1}; overwrites
 * u_prev_to_next with u^{n+1} (the update is pointwise in u^{n-1}, so this is
 * safe).  m = V^2 dt^2 (fp32, padded layout).  phi: the PML auxiliary field,
 * fp32 padded layout, read and written at PML points only (start from zeros).
 * The u fields hold g->storage elements in the padded layout: fp32
 * (SGB_FP32) or bf16 (SGB_BF16, stored with stochastic rounding, arithmetic
 * in fp32); SGB_FP16_SCALED fields go through stencil_step_scaled and the
 * difference-form formats through stencil_step_diff (INVALID_ARG here).  step
 * selects src->wavelet[step].
 * src and rec may be NULL.  All device pointers must be 16-byte aligned.
 * Asynchronous on stream.  UNSTABLE_DT when g->dt exceeds the CFL limit for
 * g->vmax.  A bounded kernel wait that gave up or a non-finite receiver sample
 * sets a bit of this device's stencil_step error word, which
 * sgb_device_status reads and clears. */
int stencil_step(const sgb_grid *g, const void *u_cur, void *u_prev_to_next, const float *m,
                 float *phi, int32_t step, const sgb_source *src, const sgb_receivers *rec,
                 void *stream);

/* stencil_step for fp16 wavefields with a per-field power-of-two scale
 * (g->storage == SGB_FP16_SCALED; the paper fixes no precision, this is the
 * reduced-precision storage form of the same step).  A stored value is u / s.
 * scale_state: device float[8], 16-byte aligned, owned by the caller:
 * [0..3] = s of u^k at index k & 3, [4..7] = max |u^k| at index k & 3.  The
 * step for `step` = n reads s and max of u^n and u^{n-1}, picks s of u^{n+1}
 * (the power of two that keeps 4 max(max|u^n|, max|u^{n-1}|) plus the
 * injected amplitude below 2^14 s), writes it to [(n+1) & 3], zeroes
 * [4 + ((n+2) & 3)] and accumulates max |u^{n+1}| into [4 + ((n+1) & 3)].
 * Start a run from zero fields with {1, 1, 1, 1, 0, 0, 0, 0}.  Receivers
 * sample u^{n+1} times its scale.  Otherwise as stencil_step. */
int stencil_step_scaled(const sgb_grid *g, const void *u_cur, void *u_prev_to_next,
                        const float *m, float *phi, float *scale_state, int32_t step,
                        const sgb_source *src, const sgb_receivers *rec, void *stream);

/* One step of Eq. 2 in difference form (g->storage SGB_FP32_DIFF or
 * SGB_BF16_DIFF, padded fields of fp32 or bf16 elements): the leapfrog state
 * is u^n and d^n = u^n - u^{n-1}.  Reads u_cur = u^n and d = d^n; writes
 * d^{n+1} = d^n + m L u^n (PML points: [(1 - e) d^n + m (L u^n + phi^n)
 * - e^2 u^n] / (1 + e) with e = eta dt; the source term added to d^{n+1}) over
 * d in place, and u^{n+1} = u^n + d^{n+1} into u_next.  The same scheme as
 * stencil_step in exact arithmetic; stored 16-bit values lose much less
 * because a rounding of u no longer enters the time difference.  u_cur,
 * u_next and d must be distinct, 16-byte aligned device buffers of
 * sgb_layout().elems elements; m and phi as for stencil_step.  Receivers sample
 * u^{n+1}.  Returns INVALID_ARG (nothing launched) for other storage formats,
 * a NULL d, or d equal to u_cur or u_next; otherwise as stencil_step. */
int stencil_step_diff(const sgb_grid *g, const void *u_cur, void *u_next, void *d,
                      const float *m, float *phi, int32_t step, const sgb_source *src,
                      const sgb_receivers *rec, void *stream);

/* Two time steps, n and n + 1, with temporal blocking (the 3.5D blocking
 * that the paper names as future work, section VI): on the box B = the inner
 * region shrunk by the stencil radius on every side (x bounds rounded inwards
 * to multiples of 4) one kernel reads u^{n-1}, u^n and m once and writes
 * u^{n+1} and u^{n+2} (the first step evaluated on each tile plus a radius-4
 * halo, the second on the tile); the rest of the grid (the PML and the inner
 * band next to it) takes two ordinary fused steps (Eq. 2 and the PML update,
 * phi updated in place).  The results are bit-identical to two stencil_step
 * calls.  All fields fp32 in the padded layout (storage SGB_FP32), 16-byte
 * aligned; u_prev = u^{n-1}, u_cur = u^n are read, u_next = u^{n+1} and
 * u_next2 = u^{n+2} written: four distinct buffers (INVALID_ARG when an
 * output overlaps an input, another output or phi).  src->wavelet[step] and
 * [step + 1] are injected.  No receivers (gather them from u_next and
 * u_next2).  Three launches on stream, asynchronous; errors are recorded in
 * the device error word of stencil_step (sgb_device_status). */
int stencil_step2(const sgb_grid *g, const float *u_prev, const float *u_cur, float *u_next,
                  float *u_next2, const float *m, float *phi, int32_t step,
                  const sgb_source *src, void *stream);

/* A whole shot (Algorithm 1): u^0 = u^{-1} = 0, nt steps, source injection and
 * receiver sampling every step.
 *   velocity  Nz*Ny*Nx fp32 compact (x fastest), host or device
 *   wavelet   nt fp32, host or device
 *   src_ijk   host int32[3] (NULL: no source)
 *   rec_ijk   host int32[nrec*3]
 *   traces    nt*nrec fp32, host or device; traces[n*nrec + r] = u^{n+1}(rec_r)
 *   final_u   Nz*Ny*Nx fp32 compact u^{nt}, host or device, or NULL
 * Scratch (two wavefields, phi, m, a device error word of this call's own)
 * comes from a library-owned stream-ordered pool and is released before
 * returning.  Enqueued on stream, then the call waits for the stream.
 * INVALID_ARG if traces or final_u overlaps velocity, wavelet or each other;
 * UNSTABLE_DT if dt exceeds the CFL limit of the model's actual maximum
 * velocity; NONFINITE if a receiver saw a NaN/Inf (traces are still written);
 * TIMEOUT if a kernel's bounded wait gave up.  Calls on different streams are
 * independent. */
int run_shot(const sgb_grid *g, const float *velocity, const float *wavelet, int32_t nt,
             const int32_t *src_ijk, const int32_t *rec_ijk, int32_t nrec, float *traces,
             float *final_u, void *stream);

/* Steps n_begin .. n_end-1 of a shot (Algorithm 1), resumable: the state
 * before step n_begin -- u_cur = u^{n_begin}, u_prev = u^{n_begin - 1}, phi =
 * phi^{n_begin}, each Nz*Ny*Nx fp32 compact, host or device -- is read, and
 * overwritten with the state before step n_end.  Zero arrays at n_begin = 0
 * start a shot.  A shot run as segments [0, k), [k, nt) with the state passed
 * along gives the same bits as run_shot over [0, nt), whatever k (the source
 * and, for bf16, the stochastic rounding use the absolute step).  Stored
 * fields round to g->storage (SGB_FP32 or SGB_BF16; SGB_FP16_SCALED is
 * rejected: its scale is not part of the state).  wavelet holds samples for
 * the absolute steps (at least n_end); traces receives n_end - n_begin rows,
 * traces[(n - n_begin)*nrec + r] = u^{n+1}(rec_r).  SGB_SCHED_PAIRS runs as
 * SGB_SCHED_STEP here.  Otherwise as run_shot (the state arrays may not
 * overlap each other, velocity, wavelet or traces). */
int run_shot_segment(const sgb_grid *g, const float *velocity, const float *wavelet,
                     int32_t n_begin, int32_t n_end, const int32_t *src_ijk,
                     const int32_t *rec_ijk, int32_t nrec, float *traces, float *u_cur,
                     float *u_prev, float *phi, void *stream);

/* Trace misfit J = 1/2 sum_{n,r} (d^n_r - observed^n_r)^2 of a shot (d as in
 * run_shot) and its gradient dJ/dv with respect to the velocity model, by the
 * exact discrete adjoint of the fused step including the PML and the source
 * (the paper has no adjoint; the derivation is in the oracle and the design
 * notes).  The forward run keeps (u^n, u^{n-1}, phi^n) every ckpt_every steps
 * (0: 100); the backward sweep recomputes each segment's forward steps and
 * runs the adjoint steps over it.  The misfit sum is fp64; the time sum of the
 * gradient is fp32 per point over blocks of 32 steps (counted from step 0, so
 * the result does not depend on ckpt_every) and fp64 across blocks;
 * everything else fp32 (SGB_FP32 storage only).
 *   velocity  Nz*Ny*Nx fp32 compact, host or device
 *   wavelet   nt fp32, host or device;  src_ijk, rec_ijk: host
 *   observed  nt*nrec fp32 (same layout as run_shot's traces), host or device
 *   misfit_out     host double
 *   grad_velocity  Nz*Ny*Nx fp64 compact, host or device
 * Calls on different streams (e.g. one host thread per stream) run
 * concurrently and independently: each call has its own scratch and its own
 * device error word.
 * Scratch: 9 padded fp32 fields and one fp64 field, ceil(nt / ckpt_every) x 3
 * checkpoint fields and
 * ckpt_every recomputation fields, from the library pool.  Synchronous. */
int adjoint_shot(const sgb_grid *g, const float *velocity, const float *wavelet, int32_t nt,
                 const int32_t *src_ijk, const int32_t *rec_ijk, int32_t nrec,
                 const float *observed, int32_t ckpt_every, double *misfit_out,
                 double *grad_velocity, void *stream);

/* Allocation-free variant of run_shot (the paper has no counterpart).  For
 * callers that cannot allocate device memory once running -- e.g. a serving
 * process whose device memory is all held by another allocator's pool, or a
 * real-time loop that forbids cudaMalloc/cudaFree after start-up.  Same
 * arguments, results and kernels as run_shot, except:
 *  - velocity, wavelet, traces and final_u must be DEVICE pointers (rec_ijk and
 *    src_ijk stay host arrays); nothing is allocated: all scratch (two
 *    wavefields, phi, m, receiver tables) lives in one fixed 32 MiB device
 *    array inside this library, which every GPU that loads the library holds
 *    until the process exits;
 *  - grids whose scratch does not fit (about 2 M padded points per field, e.g.
 *    up to ~120^3 computed points) are rejected with SGB_ERR_INVALID_ARG and a
 *    message naming the size;
 *  - the first call on a device resolves the array's device address (set-up);
 *    make that first call before any stream capture;
 *  - all calls share the array and it keeps the previous call's contents (each
 *    call clears what must start at zero, including the error word it keeps
 *    there); calls whose GPU work overlaps, on any streams, race on it and give
 *    wrong results or statuses;
 *  - like run_shot, outputs that overlap an input or each other are rejected;
 *  - the time loop is launched directly, one kernel per step (no CUDA graph). */
int run_shot_noalloc(const sgb_grid *g, const float *velocity, const float *wavelet, int32_t nt,
                     const int32_t *src_ijk, const int32_t *rec_ijk, int32_t nrec, float *traces,
                     float *final_u, void *stream);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching of shot requests (no counterpart in the paper;
 * every shot is Algorithm 1 on its own grid).  A server owns one GPU (the
 * current device at serve_create), a stream and a scheduler thread.  Requests
 * are admitted in FIFO order whenever a slot is free and the server's HBM
 * budget can hold their footprint; all resident shots, whatever their grid
 * sizes, advance together in replays of one CUDA graph that holds, for every
 * resident shot, a branch of steps_per_graph fused-step launches on that shot's
 * own grid; the branches run concurrently on the GPU.  Shots join and leave
 * between graph replays.  A shot's results equal run_shot's for the same
 * request, bit for bit.
 * ------------------------------------------------------------------------- */
typedef struct {
    uint64_t hbm_budget_bytes;  /* device memory the resident shots may hold */
    int32_t max_slots;          /* shots resident at once, 1..64 */
    int32_t steps_per_graph;    /* time steps per CUDA-graph replay, 1..256 */
} sgb_serve_config;

typedef struct {
    sgb_grid grid;              /* storage must be SGB_FP32; dt within the CFL
                                   limit of the model's maximum velocity */
    const float *velocity;      /* host, Nz*Ny*Nx compact, copied at submit */
    const float *wavelet;       /* host, nt samples, copied at submit */
    int32_t nt;                 /* time steps, >= 1 */
    int32_t src_ijk[3];         /* source, inside the inner region */
    const int32_t *rec_ijk;     /* host, nrec*3, copied at submit */
    int32_t nrec;               /* >= 1 */
} sgb_shot_request;

typedef struct {
    uint64_t ticket;
    int32_t status;             /* SGB_OK or the error that ended the shot:
                                   TIMEOUT (a kernel wait gave up), NONFINITE (a
                                   receiver sampled NaN/Inf), OUT_OF_MEMORY,
                                   CUDA_ERROR, CANCELLED (serve_cancel); each
                                   shot has its own device error word */
    int32_t nt, nrec;
    float *traces;              /* caller buffer of nt*nrec floats (or NULL);
                                   filled when serve_poll returns SGB_OK and
                                   status is SGB_OK or SGB_ERR_NONFINITE */
    double queue_ms;            /* submit -> admission */
    double latency_ms;          /* submit -> traces on the host */
} sgb_shot_result;

typedef struct {
    uint64_t submitted, completed, rejected;
    int32_t resident, queued;
    uint64_t graph_replays, step_launches;
    uint64_t device_bytes;      /* bytes held by resident shots */
    /* scheduler-thread time (ms, cumulative): setting up admitted shots (host
     * side; their copies overlap the running replays), uploading the shot
     * table and re-capturing the replay graph, retiring finished shots, and
     * waiting for enqueued replays to finish */
    double setup_ms, prepare_ms, retire_ms, wait_ms;
    uint64_t cancelled;         /* requests ended by serve_cancel */
} sgb_serve_stats;

typedef struct sgb_server sgb_server;

/* Device bytes a request holds while resident: four padded fp32 fields
 * (u^n, u^{n-1}, phi, m), the velocity upload, wavelet, receiver table and
 * traces.  Pure host arithmetic. */
int serve_footprint(const sgb_grid *g, int32_t nt, int32_t nrec, uint64_t *bytes);
/* Start a server on the current device.  OUT_OF_MEMORY / CUDA_ERROR on failure. */
int serve_create(const sgb_serve_config *cfg, sgb_server **out);
/* Queue a request (deep-copied; the caller's buffers may be reused at once).
 * REJECTED if its footprint exceeds the whole budget, INVALID_ARG /
 * UNSTABLE_DT on a bad request (checked before queueing). */
int serve_submit(sgb_server *s, const sgb_shot_request *req, uint64_t *ticket);
/* Result of a ticket.  SGB_OK: done, *out filled and traces copied (the ticket
 * is then forgotten).  SGB_PENDING: not done and timeout_us == 0.
 * SGB_ERR_TIMEOUT: not done within timeout_us (> 0).  INVALID_ARG: unknown. */
int serve_poll(sgb_server *s, uint64_t ticket, sgb_shot_result *out, int32_t timeout_us);
/* Cancel a request.  Queued: it ends at once with status SGB_ERR_CANCELLED.
 * Admitted: it is retired when the replays already enqueued finish (its
 * device memory returns to the pool; no traces).  Finished already: no effect
 * (its result stands).  The result is collected with serve_poll as usual.
 * INVALID_ARG for an unknown ticket. */
int serve_cancel(sgb_server *s, uint64_t ticket);
/* Copy of the server's counters (taken under the server's lock, so the fields
 * are consistent with each other); INVALID_ARG if s or out is NULL. */
int serve_stats(sgb_server *s, sgb_serve_stats *out);
/* Cancel queued requests, finish resident shots, stop the scheduler, free all
 * device memory. */
int serve_destroy(sgb_server *s);

/* Layout conversion between compact (Nz, Ny, Nx) fp32 arrays and the padded
 * layout (device pointers; pack zeroes the halo).  Asynchronous on stream. */
int sgb_pack(const sgb_grid *g, const float *compact, float *padded, void *stream);
int sgb_unpack(const sgb_grid *g, const float *padded, float *compact, void *stream);

/* Reads and clears, in one atomic step on the device, the current device's
 * stencil_step error word (set when a bounded kernel wait gave up or a
 * receiver sampled NaN/Inf); synchronises stream.  Returns SGB_OK,
 * SGB_ERR_TIMEOUT, SGB_ERR_NONFINITE or SGB_ERR_CUDA.  Other entry points
 * report through error words of their own and are not seen here. */
int sgb_device_status(void *stream);

/* Self-test of the failure detection the step kernels use (no counterpart in
 * the paper): launches one kernel whose bounded wait on an mbarrier that
 * nothing completes -- the wait of a step whose TMA copies never land -- gives
 * up after limit_us microseconds (1..2,000,000) and sets the timeout bit of an
 * error word of the call's own, which the host then reads.  *status_out
 * receives that status (SGB_ERR_TIMEOUT when detection works); the return
 * value is SGB_OK unless the arguments are invalid or the launch failed.  No
 * GPU fault is involved and the context stays usable.  Synchronises stream. */
int sgb_selftest_wait_timeout(int32_t limit_us, int32_t *status_out, void *stream);

/* Test hook (no counterpart in the paper; process-wide): counting the
 * library's device-pool allocations from this call on, numbers after ..
 * after + count - 1 fail with SGB_ERR_OUT_OF_MEMORY as an exhausted device
 * would (host-side: no device fault is involved); the others succeed.  count
 * 0 disarms.  Calls that fail this way leave no partial state: their scratch
 * returns to the pool; a served shot whose set-up fails ends with status
 * SGB_ERR_OUT_OF_MEMORY and the others run on. */
int sgb_debug_fail_allocations(int64_t after, int64_t count);

/* Bytes currently allocated from the current device's library pool (scratch
 * of calls in flight, resident served shots). */
int sgb_pool_used_bytes(int64_t *bytes);

/* Number of this library's kernels launched by the calling thread since the
 * last reset (graph replays count every kernel node). */
int64_t sgb_launch_count(int reset);

/* Message for the calling thread's most recent error ("" if none). */
const char *sgb_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SEISGB_H */
