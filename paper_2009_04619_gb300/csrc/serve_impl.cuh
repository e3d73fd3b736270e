// Shot server: continuous batching of shot requests on one GPU.
//
// Included at the end of seisgb.cu (it uses that file's validation, layout,
// tensor-map and launch helpers).  Each shot is Algorithm 1 on its own grid;
// nothing in the paper covers serving.
//
// - serve_submit deep-copies the request, checks it (arguments, CFL of the
//   model's maximum velocity, footprint vs. the whole budget) and queues it.
// - The scheduler thread admits queued requests in FIFO order while a slot is
//   free and the budget holds the head's footprint, sets their fields up on a
//   second stream while the current replays run, and advances every resident
//   shot with replays of one CUDA graph.  The graph has one branch per resident
//   shot: steps_per_graph launches of the fused step on that shot's own grid
//   and decomposition (arguments and tensor maps in the kernel's parameter
//   space, as in run_shot), then an increment of the shot's device step
//   counter.  The branches are independent, so the shots' kernels run
//   concurrently and fill each other's partial waves; shots of different grid
//   sizes share the GPU.
// - Each launch reads its step from the shot's counter and chooses the
//   buffers and tensor maps of that step's parity, so a replay of any length
//   repeats.  A shot of nt steps takes nt + 1 launches (the last samples the
//   receivers of the last step); launches past that return at once.
// - Composition changes (admission, retirement) happen between replays; the
//   graph is re-captured only then.  Retired shots' traces are copied to the
//   host and their device memory returned to the pool.
// - The host enqueues several replays back to back and waits only where the
//   composition can change: up to the next shot completion when no request can
//   be admitted (slots full), at most MAX_AHEAD_OPEN replays while slots are
//   free (new arrivals wait at most that long), one replay while an admission
//   is set up.
#pragma once
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <thread>

namespace {

constexpr int SERVE_MAX_SLOTS = 64;
constexpr int MAX_AHEAD_OPEN = 4;     // replays enqueued at once while slots are free
constexpr int MAX_AHEAD_FULL = 256;   // ... while every slot is taken

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b)
{
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Shot {
    uint64_t ticket = 0;
    sgb_grid g;
    sgb_layout_info L;
    int nt = 0, nrec = 0;
    int src[3] = {0, 0, 0};
    std::vector<float> vel, wav, traces;
    std::vector<int32_t> rec;
    uint64_t footprint = 0;
    int status = SGB_OK;
    std::atomic<bool> cancel{false};  // serve_cancel on an admitted shot
    // device
    float *u0 = nullptr, *u1 = nullptr, *phi = nullptr, *m = nullptr, *d_vel = nullptr,
          *d_wav = nullptr, *d_tr = nullptr;
    long long *d_off = nullptr;
    int *d_err = nullptr;   // this shot's device error word (timeouts, non-finite samples)
    int *d_step = nullptr;  // this shot's device step counter (step of a replay's first launch)
    StepArgs args;          // step constants, fields, source, receivers, decomposition
    StepMaps maps[2];       // [parity of n]
    int grid = 0;           // work units per step
    int n0 = 0;             // next step to run
    Clock::time_point t_submit, t_admit, t_done;
};

uint64_t shot_footprint(const sgb_layout_info &L, int nt, int nrec)
{
    const uint64_t f = (uint64_t)L.elems * 4;
    const uint64_t ncomp = (uint64_t)L.Nx * L.Ny * L.Nz;
    return 4 * f + ncomp * 4 + (uint64_t)nt * 4 + (uint64_t)nrec * 8 + (uint64_t)nt * nrec * 4;
}

}  // namespace

struct sgb_server {
    sgb_serve_config cfg;
    int device = 0;
    DevState *ds = nullptr;
    cudaStream_t stream = nullptr;        // replays, table uploads, retirement
    cudaStream_t setup_stream = nullptr;  // admissions, overlapped with replays
    cudaEvent_t setup_done = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Shot *> queue;
    std::vector<Shot *> resident;
    std::map<uint64_t, Shot *> done;
    std::map<uint64_t, bool> known;  // ticket -> pending
    std::map<uint64_t, Shot *> live; // submitted, not yet done
    uint64_t next_ticket = 1, budget_used = 0;
    bool stop = false;
    std::thread th;
    sgb_serve_stats stats;
    // the graph of the current composition: one branch (stream) per resident shot
    cudaGraphExec_t exec = nullptr;
    bool composition_changed = true;
    cudaStream_t branch[SERVE_MAX_SLOTS] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[SERVE_MAX_SLOTS] = {};
};

namespace {

void free_shot_device(sgb_server *sv, Shot *sh)
{
    float **ptrs[] = {&sh->u0, &sh->u1, &sh->phi, &sh->m, &sh->d_vel, &sh->d_wav, &sh->d_tr};
    for (float **p : ptrs)
        if (*p) {
            cudaFreeAsync(*p, sv->stream);
            *p = nullptr;
        }
    if (sh->d_off) {
        cudaFreeAsync(sh->d_off, sv->stream);
        sh->d_off = nullptr;
    }
    for (int **p : {&sh->d_err, &sh->d_step})
        if (*p) {
            cudaFreeAsync(*p, sv->stream);
            *p = nullptr;
        }
}

// Fields, m, receiver table and step arguments of a newly admitted shot
// (enqueued on the server's stream).
int setup_shot(sgb_server *sv, Shot *sh)
{
    const sgb_layout_info &L = sh->L;
    cudaStream_t st = sv->setup_stream;
    const size_t fbytes = (size_t)L.elems * 4;
    const long long ncomp = (long long)L.Nx * L.Ny * L.Nz;
    auto get = [&](void **p, size_t b) -> int {
        if (injected_alloc_failure())
            return fail(SGB_ERR_OUT_OF_MEMORY, "serve: allocation of %zu bytes failed (injected)", b);
        cudaError_t e = cudaMallocFromPoolAsync(p, b ? b : 16, sv->ds->pool, st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(SGB_ERR_OUT_OF_MEMORY, "serve: allocation of %zu bytes failed", b);
        }
        return SGB_OK;
    };
    int rc;
    if ((rc = get((void **)&sh->u0, fbytes)) || (rc = get((void **)&sh->u1, fbytes)) ||
        (rc = get((void **)&sh->phi, fbytes)) || (rc = get((void **)&sh->m, fbytes)) ||
        (rc = get((void **)&sh->d_vel, (size_t)ncomp * 4)) ||
        (rc = get((void **)&sh->d_wav, (size_t)sh->nt * 4)) ||
        (rc = get((void **)&sh->d_tr, (size_t)sh->nt * sh->nrec * 4)) ||
        (rc = get((void **)&sh->d_off, (size_t)sh->nrec * 8)) ||
        (rc = get((void **)&sh->d_err, sizeof(int))) || (rc = get((void **)&sh->d_step, sizeof(int))))
        return rc;
    std::vector<long long> off(sh->nrec);
    for (int r = 0; r < sh->nrec; ++r)
        off[r] = L.origin + (long long)sh->rec[3 * r + 2] * L.stride_z +
                 (long long)sh->rec[3 * r + 1] * L.sx + sh->rec[3 * r];
    CUDA_TRY(cudaMemcpyAsync(sh->d_vel, sh->vel.data(), (size_t)ncomp * 4, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(sh->d_wav, sh->wav.data(), (size_t)sh->nt * 4, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(sh->d_off, off.data(), (size_t)sh->nrec * 8, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemsetAsync(sh->d_err, 0, sizeof(int), st));
    CUDA_TRY(cudaMemsetAsync(sh->d_step, 0, sizeof(int), st));
    CUDA_TRY(cudaMemsetAsync(sh->u0, 0, fbytes, st));
    CUDA_TRY(cudaMemsetAsync(sh->u1, 0, fbytes, st));
    CUDA_TRY(cudaMemsetAsync(sh->phi, 0, fbytes, st));
    CUDA_TRY(cudaMemsetAsync(sh->m, 0, fbytes, st));
    make_m_kernel<<<ew_grid(ncomp, *sv->ds), 256, 0, st>>>(pad_geom(L), sh->d_vel, sh->g.dt, sh->m);
    CUDA_TRY(cudaGetLastError());
    ++t_launches;
    // the pageable copies above are staged before they return; wait for them so
    // the host copies can be released
    CUDA_TRY(cudaStreamSynchronize(st));
    cudaFreeAsync(sh->d_vel, st);
    sh->d_vel = nullptr;
    std::vector<float>().swap(sh->vel);

    StepArgs &a = sh->args;
    fill_step_constants(&sh->g, L, a);
    a.phi = sh->phi;
    a.err = sh->d_err;
    a.si = sh->src[0];
    a.sj = sh->src[1];
    a.sk = sh->src[2];
    a.wavelet = sh->d_wav;
    a.nrec = sh->nrec;
    a.rec_off = sh->d_off;
    a.traces = sh->d_tr;
    // the shot's own decomposition, as run_shot would choose it
    choose_decomposition(L.Nx, L.Ny, L.Nz, sv->ds->sms, sv->ds->occ, a, &sh->grid);
    float *buf[2] = {sh->u0, sh->u1};  // buf[0] = u^{-1}, buf[1] = u^0
    for (int p = 0; p < 2; ++p)  // step n reads buf[(n+1)&1], writes buf[n&1]
        if ((rc = encode_step_maps<float>(sh->maps[p], buf[(p + 1) & 1], buf[p & 1], sh->m, sh->phi, L)))
            return rc;
    sh->n0 = 0;
    return SGB_OK;
}

// Retire a finished shot: its error word decides its status (a kernel wait
// that timed out, a receiver that sampled NaN/Inf); traces to the host, device
// memory back to the pool.
int retire_shot(sgb_server *sv, Shot *sh)
{
    sh->traces.resize((size_t)sh->nt * sh->nrec);
    int rc = SGB_OK;
    if (sh->status == SGB_OK && sh->cancel) sh->status = SGB_ERR_CANCELLED;
    if (sh->status == SGB_OK) {
        int v = 0;
        cudaError_t e = cudaMemcpyAsync(&v, sh->d_err, sizeof(int), cudaMemcpyDeviceToHost,
                                        sv->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(sh->traces.data(), sh->d_tr, sh->traces.size() * 4,
                                cudaMemcpyDeviceToHost, sv->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(sv->stream);
        if (e != cudaSuccess) {
            sh->status = SGB_ERR_CUDA;
            rc = fail(SGB_ERR_CUDA, "serve: trace copy failed: %s", cudaGetErrorString(e));
        } else if (v & DEV_ERR_TIMEOUT) {
            sh->status = SGB_ERR_TIMEOUT;
        } else if (v & DEV_ERR_NONFINITE) {
            sh->status = SGB_ERR_NONFINITE;
        } else if (v) {
            sh->status = SGB_ERR_CUDA;
        }
    }
    free_shot_device(sv, sh);
    sh->t_done = Clock::now();
    return rc;
}

// (Re)capture the replay graph when the composition changed: one branch per
// resident shot with steps_per_graph launches and the counter increment.
int prepare_replay(sgb_server *sv)
{
    if (!sv->composition_changed && sv->exec) return SGB_OK;
    if (sv->exec) {
        cudaGraphExecDestroy(sv->exec);
        sv->exec = nullptr;
    }
    const int S = sv->cfg.steps_per_graph;
    cudaStream_t cs;
    CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) {
        ce = cudaEventRecord(sv->ev_fork, cs);
        for (size_t i = 0; i < sv->resident.size() && ce == cudaSuccess; ++i) {
            Shot *sh = sv->resident[i];
            cudaStream_t bs = sv->branch[i];
            ce = cudaStreamWaitEvent(bs, sv->ev_fork, 0);
            const StepMaps &p0 = sh->maps[0], &p1 = sh->maps[1];
            for (int k = 0; k < S && ce == cudaSuccess; ++k) {
                ShotRun r;
                r.buf[0] = sh->u0;
                r.buf[1] = sh->u1;
                r.step_ptr = sh->d_step;
                r.step_add = k;
                r.n_end = sh->nt;
                ce = launch_dependent(shot_step_kernel<Cfg>, sh->grid, Cfg::BLOCK,
                                      Stage<Cfg, float>::SMEM_BYTES, bs, sh->args, r, p0.ucur,
                                      p0.ucur_in, p0.uprev, p0.m, p0.phi, p1.ucur, p1.ucur_in,
                                      p1.uprev, p1.m, p1.phi);
            }
            if (ce == cudaSuccess) {
                advance_kernel<<<1, 32, 0, bs>>>(sh->d_step, S);
                ce = cudaGetLastError();
            }
            if (ce == cudaSuccess) ce = cudaEventRecord(sv->ev_join[i], bs);
            if (ce == cudaSuccess) ce = cudaStreamWaitEvent(cs, sv->ev_join[i], 0);
        }
        cudaError_t ee = cudaStreamEndCapture(cs, &graph);
        if (ce == cudaSuccess) ce = ee;
    }
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&sv->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    CUDA_TRY(ce);
    sv->composition_changed = false;
    return SGB_OK;
}

void scheduler(sgb_server *sv)
{
    cudaSetDevice(sv->device);
    const int S = sv->cfg.steps_per_graph;
    for (;;) {
        std::vector<Shot *> admit;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            // FIFO admission by slots and HBM budget
            while (!sv->queue.empty()) {
                Shot *h = sv->queue.front();
                if ((int)(sv->resident.size() + admit.size()) >= sv->cfg.max_slots) break;
                if (sv->budget_used + h->footprint > sv->cfg.hbm_budget_bytes) break;
                sv->queue.pop_front();
                sv->budget_used += h->footprint;
                admit.push_back(h);
            }
            if (sv->resident.empty() && admit.empty()) {
                if (sv->stop) break;
                sv->cv_work.wait(lk, [&] { return sv->stop || !sv->queue.empty(); });
                continue;
            }
            sv->stats.queued = (int)sv->queue.size();
        }
        // 1. replay the resident shots (asynchronous), R replays back to back
        int rc = SGB_OK;
        cudaError_t e = cudaSuccess;
        const bool replay = !sv->resident.empty();
        int R = 1;
        if (replay && admit.empty()) {
            int to_finish = MAX_AHEAD_FULL;  // replays until the first resident shot is done
            for (Shot *sh : sv->resident)
                to_finish = std::min(to_finish, std::max(1, (sh->nt + 1 - sh->n0 + S - 1) / S));
            const bool open = (int)sv->resident.size() < sv->cfg.max_slots;
            R = open ? std::min(to_finish, MAX_AHEAD_OPEN) : to_finish;
        }
        Clock::time_point tp = Clock::now();
        double t_prep = 0.0, t_setup = 0.0, t_wait = 0.0, t_retire = 0.0;
        if (replay) {
            rc = prepare_replay(sv);
            t_prep = ms_between(tp, Clock::now());
            for (int r = 0; r < R && rc == SGB_OK && e == cudaSuccess; ++r)
                e = cudaGraphLaunch(sv->exec, sv->stream);
            t_launches += (int64_t)R * (S + 1) * (int64_t)sv->resident.size();
        }
        tp = Clock::now();
        // 2. meanwhile, set up the admitted shots on the setup stream; they join
        //    at the next replay
        std::vector<Shot *> joined;
        for (Shot *sh : admit) {
            sh->t_admit = Clock::now();
            int src = setup_shot(sv, sh);
            if (src != SGB_OK) {
                sh->status = src;
                cudaStreamSynchronize(sv->setup_stream);
                free_shot_device(sv, sh);
                sh->t_done = Clock::now();
                std::lock_guard<std::mutex> lk(sv->mu);
                sv->budget_used -= sh->footprint;
                sv->done[sh->ticket] = sh;
                sv->live.erase(sh->ticket);
                sv->cv_done.notify_all();
                continue;
            }
            joined.push_back(sh);
        }
        if (!joined.empty()) {
            cudaEventRecord(sv->setup_done, sv->setup_stream);
            cudaStreamWaitEvent(sv->stream, sv->setup_done, 0);
        }
        t_setup = ms_between(tp, Clock::now());
        tp = Clock::now();
        // 3. wait for the replay, advance and retire
        if (replay && e == cudaSuccess) e = cudaStreamSynchronize(sv->stream);
        t_wait = ms_between(tp, Clock::now());
        tp = Clock::now();
        std::vector<Shot *> keep, finished;
        if (replay) {
            for (Shot *sh : sv->resident) {
                sh->n0 += R * S;
                if (rc != SGB_OK || e != cudaSuccess) sh->status = SGB_ERR_CUDA;
                if (sh->n0 > sh->nt || sh->status != SGB_OK || sh->cancel) finished.push_back(sh);
                else keep.push_back(sh);
            }
        }
        for (Shot *sh : joined) {  // cancelled while being set up: never runs
            if (sh->cancel) {
                cudaStreamSynchronize(sv->setup_stream);
                finished.push_back(sh);
            } else {
                keep.push_back(sh);
            }
        }
        for (Shot *sh : finished) retire_shot(sv, sh);
        if (!finished.empty() || !joined.empty()) sv->composition_changed = true;
        t_retire = ms_between(tp, Clock::now());
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            if (replay) {
                sv->stats.graph_replays += R;
                sv->stats.step_launches += (uint64_t)R * S;
            }
            sv->stats.prepare_ms += t_prep;
            sv->stats.setup_ms += t_setup;
            sv->stats.wait_ms += t_wait;
            sv->stats.retire_ms += t_retire;
            sv->resident = keep;
            sv->stats.resident = (int)keep.size();
            for (Shot *sh : finished) {
                sv->budget_used -= sh->footprint;
                sv->done[sh->ticket] = sh;
                sv->live.erase(sh->ticket);
                if (sh->status == SGB_ERR_CANCELLED) sv->stats.cancelled += 1;
                else sv->stats.completed += 1;
            }
            sv->stats.device_bytes = sv->budget_used;
            if (!finished.empty()) sv->cv_done.notify_all();
        }
    }
}

}  // namespace

// Streams and events of a server (those that were created).
static void server_release_handles(sgb_server *sv)
{
    for (int i = 0; i < SERVE_MAX_SLOTS; ++i) {
        if (sv->branch[i]) cudaStreamDestroy(sv->branch[i]);
        if (sv->ev_join[i]) cudaEventDestroy(sv->ev_join[i]);
    }
    if (sv->ev_fork) cudaEventDestroy(sv->ev_fork);
    if (sv->setup_done) cudaEventDestroy(sv->setup_done);
    if (sv->setup_stream) cudaStreamDestroy(sv->setup_stream);
    if (sv->stream) cudaStreamDestroy(sv->stream);
}

extern "C" int serve_footprint(const sgb_grid *g, int32_t nt, int32_t nrec, uint64_t *bytes)
{
    sgb_layout_info L;
    int rc = check_grid(g, &L);
    if (rc) return rc;
    if (nt < 1 || nrec < 1 || !bytes) return fail(SGB_ERR_INVALID_ARG, "nt and nrec must be >= 1");
    *bytes = shot_footprint(L, nt, nrec);
    return SGB_OK;
}

extern "C" int serve_create(const sgb_serve_config *cfg, sgb_server **out)
{
    if (!cfg || !out) return fail(SGB_ERR_INVALID_ARG, "NULL argument");
    if (cfg->max_slots < 1 || cfg->max_slots > SERVE_MAX_SLOTS)
        return fail(SGB_ERR_INVALID_ARG, "max_slots must be in 1..%d", SERVE_MAX_SLOTS);
    if (cfg->steps_per_graph < 1 || cfg->steps_per_graph > 256)
        return fail(SGB_ERR_INVALID_ARG, "steps_per_graph must be in 1..256");
    if (cfg->hbm_budget_bytes == 0) return fail(SGB_ERR_INVALID_ARG, "hbm_budget_bytes is 0");
    DevState *ds;
    int rc = device_state(&ds);
    if (rc) return rc;
    CUDA_TRY(cudaFuncSetAttribute(shot_step_kernel<Cfg>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)Stage<Cfg, float>::SMEM_BYTES));
    sgb_server *sv = new sgb_server();
    sv->cfg = *cfg;
    sv->ds = ds;
    memset(&sv->stats, 0, sizeof sv->stats);
    cudaError_t e = cudaGetDevice(&sv->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->setup_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sv->setup_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sv->ev_fork, cudaEventDisableTiming);
    for (int i = 0; i < cfg->max_slots && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&sv->branch[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sv->ev_join[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        server_release_handles(sv);
        delete sv;
        return fail(e == cudaErrorMemoryAllocation ? SGB_ERR_OUT_OF_MEMORY : SGB_ERR_CUDA,
                    "serve_create: %s", cudaGetErrorString(e));
    }
    sv->th = std::thread(scheduler, sv);
    *out = sv;
    return SGB_OK;
}

extern "C" int serve_submit(sgb_server *sv, const sgb_shot_request *req, uint64_t *ticket)
{
    if (!sv || !req || !ticket) return fail(SGB_ERR_INVALID_ARG, "NULL argument");
    sgb_layout_info L;
    int rc = check_grid(&req->grid, &L);
    if (rc) return rc;
    const sgb_grid *g = &req->grid;
    if (g->storage != SGB_FP32) return fail(SGB_ERR_INVALID_ARG, "serve: SGB_FP32 storage only");
    if (!req->velocity || !req->wavelet || !req->rec_ijk)
        return fail(SGB_ERR_INVALID_ARG, "serve: NULL request buffer");
    if (req->nt < 1 || req->nrec < 1) return fail(SGB_ERR_INVALID_ARG, "serve: nt and nrec must be >= 1");
    if (!in_inner(g, req->src_ijk[0], req->src_ijk[1], req->src_ijk[2]))
        return fail(SGB_ERR_INVALID_ARG, "serve: source outside the inner region");
    for (int r = 0; r < req->nrec; ++r)
        if (!in_inner(g, req->rec_ijk[3 * r], req->rec_ijk[3 * r + 1], req->rec_ijk[3 * r + 2]))
            return fail(SGB_ERR_INVALID_ARG, "serve: receiver %d outside the inner region", r);
    const uint64_t fp = shot_footprint(L, req->nt, req->nrec);
    if (fp > sv->cfg.hbm_budget_bytes) {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stats.rejected += 1;
        return fail(SGB_ERR_REJECTED, "serve: footprint %llu bytes above the budget %llu",
                    (unsigned long long)fp, (unsigned long long)sv->cfg.hbm_budget_bytes);
    }
    const long long ncomp = (long long)L.Nx * L.Ny * L.Nz;
    float vmax = 0.0f;
    for (long long c = 0; c < ncomp; ++c) {
        const float v = req->velocity[c];
        if (!(v > 0.0f) || !std::isfinite(v))
            return fail(SGB_ERR_INVALID_ARG, "serve: velocity has non-positive or non-finite values");
        vmax = std::max(vmax, v);
    }
    if ((double)g->dt > cfl_limit(g, vmax))
        return fail(SGB_ERR_UNSTABLE_DT, "serve: dt %g above the CFL limit %g of the model",
                    (double)g->dt, cfl_limit(g, vmax));
    Shot *sh = new Shot();
    sh->g = *g;
    sh->L = L;
    sh->nt = req->nt;
    sh->nrec = req->nrec;
    for (int q = 0; q < 3; ++q) sh->src[q] = req->src_ijk[q];
    sh->vel.assign(req->velocity, req->velocity + ncomp);
    sh->wav.assign(req->wavelet, req->wavelet + req->nt);
    sh->rec.assign(req->rec_ijk, req->rec_ijk + 3 * (size_t)req->nrec);
    sh->footprint = fp;
    sh->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stop) {
            delete sh;
            return fail(SGB_ERR_REJECTED, "serve: server is shutting down");
        }
        sh->ticket = sv->next_ticket++;
        sv->known[sh->ticket] = true;
        sv->live[sh->ticket] = sh;
        sv->queue.push_back(sh);
        sv->stats.submitted += 1;
        sv->stats.queued = (int)sv->queue.size();
    }
    sv->cv_work.notify_all();
    *ticket = sh->ticket;
    return SGB_OK;
}

extern "C" int serve_poll(sgb_server *sv, uint64_t ticket, sgb_shot_result *out, int32_t timeout_us)
{
    if (!sv || !out) return fail(SGB_ERR_INVALID_ARG, "NULL argument");
    std::unique_lock<std::mutex> lk(sv->mu);
    if (!sv->known.count(ticket)) return fail(SGB_ERR_INVALID_ARG, "serve: unknown ticket %llu",
                                              (unsigned long long)ticket);
    auto ready = [&] { return sv->done.count(ticket) > 0; };
    if (!ready()) {
        if (timeout_us <= 0) return SGB_PENDING;
        sv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready);
        if (!ready()) return fail(SGB_ERR_TIMEOUT, "serve: ticket %llu not done within %d us",
                                  (unsigned long long)ticket, timeout_us);
    }
    Shot *sh = sv->done[ticket];
    out->ticket = ticket;
    out->status = sh->status;
    out->nt = sh->nt;
    out->nrec = sh->nrec;
    out->queue_ms = ms_between(sh->t_submit, sh->t_admit);
    out->latency_ms = ms_between(sh->t_submit, sh->t_done);
    if (out->traces && (sh->status == SGB_OK || sh->status == SGB_ERR_NONFINITE))
        memcpy(out->traces, sh->traces.data(), sh->traces.size() * 4);
    sv->done.erase(ticket);
    sv->known.erase(ticket);
    delete sh;
    return SGB_OK;
}

extern "C" int serve_cancel(sgb_server *sv, uint64_t ticket)
{
    if (!sv) return fail(SGB_ERR_INVALID_ARG, "NULL server");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (!sv->known.count(ticket))
        return fail(SGB_ERR_INVALID_ARG, "serve: unknown ticket %llu", (unsigned long long)ticket);
    if (sv->done.count(ticket)) return SGB_OK;  // finished already: its result stands
    Shot *sh = sv->live[ticket];
    auto it = std::find(sv->queue.begin(), sv->queue.end(), sh);
    if (it != sv->queue.end()) {  // never admitted: done at once
        sv->queue.erase(it);
        sh->status = SGB_ERR_CANCELLED;
        sh->t_admit = sh->t_done = Clock::now();
        sv->done[ticket] = sh;
        sv->live.erase(ticket);
        sv->stats.cancelled += 1;
        sv->stats.queued = (int)sv->queue.size();
        sv->cv_done.notify_all();
        return SGB_OK;
    }
    sh->cancel = true;  // admitted: retired at the end of the current replays
    return SGB_OK;
}

extern "C" int serve_stats(sgb_server *sv, sgb_serve_stats *out)
{
    if (!sv || !out) return fail(SGB_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    *out = sv->stats;
    return SGB_OK;
}

extern "C" int serve_destroy(sgb_server *sv)
{
    if (!sv) return fail(SGB_ERR_INVALID_ARG, "NULL server");
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        for (Shot *sh : sv->queue) {  // cancel what was never admitted
            sh->status = SGB_ERR_REJECTED;
            sv->live.erase(sh->ticket);
            delete sh;
        }
        sv->queue.clear();
    }
    sv->cv_work.notify_all();
    if (sv->th.joinable()) sv->th.join();
    for (auto &kv : sv->done) delete kv.second;
    if (sv->exec) cudaGraphExecDestroy(sv->exec);
    cudaStreamSynchronize(sv->stream);
    cudaStreamSynchronize(sv->setup_stream);
    server_release_handles(sv);
    delete sv;
    return SGB_OK;
}
