// Misfit gradient with respect to the velocity model: forward shot with
// checkpoints, then a backward sweep of hand-written adjoint steps with the
// forward recomputed segment by segment.  Included at the end of seisgb.cu.
//
// Adjoint notes (the paper has no adjoint; this is the exact discrete adjoint
// of the fused step).  With lambda^k the multiplier of u^k and M the
// coefficient of (L u + phi + f) in the update (m inside, m / (1 + e) in the
// PML), the scaled multiplier w = M lambda obeys, for k = nt .. 1:
//   w^k   = 2 w^{k+1} - w^{k+2} + m (L w^{k+1} + psi + K^T r^{k-1})         inside
//   w^k   = [(2 - e^2) w^{k+1} - (1 - e) w^{k+2} + m (L w^{k+1} + psi)] / (1 + e)  PML
//   nu^k  = nu^{k+1} / (1 + e) + w^{k+1}                             PML points
//   psi   = sum_a [c_a nu^{k+1}](x + e_a) - [c_a nu^{k+1}](x - e_a),  over PML
//           neighbours, c_a / (2 h_a) = k_a (d(+1)^2 - d(-1)^2) / (1 + e)
//   dJ/dm += w^k g^{k-1} / m,   g^n = L u^n + phi^n + f^n
// i.e. the forward step run backward in time with the trace residual r
// injected at the receivers.  dJ/dv = dJ/dm * 2 v dt^2 (dt held fixed).
#pragma once

namespace {

using CfgAdj = TileCfg<SGB_TXT, SGB_TYT, SGB_TY, SGB_NU, 3, SGB_MINB, SGB_UNROLL>;

// psi from nu^{k+1} on the PML and the inner points next to it; nu^k on the
// PML.  One thread per computed point (points far from the PML return).
__global__ void psi_nu_kernel(StepArgs a, const float *__restrict__ w1,
                              const float *__restrict__ nu_in, float *__restrict__ nu_out,
                              float *__restrict__ psi)
{
    const long long npts = (long long)a.Nx * a.Ny * a.Nz;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const int nin[3] = {a.nx, a.ny, a.nz};
    const float ka[3] = {a.kx, a.ky, a.kz};
    const float ea[3] = {a.ax, a.ay, a.az};
    const long long st3[3] = {1, a.sx, a.sxy};
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < npts; c += stride) {
        const int i = (int)(c % a.Nx);
        const long long t = c / a.Nx;
        const int j = (int)(t % a.Ny), k = (int)(t / a.Ny);
        const int x[3] = {i, j, k};
        int d[3];
        bool pml = false, band = false;
        for (int q = 0; q < 3; ++q) {
            d[q] = pml_depth(nin[q], a.nb, x[q]);
            pml |= d[q] > 0;
            band |= x[q] == a.nb || x[q] == a.nb + nin[q] - 1;
        }
        if (!pml && !band) continue;
        const long long p = a.origin + (long long)k * a.sxy + (long long)j * a.sx + i;
        float s = 0.0f;
        for (int ax = 0; ax < 3; ++ax)
            for (int sg = -1; sg <= 1; sg += 2) {
                int y[3] = {x[0], x[1], x[2]};
                y[ax] += sg;
                if (y[ax] < 0 || y[ax] >= (ax == 0 ? a.Nx : ax == 1 ? a.Ny : a.Nz)) continue;
                int dy[3];
                float e = 0.0f;
                bool ypml = false;
                for (int q = 0; q < 3; ++q) {
                    dy[q] = pml_depth(nin[q], a.nb, y[q]);
                    ypml |= dy[q] > 0;
                    e += ea[q] * float(dy[q] * dy[q]);
                }
                if (!ypml) continue;
                const int dp = pml_depth(nin[ax], a.nb, y[ax] + 1);
                const int dm = pml_depth(nin[ax], a.nb, y[ax] - 1);
                const float cy = ka[ax] * float(dp * dp - dm * dm) / (1.0f + e);
                s += float(sg) * cy * nu_in[p + sg * st3[ax]];
            }
        psi[p] = s;
        if (pml) {
            float e = 0.0f;
            for (int q = 0; q < 3; ++q) e += ea[q] * float(d[q] * d[q]);
            nu_out[p] = nu_in[p] / (1.0f + e) + w1[p];
        }
    }
}

// Residual of step k-1 enters at the receivers: w^k += m r, and the gradient
// term of that part (m r g / m = r g).
__global__ void inject_residual_kernel(float *__restrict__ w, const float *__restrict__ m,
                                       const float *__restrict__ acc, double *__restrict__ grad_m,
                                       const long long *__restrict__ rec_off, int nrec,
                                       const float *__restrict__ traces_row,
                                       const float *__restrict__ obs_row)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < nrec) {
        const long long p = rec_off[r];
        const float res = traces_row[r] - obs_row[r];
        w[p] += m[p] * res;
        grad_m[p] += (double)res * (double)acc[p];
    }
}

// J = 1/2 sum (traces - observed)^2 in fp64, in a fixed order (two passes:
// per-block partial sums, then one block), so repeated runs agree to the bit.
constexpr int MISFIT_BLOCKS = 256;

__global__ void misfit_partial_kernel(const float *__restrict__ tr, const float *__restrict__ obs,
                                      long long n, double *partial)
{
    __shared__ double ws[8];
    double s = 0.0;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        const double d = (double)tr[q] - (double)obs[q];
        s += 0.5 * d * d;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        partial[blockIdx.x] = t;
    }
}

__global__ void misfit_final_kernel(const double *partial, int n, double *J)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double t = 0.0;
        for (int b = 0; b < n; ++b) t += partial[b];
        *J = t;
    }
}

// dJ/dv = dJ/dm * 2 v dt^2 on the compact grid.
__global__ void chain_kernel(PadGeom g, const double *__restrict__ grad_m,
                             const float *__restrict__ vel, float dt, double *__restrict__ grad_v)
{
    const long long n = (long long)g.Nx * g.Ny * g.Nz;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        const long long i = c % g.Nx, t = c / g.Nx;
        const long long j = t % g.Ny, k = t / g.Ny;
        const double v = vel[c];
        grad_v[c] = grad_m[g.origin + k * g.sxy + j * g.sx + i] * 2.0 * v * (double)dt * (double)dt;
    }
}

int adjoint_prepared = 0;

}  // namespace

extern "C" int adjoint_shot(const sgb_grid *g, const float *velocity, const float *wavelet,
                            int32_t nt, const int32_t *src_ijk, const int32_t *rec_ijk,
                            int32_t nrec, const float *observed, int32_t ckpt_every,
                            double *misfit_out, double *grad_velocity, void *stream)
{
    sgb_layout_info L;
    int rc = check_grid(g, &L);
    if (rc) return rc;
    if (g->storage != SGB_FP32) return fail(SGB_ERR_INVALID_ARG, "adjoint_shot: SGB_FP32 only");
    if (!velocity || !wavelet || !src_ijk || !rec_ijk || !observed || !misfit_out || !grad_velocity)
        return fail(SGB_ERR_INVALID_ARG, "adjoint_shot: NULL argument");
    if (nt < 1 || nrec < 1) return fail(SGB_ERR_INVALID_ARG, "adjoint_shot: nt and nrec must be >= 1");
    if (ckpt_every < 0) return fail(SGB_ERR_INVALID_ARG, "adjoint_shot: ckpt_every < 0");
    const int C = ckpt_every == 0 ? 100 : std::min<int>(ckpt_every, nt);
    if (!in_inner(g, src_ijk[0], src_ijk[1], src_ijk[2]))
        return fail(SGB_ERR_INVALID_ARG, "adjoint_shot: source outside the inner region");
    std::vector<long long> off(nrec);
    for (int r = 0; r < nrec; ++r) {
        const int i = rec_ijk[3 * r], j = rec_ijk[3 * r + 1], k = rec_ijk[3 * r + 2];
        if (!in_inner(g, i, j, k))
            return fail(SGB_ERR_INVALID_ARG, "adjoint_shot: receiver %d outside the inner region", r);
        off[r] = L.origin + (long long)k * L.stride_z + (long long)j * L.sx + i;
    }
    DevState *ds;
    if ((rc = device_state(&ds))) return rc;
    if (!adjoint_prepared) {
        std::lock_guard<std::mutex> lk(g_mu);
        CUDA_TRY(cudaFuncSetAttribute(fwd_acc_kernel<Cfg>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)Stage<Cfg, float, MODE_FWD_ACC>::SMEM_BYTES));
        CUDA_TRY(cudaFuncSetAttribute(adjoint_step_kernel<CfgAdj>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)Stage<CfgAdj, float, MODE_ADJ>::SMEM_BYTES));
        adjoint_prepared = 1;
    }
    cudaStream_t st = (cudaStream_t)stream;
    {
        int pending = 0;
        if ((rc = read_and_clear_dev_err(*ds, st, &pending))) return rc;
    }
    const long long ncomp = (long long)L.Nx * L.Ny * L.Nz;
    const size_t fbytes = (size_t)L.elems * 4;
    const int nseg = (nt + C - 1) / C;
    Scratch sc{st, ds->pool, {}};
    // inputs on the device
    auto to_dev = [&](const void *src, size_t bytes, void **dst) -> int {
        if (is_device_ptr(src)) {
            *dst = const_cast<void *>(src);
            return SGB_OK;
        }
        int r2 = sc.get(dst, bytes);
        if (r2) return r2;
        CUDA_TRY(cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, st));
        return SGB_OK;
    };
    float *d_vel, *d_wav, *d_obs;
    if ((rc = to_dev(velocity, (size_t)ncomp * 4, (void **)&d_vel)) ||
        (rc = to_dev(wavelet, (size_t)nt * 4, (void **)&d_wav)) ||
        (rc = to_dev(observed, (size_t)nt * nrec * 4, (void **)&d_obs)))
        return rc;
    // CFL against the model's maximum
    int *d_range;
    if ((rc = sc.get((void **)&d_range, 16))) return rc;
    int init[4] = {0, 0x7f7fffff, 0, 0};
    CUDA_TRY(cudaMemcpyAsync(d_range, init, sizeof init, cudaMemcpyHostToDevice, st));
    vel_range_kernel<<<ew_grid(ncomp, *ds), 256, 0, st>>>(d_vel, ncomp, d_range);
    CUDA_TRY(cudaGetLastError());
    int range[4];
    CUDA_TRY(cudaMemcpyAsync(range, d_range, sizeof range, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (range[2] != 0) return fail(SGB_ERR_INVALID_ARG, "velocity has non-positive or non-finite values");
    float vmax_model;
    memcpy(&vmax_model, &range[0], 4);
    if ((double)g->dt > cfl_limit(g, vmax_model))
        return fail(SGB_ERR_UNSTABLE_DT, "dt %g above the CFL limit %g of the model", (double)g->dt,
                    cfl_limit(g, vmax_model));
    // fields
    float *u0, *u1, *phi, *m, *w0, *w1, *nu0, *nu1, *psi, *ck, *seg, *d_tr;
    double *grad_m, *d_J;
    long long *d_off;
    if ((rc = sc.get((void **)&u0, fbytes)) || (rc = sc.get((void **)&u1, fbytes)) ||
        (rc = sc.get((void **)&phi, fbytes)) || (rc = sc.get((void **)&m, fbytes)) ||
        (rc = sc.get((void **)&w0, fbytes)) || (rc = sc.get((void **)&w1, fbytes)) ||
        (rc = sc.get((void **)&nu0, fbytes)) || (rc = sc.get((void **)&nu1, fbytes)) ||
        (rc = sc.get((void **)&psi, fbytes)) ||
        (rc = sc.get((void **)&ck, fbytes * 3 * (size_t)nseg)) ||
        (rc = sc.get((void **)&seg, fbytes * (size_t)C)) ||
        (rc = sc.get((void **)&d_tr, (size_t)nt * nrec * 4)) ||
        (rc = sc.get((void **)&grad_m, (size_t)L.elems * 8)) || (rc = sc.get((void **)&d_J, 8)) ||
        (rc = sc.get((void **)&d_off, (size_t)nrec * 8)))
        return rc;
    CUDA_TRY(cudaMemcpyAsync(d_off, off.data(), (size_t)nrec * 8, cudaMemcpyHostToDevice, st));
    for (float *f : {u0, u1, phi, m, w0, w1, nu0, nu1, psi}) CUDA_TRY(cudaMemsetAsync(f, 0, fbytes, st));
    CUDA_TRY(cudaMemsetAsync(grad_m, 0, (size_t)L.elems * 8, st));
    CUDA_TRY(cudaMemsetAsync(d_J, 0, 8, st));
    make_m_kernel<<<ew_grid(ncomp, *ds), 256, 0, st>>>(pad_geom(L), d_vel, g->dt, m);
    CUDA_TRY(cudaGetLastError());

    StepArgs base;
    fill_step_constants(g, L, base);
    base.phi = phi;
    base.err = ds->err;
    base.si = src_ijk[0];
    base.sj = src_ijk[1];
    base.sk = src_ijk[2];
    base.wavelet = d_wav;
    int grid = 0;
    choose_decomposition(L.Nx, L.Ny, L.Nz, ds->sms, ds->occ, base, &grid);
    float *ubuf[2] = {u0, u1};  // ubuf[0] = u^{-1}, ubuf[1] = u^0
    StepMaps fmaps[2];
    for (int p = 0; p < 2; ++p)
        if ((rc = encode_step_maps<float>(fmaps[p], ubuf[(p + 1) & 1], ubuf[p & 1], m, phi, L))) return rc;

    // 1. forward with checkpoints (u^n, u^{n-1}, phi^n before step n = s C)
    for (int n = 0; n < nt; ++n) {
        if (n % C == 0) {
            float *dst = ck + (size_t)(n / C) * 3 * L.elems;
            CUDA_TRY(cudaMemcpyAsync(dst, ubuf[(n + 1) & 1], fbytes, cudaMemcpyDeviceToDevice, st));
            CUDA_TRY(cudaMemcpyAsync(dst + L.elems, ubuf[n & 1], fbytes, cudaMemcpyDeviceToDevice, st));
            CUDA_TRY(cudaMemcpyAsync(dst + 2 * L.elems, phi, fbytes, cudaMemcpyDeviceToDevice, st));
        }
        StepArgs a = base;
        a.u_out = ubuf[n & 1];
        a.u_cur = ubuf[(n + 1) & 1];
        a.step_add = n;
        a.nrec = nrec;
        a.rec_off = d_off;
        a.traces = d_tr;
        if ((rc = launch_step<float>(a, fmaps[n & 1], grid, st))) return rc;
    }
    gather_kernel<<<(nrec + 255) / 256, 256, 0, st>>>(ubuf[(nt - 1) & 1], d_off, nrec,
                                                      d_tr + (size_t)(nt - 1) * nrec, ds->err);
    CUDA_TRY(cudaGetLastError());
    double *d_part;
    if ((rc = sc.get((void **)&d_part, MISFIT_BLOCKS * 8))) return rc;
    misfit_partial_kernel<<<MISFIT_BLOCKS, 256, 0, st>>>(d_tr, d_obs, (long long)nt * nrec, d_part);
    CUDA_TRY(cudaGetLastError());
    misfit_final_kernel<<<1, 32, 0, st>>>(d_part, MISFIT_BLOCKS, d_J);
    CUDA_TRY(cudaGetLastError());

    // 2. backward sweep, segment by segment from the last
    float *wbuf[2] = {w0, w1};  // w^k lives in wbuf[k & 1]
    float *nbuf[2] = {nu0, nu1};
    std::vector<CUtensorMap> acc_maps(C);
    for (int q = 0; q < C; ++q)
        if ((rc = encode_map<float>(&acc_maps[q], seg + (size_t)q * L.elems, L, CfgAdj::BX, CfgAdj::BY)))
            return rc;
    StepMaps amaps[2];  // [k & 1]: reads w^{k+1} = wbuf[(k+1)&1], writes wbuf[k&1]
    for (int p = 0; p < 2; ++p)
        if ((rc = encode_step_maps<float>(amaps[p], wbuf[(p + 1) & 1], wbuf[p & 1], m, psi, L))) return rc;
    StepArgs abase = base;
    abase.phi = nullptr;
    abase.sk = -1;  // the adjoint's sources are the receivers (injected separately)
    abase.grad_m = grad_m;
    int agrid = 0;
    choose_decomposition(L.Nx, L.Ny, L.Nz, ds->sms, ds->occ, abase, &agrid);
    const int pgrid = ew_grid(ncomp, *ds);
    for (int s = nseg - 1; s >= 0; --s) {
        const int na = s * C, nbnd = std::min(na + C, nt);
        const float *src_ck = ck + (size_t)s * 3 * L.elems;
        CUDA_TRY(cudaMemcpyAsync(ubuf[(na + 1) & 1], src_ck, fbytes, cudaMemcpyDeviceToDevice, st));
        CUDA_TRY(cudaMemcpyAsync(ubuf[na & 1], src_ck + L.elems, fbytes, cudaMemcpyDeviceToDevice, st));
        CUDA_TRY(cudaMemcpyAsync(phi, src_ck + 2 * L.elems, fbytes, cudaMemcpyDeviceToDevice, st));
        for (int n = na; n < nbnd; ++n) {  // recompute, keeping g^n
            StepArgs a = base;
            a.u_out = ubuf[n & 1];
            a.u_cur = ubuf[(n + 1) & 1];
            a.step_add = n;
            a.acc_out = seg + (size_t)(n - na) * L.elems;
            const StepMaps &mp = fmaps[n & 1];
            fwd_acc_kernel<Cfg><<<grid, Cfg::BLOCK, Stage<Cfg, float, MODE_FWD_ACC>::SMEM_BYTES, st>>>(
                a, mp.ucur, mp.ucur_in, mp.uprev, mp.m, mp.phi);
            CUDA_TRY(cudaGetLastError());
            ++t_launches;
        }
        for (int k = nbnd; k >= na + 1; --k) {  // adjoint steps
            StepArgs a = abase;
            a.u_out = wbuf[k & 1];
            a.u_cur = wbuf[(k + 1) & 1];
            a.step_add = k;
            psi_nu_kernel<<<pgrid, 256, 0, st>>>(a, wbuf[(k + 1) & 1], nbuf[(k + 1) & 1],
                                                  nbuf[k & 1], psi);
            CUDA_TRY(cudaGetLastError());
            const StepMaps &mp = amaps[k & 1];
            adjoint_step_kernel<CfgAdj><<<agrid, CfgAdj::BLOCK,
                                          Stage<CfgAdj, float, MODE_ADJ>::SMEM_BYTES, st>>>(
                a, mp.ucur, mp.ucur_in, mp.uprev, mp.m, mp.phi, acc_maps[k - 1 - na]);
            CUDA_TRY(cudaGetLastError());
            inject_residual_kernel<<<(nrec + 255) / 256, 256, 0, st>>>(
                wbuf[k & 1], m, seg + (size_t)(k - 1 - na) * L.elems, grad_m, d_off, nrec,
                d_tr + (size_t)(k - 1) * nrec, d_obs + (size_t)(k - 1) * nrec);
            CUDA_TRY(cudaGetLastError());
            t_launches += 3;
        }
    }
    // 3. chain rule to velocity, outputs
    double *d_gv = grad_velocity;
    const bool host_gv = !is_device_ptr(grad_velocity);
    if (host_gv && (rc = sc.get((void **)&d_gv, (size_t)ncomp * 8))) return rc;
    chain_kernel<<<ew_grid(ncomp, *ds), 256, 0, st>>>(pad_geom(L), grad_m, d_vel, g->dt, d_gv);
    CUDA_TRY(cudaGetLastError());
    if (host_gv)
        CUDA_TRY(cudaMemcpyAsync(grad_velocity, d_gv, (size_t)ncomp * 8, cudaMemcpyDeviceToHost, st));
    double J = 0.0;
    CUDA_TRY(cudaMemcpyAsync(&J, d_J, 8, cudaMemcpyDeviceToHost, st));
    int dev_err = 0;
    if ((rc = read_and_clear_dev_err(*ds, st, &dev_err))) return rc;
    *misfit_out = J;
    if (dev_err & DEV_ERR_TIMEOUT) return fail(SGB_ERR_TIMEOUT, "a kernel wait timed out");
    return SGB_OK;
}
