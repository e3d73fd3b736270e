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
// injected at the receivers.  dJ/dv = dJ/dm * 2 v dt^2 = 2 (sum_k w^k g^{k-1}) / v
// (dt held fixed, m = (v dt)^2).
//
// The GPU keeps mu = nu / (1 + e) instead of nu: then mu^k = (mu^{k+1} +
// w^{k+1}) / (1 + e) and psi = sum_a k_a [G_a mu^{k+1}](x + e_a) - [G_a
// mu^{k+1}](x - e_a) with G_a(y) = d_a(y+1)^2 - d_a(y-1)^2, both computed by the
// adjoint step kernel at its PML tiles (mu is zero off the PML).  The time sum
// sum_k w^k g^{k-1} runs in fp32 per point over blocks of FOLD_EVERY steps
// (counted from step 0, so the grouping does not depend on the checkpoint
// interval) and is folded into an fp64 sum after each block.
#pragma once

namespace {

using CfgAdj = TileCfg<SGB_TXT, SGB_TYT, SGB_TY, SGB_NU, 2, SGB_MINB, SGB_UNROLL>;
constexpr int FOLD_EVERY = 32;

// G += S, S = 0 over the padded arrays (the fp64 time sum of the gradient).
__global__ void fold_kernel(float *__restrict__ S, double *__restrict__ G, long long n)
{
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        G[q] += (double)S[q];
        S[q] = 0.0f;
    }
}

// Residual of step k-1 enters at the receivers: w^k += m r, and its term of
// the gradient sum, S += (m r) g^{k-1}.
__global__ void inject_residual_kernel(float *__restrict__ w, const float *__restrict__ m,
                                       const float *__restrict__ acc, float *__restrict__ S,
                                       const long long *__restrict__ rec_off, int nrec,
                                       const float *__restrict__ traces_row,
                                       const float *__restrict__ obs_row)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < nrec) {
        const long long p = rec_off[r];
        const float add = m[p] * (traces_row[r] - obs_row[r]);
        w[p] += add;
        S[p] = fmaf(add, acc[p], S[p]);
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

// dJ/dv = 2 (sum_k w^k g^{k-1}) / v on the compact grid.
__global__ void chain_kernel(PadGeom g, const double *__restrict__ G,
                             const float *__restrict__ vel, double *__restrict__ grad_v)
{
    const long long n = (long long)g.Nx * g.Ny * g.Nz;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        const long long i = c % g.Nx, t = c / g.Nx;
        const long long j = t % g.Ny, k = t / g.Ny;
        grad_v[c] = 2.0 * G[g.origin + k * g.sxy + j * g.sx + i] / (double)vel[c];
    }
}

int adjoint_prepared = 0;
int adjoint_occ = 0;  // resident adjoint-step CTAs per SM

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
        CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &adjoint_occ, adjoint_step_kernel<CfgAdj>, CfgAdj::BLOCK,
            Stage<CfgAdj, float, MODE_ADJ>::SMEM_BYTES));
        if (adjoint_occ < 1) return fail(SGB_ERR_CUDA, "adjoint step kernel does not fit on an SM");
        adjoint_prepared = 1;
    }
    cudaStream_t st = (cudaStream_t)stream;
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
    float *u0, *u1, *phi, *m, *w0, *w1, *mu0, *mu1, *gsum, *ck, *seg, *d_tr;
    double *gsum64, *d_J;
    long long *d_off;
    int *d_err;  // this call's device error word: concurrent calls stay independent
    if ((rc = sc.get((void **)&u0, fbytes)) || (rc = sc.get((void **)&u1, fbytes)) ||
        (rc = sc.get((void **)&phi, fbytes)) || (rc = sc.get((void **)&m, fbytes)) ||
        (rc = sc.get((void **)&w0, fbytes)) || (rc = sc.get((void **)&w1, fbytes)) ||
        (rc = sc.get((void **)&mu0, fbytes)) || (rc = sc.get((void **)&mu1, fbytes)) ||
        (rc = sc.get((void **)&gsum, fbytes)) ||
        (rc = sc.get((void **)&ck, fbytes * 3 * (size_t)nseg)) ||
        (rc = sc.get((void **)&seg, fbytes * (size_t)C)) ||
        (rc = sc.get((void **)&d_tr, (size_t)nt * nrec * 4)) ||
        (rc = sc.get((void **)&gsum64, (size_t)L.elems * 8)) || (rc = sc.get((void **)&d_J, 8)) ||
        (rc = sc.get((void **)&d_off, (size_t)nrec * 8)) || (rc = sc.get((void **)&d_err, 16)))
        return rc;
    CUDA_TRY(cudaMemsetAsync(d_err, 0, sizeof(int), st));
    CUDA_TRY(cudaMemcpyAsync(d_off, off.data(), (size_t)nrec * 8, cudaMemcpyHostToDevice, st));
    for (float *f : {u0, u1, phi, m, w0, w1, mu0, mu1, gsum})
        CUDA_TRY(cudaMemsetAsync(f, 0, fbytes, st));
    CUDA_TRY(cudaMemsetAsync(gsum64, 0, (size_t)L.elems * 8, st));
    CUDA_TRY(cudaMemsetAsync(d_J, 0, 8, st));
    make_m_kernel<<<ew_grid(ncomp, *ds), 256, 0, st>>>(pad_geom(L), d_vel, g->dt, m);
    CUDA_TRY(cudaGetLastError());

    StepArgs base;
    fill_step_constants(g, L, base);
    base.phi = phi;
    base.err = d_err;
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
                                                      d_tr + (size_t)(nt - 1) * nrec, d_err);
    CUDA_TRY(cudaGetLastError());
    double *d_part;
    if ((rc = sc.get((void **)&d_part, MISFIT_BLOCKS * 8))) return rc;
    misfit_partial_kernel<<<MISFIT_BLOCKS, 256, 0, st>>>(d_tr, d_obs, (long long)nt * nrec, d_part);
    CUDA_TRY(cudaGetLastError());
    misfit_final_kernel<<<1, 32, 0, st>>>(d_part, MISFIT_BLOCKS, d_J);
    CUDA_TRY(cudaGetLastError());

    // 2. backward sweep, segment by segment from the last
    float *wbuf[2] = {w0, w1};  // w^k lives in wbuf[k & 1]
    float *mbuf[2] = {mu0, mu1};  // mu^k lives in mbuf[k & 1]
    std::vector<CUtensorMap> acc_maps(C);
    for (int q = 0; q < C; ++q)
        if ((rc = encode_map<float>(&acc_maps[q], seg + (size_t)q * L.elems, L, CfgAdj::BX, CfgAdj::BY)))
            return rc;
    // [k & 1]: reads w^{k+1} = wbuf[(k+1)&1] and mu^{k+1}, writes wbuf[k&1]
    StepMaps amaps[2];
    for (int p = 0; p < 2; ++p) {
        if ((rc = encode_step_maps<float>(amaps[p], wbuf[(p + 1) & 1], wbuf[p & 1], m,
                                          mbuf[(p + 1) & 1], L)))
            return rc;
        // mu^{k+1} as a box with its x-y neighbours (x halo 4, y halo 1)
        using GA = Stage<CfgAdj, float, MODE_ADJ>;
        if ((rc = encode_map<float>(&amaps[p].phi, mbuf[(p + 1) & 1], L, GA::MBW, GA::MBH, SGB_L2PROMO)))
            return rc;
    }
    CUtensorMap gs_map;
    if ((rc = encode_map<float>(&gs_map, gsum, L, CfgAdj::BX, CfgAdj::BY))) return rc;
    StepArgs abase = base;
    abase.sk = -1;  // the adjoint's sources are the receivers (injected separately)
    abase.gsum = gsum;
    int agrid = 0;
    choose_decomposition(L.Nx, L.Ny, L.Nz, ds->sms, adjoint_occ, abase, &agrid);
    const int fgrid = ew_grid(L.elems, *ds);
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
            CUDA_TRY(launch_dependent(fwd_acc_kernel<Cfg>, grid, Cfg::BLOCK,
                                      Stage<Cfg, float, MODE_FWD_ACC>::SMEM_BYTES, st, a, mp.ucur,
                                      mp.ucur_in, mp.uprev, mp.m, mp.phi));
            ++t_launches;
        }
        for (int k = nbnd; k >= na + 1; --k) {  // adjoint steps
            StepArgs a = abase;
            a.u_out = wbuf[k & 1];
            a.u_cur = wbuf[(k + 1) & 1];
            a.phi = mbuf[k & 1];
            a.mu_in = mbuf[(k + 1) & 1];
            a.step_add = k;
            const StepMaps &mp = amaps[k & 1];
            CUDA_TRY(launch_dependent(adjoint_step_kernel<CfgAdj>, agrid, CfgAdj::BLOCK,
                                      Stage<CfgAdj, float, MODE_ADJ>::SMEM_BYTES, st, a, mp.ucur,
                                      mp.ucur_in, mp.uprev, mp.m, mp.phi, acc_maps[k - 1 - na],
                                      gs_map));
            inject_residual_kernel<<<(nrec + 255) / 256, 256, 0, st>>>(
                wbuf[k & 1], m, seg + (size_t)(k - 1 - na) * L.elems, gsum, d_off, nrec,
                d_tr + (size_t)(k - 1) * nrec, d_obs + (size_t)(k - 1) * nrec);
            CUDA_TRY(cudaGetLastError());
            t_launches += 2;
            if ((k - 1) % FOLD_EVERY == 0) {  // blocks of steps counted from step 0
                fold_kernel<<<fgrid, 256, 0, st>>>(gsum, gsum64, (long long)L.elems);
                CUDA_TRY(cudaGetLastError());
                ++t_launches;
            }
        }
    }
    // 3. chain rule to velocity, outputs
    double *d_gv = grad_velocity;
    const bool host_gv = !is_device_ptr(grad_velocity);
    if (host_gv && (rc = sc.get((void **)&d_gv, (size_t)ncomp * 8))) return rc;
    chain_kernel<<<ew_grid(ncomp, *ds), 256, 0, st>>>(pad_geom(L), gsum64, d_vel, d_gv);
    CUDA_TRY(cudaGetLastError());
    if (host_gv)
        CUDA_TRY(cudaMemcpyAsync(grad_velocity, d_gv, (size_t)ncomp * 8, cudaMemcpyDeviceToHost, st));
    double J = 0.0;
    CUDA_TRY(cudaMemcpyAsync(&J, d_J, 8, cudaMemcpyDeviceToHost, st));
    int dev_err = 0;
    CUDA_TRY(cudaMemcpyAsync(&dev_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    *misfit_out = J;
    if (dev_err & DEV_ERR_TIMEOUT) return fail(SGB_ERR_TIMEOUT, "a kernel wait timed out");
    return SGB_OK;
}
