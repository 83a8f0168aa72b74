// adjoint_api.cu -- fit_adjoint_grad: the adjoint gradient's schedule on
// the host (kernels in adjoint.cu and the fused step kernels).
#include "grid.h"

using namespace fitgb;

namespace {

// Adjoint gradient (see adjoint.cu for the reverse sweep and the gradient
// formula).  Schedule: one forward pass of N steps from zero state records the
// probe trace and a checkpoint of (e, h) every C steps; then, segment by
// segment from the last, the checkpoint is re-advanced through a ring of
// C+1 state slots (slot q holds step A+q), and the adjoint state steps back
// through the segment, each adjoint step followed by the gradient update from
// ring slots q and q+1.  Memory: N/C checkpoints + C+1 ring slots.
template <typename T>
int adjoint_impl(fit_grid *g, double dt, long long N, const fit_source *src, int nsrc, const fit_probe *prb,
                 int nprb, int C, double *J_out, double *grad_out, const fit_run_opts *opts, cudaStream_t s) {
    const int scheme = opts ? opts->sigma_scheme : 0;
    int rc;
    g->stats = fit_run_stats{0, 0, 0, 0.0, 0.0, 0, 0, 0.0, 0.0};
    if (nprb < 1 || nprb > kMaxSrc || nsrc > kMaxSrc) return FIT_ERR_UNSUPPORTED;
    if ((rc = ensure_coeffs<T>(g, dt, scheme, false, s))) return rc;
    // without a gradient output only the forward run and J are computed: no
    // checkpoints and no reverse sweep
    const bool want_grad = grad_out != nullptr;
    if (C <= 0) C = std::max(1, (int)std::ceil(std::sqrt((double)N)));
    if (C > N) C = (int)N;
    if (!want_grad) C = 1;
    const long long nseg = (N + C - 1) / C;
    const long long ncp = g->ncp;
    const size_t n6 = 6 * (size_t)ncp;
    if (want_grad && (rc = ensure(g->ckpt, (size_t)nseg * n6 * sizeof(T)))) return rc;
    if ((rc = ensure(g->ring, (size_t)(C + 1) * n6 * sizeof(T)))) return rc;
    if (want_grad && (rc = ensure(g->lam, 2 * n6 * sizeof(T)))) return rc;
    if (want_grad && (rc = ensure(g->gacc, 3 * (size_t)ncp * sizeof(double)))) return rc;
    // FP32 fields: the gradient of each block of kGradBlock adjoint steps is summed in FP32 and
    // then added into the FP64 total (block boundaries fixed in the adjoint step index, so the
    // result does not depend on the checkpoint interval)
    constexpr int kGradBlock = 64;
    const bool fp32_blocks = want_grad && sizeof(T) == 4;
    if (fp32_blocks && (rc = ensure(g->gblk, 3 * (size_t)ncp * sizeof(float)))) return rc;
    if ((rc = ensure(g->aprobe, (size_t)N * nprb * sizeof(double)))) return rc;
    if (want_grad && (rc = ensure(g->aamp, (size_t)N * nprb * sizeof(double)))) return rc;
    if ((rc = ensure(g->adjmem, (size_t)(C + 2) * sizeof(Member)))) return rc;
    if ((rc = ensure(g->err, sizeof(int)))) return rc;
    if ((rc = ensure(g->scalar, 2 * sizeof(double)))) return rc;
    if (nsrc > 0) {
        if ((rc = ensure(g->amp, sizeof(double) * (size_t)N * nsrc))) return rc;
        if ((rc = ensure(g->srcdev, sizeof(fit_source) * nsrc))) return rc;
        FIT_CHECK(cudaMemcpyAsync(g->srcdev.p, src, sizeof(fit_source) * nsrc, cudaMemcpyHostToDevice, s));
        FIT_CHECK(source_table((const fit_source *)g->srcdev.p, nsrc, 0, N, dt, (double *)g->amp.p, s));
        g->stats.kernel_launches += 1;
    }
    T *ring = (T *)g->ring.p, *lam = (T *)g->lam.p, *ckpt = (T *)g->ckpt.p;
    double *gacc = (double *)g->gacc.p, *aprobe = (double *)g->aprobe.p, *aamp = (double *)g->aamp.p;
    FIT_CHECK(cudaMemsetAsync(ring, 0, n6 * sizeof(T), s));
    if (want_grad) {
        FIT_CHECK(cudaMemsetAsync(lam, 0, 2 * n6 * sizeof(T), s));
        FIT_CHECK(cudaMemsetAsync(gacc, 0, 3 * (size_t)ncp * sizeof(double), s));
    }
    if (fp32_blocks) FIT_CHECK(cudaMemsetAsync(g->gblk.p, 0, 3 * (size_t)ncp * sizeof(float), s));
    FIT_CHECK(cudaMemsetAsync(g->err.p, 0, sizeof(int), s));

    // member table: [0] forward ping-pong in ring slots 0/1, [1+q] ring slot q -> q+1,
    // [C+1] the adjoint state's ping-pong
    std::vector<Member> mt((size_t)C + 2);
    memset(mt.data(), 0, sizeof(Member) * mt.size());
    for (auto &m : mt) {
        m.src_lo = -(1LL << 62);
        m.src_hi = (1LL << 62);
        m.end = (1LL << 62);
    }
    mt[0].st[0] = ring;
    mt[0].st[1] = ring + n6;
    mt[0].blk[0] = 0;
    mt[0].blk[1] = 1;
    mt[0].probe = aprobe;
    for (int q = 0; q < C; ++q) {
        Member &m = mt[1 + q];
        m.st[0] = ring + (size_t)q * n6;
        m.st[1] = ring + (size_t)(q + 1) * n6;
        m.blk[0] = q;
        m.blk[1] = q + 1;
        m.start = q;   // + the segment start passed as the iteration
    }
    mt[C + 1].st[0] = lam;
    mt[C + 1].st[1] = lam + n6;
    mt[C + 1].blk[0] = 0;
    mt[C + 1].blk[1] = 1;
    Member *mdev = (Member *)g->adjmem.p;
    FIT_CHECK(cudaMemcpyAsync(mdev, mt.data(), sizeof(Member) * mt.size(), cudaMemcpyHostToDevice, s));

    Tile tile = pick_tile(g, opts);
    TmaMaps ring_maps, lam_maps;
    if (tile.kernel == 2 &&
        !(encode_tma_maps(&ring_maps, (int)sizeof(T), g->nx, g->ny, g->nz, g->pitch, ring, C + 1, g->coef.p,
                          g->lossy ? 6 : 3, tile.tx, tile.ty) &&
          (!want_grad || encode_tma_maps(&lam_maps, (int)sizeof(T), g->nx, g->ny, g->nz, g->pitch, lam, 2,
                                         g->coef.p, g->lossy ? 6 : 3, tile.tx, tile.ty)))) {
        tile.kernel = 1;
        if (!tile_supported(tile.tx, tile.ty)) tile.tx = 32, tile.ty = 8;
    }
    StepArgs<T> a;
    memset(&a, 0, sizeof(a));
    a.nx = g->nx; a.ny = g->ny; a.nz = g->nz; a.pitch = g->pitch; a.ncell = ncp;
    a.tiles_x = (g->nx + tile.tx - 1) / tile.tx;
    a.tiles_y = (g->ny + tile.ty - 1) / tile.ty;
    a.kz = tile.kz;
    a.nchunk = (g->nz + tile.kz - 1) / tile.kz;
    a.cb = (const T *)g->coef.p;
    a.ca = g->lossy ? (const T *)g->coef.p + 3 * ncp : nullptr;
    a.ch = (const T *)g->ch.p;
    a.nmem = 1;
    a.err = (int *)g->err.p;
    {   // z chunks from the plain step kernel's CTAs per SM (unless the caller fixed them)
        int per_sm = 0, nsm = 0, dev = 0;
        cudaError_t qe = cudaGetDevice(&dev);
        if (qe == cudaSuccess) qe = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (qe == cudaSuccess && !tile.kz_fixed) {
            StepArgs<T> q = a;
            q.occ_out = &per_sm;
            qe = tile.kernel == 2 ? launch_step_tma<T>(q, ring_maps, tile, g->lossy, g->mu_array, false, s)
                                  : launch_step<T>(q, tile, g->lossy, g->mu_array, false, s);
        }
        if (qe != cudaSuccess) {
            cudaGetLastError();
            per_sm = 0;
        }
        tile.kz = chunk_length(g->nx, g->ny, g->nz, tile, 1, (long long)per_sm * nsm, nsm > 0 ? nsm : 152);
        a.kz = tile.kz;
        a.nchunk = (g->nz + tile.kz - 1) / tile.kz;
    }
    // FP32 TMA runs fuse the gradient accumulation into the adjoint step
    const bool fused = fp32_blocks && tile.kernel == 2 && step_grad_supported(tile);
    // With a memory budget (opts->adjoint_mem_mb, two-cell FP32 kernel) the forward sweep keeps
    // d^n = e^{n+1} - e^n of its last segments; those segments skip the recompute, and their
    // adjoint steps read d^n instead of two ring states.  The kernel forms d^n with the same
    // float subtraction the adjoint step would, so the gradient is the same bits.
    long long seg_keep0 = nseg;   // first segment whose differences are kept
    if (fused && !tile.single && opts && opts->adjoint_mem_mb > 0) {
        const double per_step = 3.0 * (double)ncp * sizeof(float);
        const double budget = (double)opts->adjoint_mem_mb * 1048576.0;
        while (seg_keep0 > 0 && (double)(N - (seg_keep0 - 1) * C) * per_step <= budget) --seg_keep0;
        if (seg_keep0 < nseg &&
            ensure(g->dhist, (size_t)(N - seg_keep0 * C) * 3 * (size_t)ncp * sizeof(float)) != FIT_OK)
            seg_keep0 = nseg;   // no room after all: recompute every segment
    }
    const long long A_keep = seg_keep0 * C;   // steps n >= A_keep keep d^n
    float *dhist = (float *)g->dhist.p;
    // opts->profile: every step and gradient launch timed by CUDA events on the stream
    // (stats.step_ms) with its algorithmic bytes (stats.alg_bytes)
    const bool profile = opts && opts->profile;
    long long nev = 0;
    const double ncell_d = (double)g->ncell;
    const double step_bytes = (12.0 * sizeof(T) + ((g->lossy ? 6.0 : 3.0) + (g->mu_array ? 3.0 : 0.0)) * sizeof(T)) *
                              ncell_d;   // e, h in and out, coefficients once
    auto timed = [&](double bytes, auto &&fn) -> cudaError_t {
        if (profile) {
            while ((long long)g->ev.size() < 2 * (nev + 1)) {
                cudaEvent_t e;
                cudaError_t ce = cudaEventCreate(&e);
                if (ce != cudaSuccess) return ce;
                g->ev.push_back(e);
            }
            cudaError_t ce = cudaEventRecord(g->ev[2 * nev], s);
            if (ce != cudaSuccess) return ce;
        }
        cudaError_t ce = fn();
        if (ce != cudaSuccess) return ce;
        if (profile) {
            if ((ce = cudaEventRecord(g->ev[2 * nev + 1], s)) != cudaSuccess) return ce;
            ++nev;
        }
        g->stats.alg_bytes += bytes;
        return cudaSuccess;
    };
    auto step = [&](const TmaMaps &maps) -> cudaError_t {
        g->stats.step_launches += 1;
        g->stats.kernel_launches += 1;
        g->stats.cell_updates += g->ncell;
        // the fused gradient adds e^{n+1}, e^n (or d^n) read and the FP32 block sum read and
        // written; keeping d^n adds its write
        const double bytes = step_bytes + (a.gb ? (a.ge0 ? 12.0 : 9.0) * sizeof(float) * ncell_d : 0.0) +
                             (a.gd ? 3.0 * sizeof(float) * ncell_d : 0.0);
        return timed(bytes, [&]() {
            if (tile.kernel == 2) return launch_step_tma<T>(a, maps, tile, g->lossy, g->mu_array, false, s);
            return launch_step<T>(a, tile, g->lossy, g->mu_array, false, s);
        });
    };
    auto set_forward_sources = [&]() {
        a.nsrc = nsrc;
        for (int q = 0; q < nsrc; ++q) a.src[q] = {src[q].axis, src[q].i, src[q].j, src[q].k};
        a.amp = (const double *)g->amp.p;
        a.amp_base = 0;
        a.amp_len = N;
    };

    // forward pass with checkpoints and the probe record
    set_forward_sources();
    a.nprb = nprb;
    for (int q = 0; q < nprb; ++q) a.prb[q] = {prb[q].axis, prb[q].i, prb[q].j, prb[q].k};
    a.mem = mdev;
    for (long long n = 0; n < N; ++n) {
        if (want_grad && n % C == 0 && n < A_keep)
            FIT_CHECK(cudaMemcpyAsync(ckpt + (size_t)(n / C) * n6, ring + (size_t)(n & 1) * n6, n6 * sizeof(T),
                                      cudaMemcpyDeviceToDevice, s));
        a.it = (int)n;
        a.parity = (int)(n & 1);
        a.gd = (want_grad && n >= A_keep) ? dhist + (size_t)(n - A_keep) * 3 * (size_t)ncp : nullptr;
        FIT_CHECK(step(ring_maps));
    }
    a.gd = nullptr;
    a.nprb = 0;
    // each probe edge's length: the grid step, or on a graded grid the size of
    // the cell the edge runs through along its axis
    double plen[kMaxSrc];
    for (int q = 0; q < nprb; ++q) {
        const int ax = prb[q].axis, idx[3] = {prb[q].i, prb[q].j, prb[q].k};
        const size_t off = ax == 0 ? 0 : (ax == 1 ? (size_t)g->nx : (size_t)g->nx + g->ny);
        plen[q] = g->graded ? g->spc_host[off + idx[ax]] : g->d[ax];
    }
    double *Jdev = (double *)g->scalar.p;
    FIT_CHECK(probe_functional(prb, nprb, plen, aprobe, N, Jdev, s));
    g->stats.kernel_launches += 1;
    if (!want_grad) {
        if (J_out) FIT_CHECK(cudaMemcpyAsync(J_out, Jdev, sizeof(double), kind_from_dev(J_out), s));
        return finish(g, s, J_out && !is_device(J_out));
    }
    // adjoint state at N and the adjoint sources
    FIT_CHECK(adjoint_init<T>(prb, nprb, plen, aprobe + (size_t)(N - 1) * nprb, (const T *)g->coef.p, lam, g->pitch,
                              g->ny, ncp, s));
    FIT_CHECK(adjoint_sources(prb, nprb, plen, aprobe, N, aamp, s));
    g->stats.kernel_launches += 2;
    // -eps0 A_a / (L_a dt) per axis; on a graded grid the geometry goes into the scatter
    const double K[3] = {g->graded ? -kEps0 / dt : -kEps0 * (g->d[1] * g->d[2] / g->d[0]) / dt,
                         g->graded ? -kEps0 / dt : -kEps0 * (g->d[2] * g->d[0] / g->d[1]) / dt,
                         g->graded ? -kEps0 / dt : -kEps0 * (g->d[0] * g->d[1] / g->d[2]) / dt};

    for (long long sg = nseg - 1; sg >= 0; --sg) {
        const long long A = sg * C, B = std::min<long long>(A + C, N);
        const bool kept = sg >= seg_keep0;   // d^n of this segment came from the forward sweep
        if (!kept)
            FIT_CHECK(cudaMemcpyAsync(ring, ckpt + (size_t)sg * n6, n6 * sizeof(T), cudaMemcpyDeviceToDevice, s));
        set_forward_sources();
        for (long long q = 0; !kept && q < B - A; ++q) {   // ring slot q -> q+1: step A+q
            a.mem = mdev + 1 + q;
            a.it = (int)A;
            a.parity = 0;
            FIT_CHECK(step(ring_maps));
        }
        // adjoint: probe edges are the sources
        a.nsrc = nprb;
        for (int q = 0; q < nprb; ++q) a.src[q] = {prb[q].axis, prb[q].i, prb[q].j, prb[q].k};
        a.amp = aamp;
        a.amp_base = 0;
        a.amp_len = N;
        a.mem = mdev + C + 1;
        for (long long n = B - 1; n >= A; --n) {
            const long long t = N - 1 - n;
            a.it = (int)t;
            a.parity = (int)(t & 1);
            const T *e1 = ring + (size_t)(n + 1 - A) * n6, *e0 = ring + (size_t)(n - A) * n6;
            if (fused) {   // gb += K mu^{n+1} (e^{n+1} - e^n) inside the adjoint step
                a.ge1 = kept ? (const T *)(dhist + (size_t)(n - A_keep) * 3 * (size_t)ncp) : e1;
                a.ge0 = kept ? nullptr : e0;
                a.gb = (float *)g->gblk.p;
                for (int q = 0; q < 3; ++q) a.gk[q] = (float)K[q];
            }
            FIT_CHECK(step(lam_maps));
            a.gb = nullptr;
            const T *mu_in = lam + (size_t)(t & 1) * n6;
            if (fp32_blocks) {
                if (!fused) {
                    FIT_CHECK(timed(15.0 * sizeof(float) * (double)ncp, [&]() {
                        return grad_accumulate_block(ncp, (const float *)mu_in, (const float *)e1, (const float *)e0, K,
                                                     (float *)g->gblk.p, s);
                    }));
                    g->stats.kernel_launches += 1;
                }
                if ((t + 1) % kGradBlock == 0 || t == N - 1) {
                    FIT_CHECK(timed(18.0 * sizeof(float) * (double)ncp,
                                    [&]() { return grad_flush(ncp, (float *)g->gblk.p, gacc, s); }));
                    g->stats.kernel_launches += 1;
                }
            } else {
                FIT_CHECK(timed(3.0 * (3.0 * sizeof(T) + 2.0 * sizeof(double)) * (double)ncp, [&]() {
                    return grad_accumulate<T>(ncp, mu_in, e1, e0, K, gacc, s);
                }));
                g->stats.kernel_launches += 1;
            }
        }
    }
    // per-cell gradient and J
    double *gout = grad_out;
    const bool grad_host = !is_device(grad_out);
    if (grad_host) {
        if ((rc = ensure(g->grad_ws, sizeof(double) * (size_t)g->ncell))) return rc;
        gout = (double *)g->grad_ws.p;
    }
    FIT_CHECK(grad_scatter(g->nx, g->ny, g->nz, g->pitch, ncp, gacc, g->graded ? (const double *)g->spc.p : nullptr,
                           gout, s));
    g->stats.kernel_launches += 1;
    if (grad_host)
        FIT_CHECK(cudaMemcpyAsync(grad_out, gout, sizeof(double) * (size_t)g->ncell, cudaMemcpyDeviceToHost, s));
    if (J_out) FIT_CHECK(cudaMemcpyAsync(J_out, Jdev, sizeof(double), kind_from_dev(J_out), s));
    if (profile && nev > 0) {
        FIT_CHECK(cudaStreamSynchronize(s));
        double ms = 0.0;
        for (long long q = 0; q < nev; ++q) {
            float t = 0.f;
            FIT_CHECK(cudaEventElapsedTime(&t, g->ev[2 * q], g->ev[2 * q + 1]));
            ms += t;
        }
        g->stats.step_ms = ms;
    }
    const bool host_out = grad_host || (J_out && !is_device(J_out));
    return finish(g, s, host_out);
}

}  // namespace

extern "C" {

int fit_adjoint_grad(fit_grid *g, double dt, long nsteps, const fit_source *src, int nsrc, const fit_probe *prb,
                     int nprb, int ckpt_every, double *J_out, double *grad_eps_r, const fit_run_opts *opts,
                     void *stream) {
    if (!g || nsteps < 1 || ckpt_every < 0) return FIT_ERR_ARG;
    if (any_foreign({J_out, grad_eps_r})) return FIT_ERR_ARG;
    int rc;
    if ((rc = check_dt(g, dt, opts))) return rc;
    if ((rc = check_sources_probes(g, src, nsrc, prb, nprb))) return rc;
    if (opts && (opts->sigma_scheme < 0 || opts->sigma_scheme > 1)) return FIT_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (g->prec == 64)
        return adjoint_impl<double>(g, dt, nsteps, src, nsrc, prb, nprb, ckpt_every, J_out, grad_eps_r, opts, s);
    if (g->prec == 48 || g->prec == 40) return FIT_ERR_UNSUPPORTED;
    return adjoint_impl<float>(g, dt, nsteps, src, nsrc, prb, nprb, ckpt_every, J_out, grad_eps_r, opts, s);
}

}  // extern "C"
