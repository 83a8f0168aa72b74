// expo_api.cu -- the exponential propagators of the homogeneous ParaExp
// problems behind the C ABI (Sec. III-B; kernels in expo.cu and expo_tma.cu,
// parameters in expo_plan.cu): the member engine for Leja / Taylor
// propagation, fit_expo_propagate, and ParaExp with exponential homogeneous
// problems (paraexp_run with opts.homogeneous).
#include "grid.h"

using namespace fitgb;

namespace fitgb {

// ----------------------------------------------------------------------------
// Exponential propagators of the homogeneous problems (Sec. III-B; kernels in
// expo.cu, parameters in expo_plan.cu).  Every member owns three state blocks
// P, R, Y in g->xblocks (member idx at 3*n6*idx), P filled by the caller.
// Members advance substep-aligned: at substep s every member with more than s
// substeps takes one, so the active members are a prefix of the table sorted
// by decreasing substep count.  A member's final state (e at the end of its
// interval, h there or half a step earlier) is added to the FP64
// superposition, shortest member first; its probe rows come from the Newton
// basis recorded at the probe edges (dense output) and are added in member
// order at the end.
// ----------------------------------------------------------------------------
struct ExpoSpec {
    long long nsteps;   // leapfrog steps the member covers (>= 1)
    long long row0;     // probe row of its first output step
    bool stagger;       // final h half a step before the final e
};

struct ExpoParams {
    int kind, q, m;
    double u, c;   // u = dt/dt_CFL, c = q u
};

// 2/beta, beta the bound on ||A||_2 the propagators interpolate on: 2/dt_CFL on a uniform grid
// (the Yee bound eq. (cfl) comes from), ||A||_1 on a graded grid (where eq. (cfl) is only an
// estimate)
double expo_unit(const fit_grid *g) { return g->graded ? 2.0 / g->rowsum : cfl_of(g); }

int expo_params(const fit_grid *g, double dt, const fit_run_opts *o, ExpoParams *P) {
    const int kind = o ? o->homogeneous : FIT_HOMOG_LEAPFROG;
    if (kind != FIT_HOMOG_LEJA && kind != FIT_HOMOG_TAYLOR) return FIT_ERR_ARG;
    P->kind = kind;
    P->u = dt / expo_unit(g);
    const double tol = (o->expo_tol > 0.0) ? o->expo_tol : (g->prec == 64 ? 1e-12 : 1e-6);
    if (!std::isfinite(tol)) return FIT_ERR_ARG;
    if (o->expo_substep > 0 || o->expo_degree > 0) {
        P->q = o->expo_substep;
        P->m = o->expo_degree;
        if (P->q < 1 || P->m < 2 || (P->m & 1) || P->m > kExpoMaxDegree || P->q * P->u > 64.0) return FIT_ERR_ARG;
    } else {
        int rc = expo_plan(kind, P->u, tol, g->prec == 64 ? 64 : 32, &P->q, &P->m);
        if (rc) return rc;
    }
    P->c = P->q * P->u;
    return FIT_OK;
}

template <typename T>
int expo_members(fit_grid *g, double dt, const ExpoParams &X, const std::vector<ExpoSpec> &specs, bool sync_first,
                 const fit_probe *prb, int nprb, double *probe_dev, long long probe_rows, double *acc_e,
                 double *acc_h, void *out_e, void *out_h, const fit_run_opts *opts, cudaStream_t s) {
    const int nmem = (int)specs.size();
    if (nmem == 0) return FIT_OK;
    const long long ncp = g->ncp, ncell = g->ncell;
    const size_t n6 = 6 * (size_t)ncp;
    const int J = X.m / 2, m1 = X.m + 1, q = X.q;
    const bool probes = probe_dev && nprb > 0 && probe_rows > 0;
    const bool profile = opts && opts->profile;
    int rc;
    if (nprb > kMaxPrb) return FIT_ERR_UNSUPPORTED;
    if ((rc = ensure_coeffs<T>(g, dt, opts ? opts->sigma_scheme : 0, false, s))) return rc;

    // host tables: pair coefficients at tau = 1, dense-output rows tau = i/q, final substeps
    std::vector<double> al(J), ga(J), eta2(J), tmp(J), reg(2 * J), D((size_t)q * m1);
    if ((rc = expo_pair_coeffs(X.kind, X.m, X.c, al.data(), ga.data(), eta2.data()))) return rc;
    for (int j = 0; j < J; ++j) reg[2 * j] = al[j], reg[2 * j + 1] = ga[j];
    for (int i = 1; i <= q; ++i) {
        if ((rc = expo_pair_coeffs(X.kind, X.m, ((double)i / q) * X.c, al.data(), ga.data(), tmp.data()))) return rc;
        double *row = D.data() + (size_t)(i - 1) * m1;
        row[0] = 1.0;
        for (int j = 0; j < J; ++j) row[2 * j + 1] = al[j], row[2 * j + 2] = ga[j];
    }
    std::vector<long long> nsub(nmem), nrem(nmem), row0(nmem);
    std::vector<double> fin((size_t)nmem * J * 4);
    for (int t = 0; t < nmem; ++t) {
        const long long ns = specs[t].nsteps;
        if (ns < 1) return FIT_ERR_ARG;
        nsub[t] = (ns + q - 1) / q;
        const long long rem = ns - (nsub[t] - 1) * q;
        std::vector<double> ae(J), ge(J), ah(J), gh(J);
        if ((rc = expo_pair_coeffs(X.kind, X.m, ((double)rem / q) * X.c, ae.data(), ge.data(), tmp.data())))
            return rc;
        const double th = specs[t].stagger ? ((double)rem - 0.5) / q : (double)rem / q;
        if ((rc = expo_pair_coeffs(X.kind, X.m, th * X.c, ah.data(), gh.data(), tmp.data()))) return rc;
        for (int j = 0; j < J; ++j) {
            double *f = fin.data() + ((size_t)t * J + j) * 4;
            f[0] = ae[j], f[1] = ge[j], f[2] = ah[j], f[3] = gh[j];
        }
        nrem[t] = ns;
        row0[t] = specs[t].row0;
    }
    // table order: decreasing substep count (stable)
    std::vector<int> order(nmem);
    for (int t = 0; t < nmem; ++t) order[t] = t;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return nsub[x] > nsub[y]; });

    // probe basis per member: nsub * m1 * nprb doubles
    std::vector<size_t> boff(nmem, 0);
    size_t btotal = 0;
    for (int t = 0; t < nmem; ++t) {
        boff[t] = btotal;
        btotal += probes ? (size_t)nsub[t] * m1 * nprb : 0;
    }
    if (probes) {
        if ((rc = ensure(g->xbasis, btotal * sizeof(double)))) return rc;
        if ((rc = ensure(g->xpm, (size_t)nmem * probe_rows * nprb * sizeof(double)))) return rc;
        FIT_CHECK(cudaMemsetAsync(g->xbasis.p, 0, btotal * sizeof(double), s));
        FIT_CHECK(cudaMemsetAsync(g->xpm.p, 0, (size_t)nmem * probe_rows * nprb * sizeof(double), s));
    }
    // device table: reg | D | fin | nrem | row0 | basis pointers | members (table order)
    auto up16 = [](size_t v) { return (v + 15) & ~(size_t)15; };
    const size_t o_reg = 0, o_D = up16(o_reg + reg.size() * 8), o_fin = up16(o_D + D.size() * 8),
                 o_nrem = up16(o_fin + fin.size() * 8), o_row0 = up16(o_nrem + nmem * 8),
                 o_bp = up16(o_row0 + nmem * 8), o_mem = up16(o_bp + nmem * sizeof(void *)),
                 total = up16(o_mem + nmem * sizeof(ExpoMember<T>));
    if ((rc = ensure(g->xtab, total))) return rc;
    char *dt_base = (char *)g->xtab.p;
    std::vector<char> host(total, 0);
    memcpy(host.data() + o_reg, reg.data(), reg.size() * 8);
    memcpy(host.data() + o_D, D.data(), D.size() * 8);
    std::vector<long long> nrem_o(nmem), row0_o(nmem);
    std::vector<const double *> bp(nmem);
    std::vector<ExpoMember<T>> mem(nmem);
    std::vector<double> fin_o(fin.size());
    for (int r = 0; r < nmem; ++r) {
        const int t = order[r];
        memcpy(fin_o.data() + (size_t)r * J * 4, fin.data() + (size_t)t * J * 4, (size_t)J * 4 * 8);
        nrem_o[r] = nrem[t];
        row0_o[r] = row0[t];
        T *P = (T *)g->xblocks.p + 3 * n6 * (size_t)t;
        mem[r].P = P;
        mem[r].R = P + n6;
        mem[r].Y = P + 2 * n6;
        mem[r].nsub = (int)nsub[t];
        mem[r].blk = 3 * t;
        mem[r].fin = (const double *)(dt_base + o_fin) + (size_t)r * J * 4;
        mem[r].basis = probes ? (double *)g->xbasis.p + boff[t] : nullptr;
        bp[r] = mem[r].basis;
    }
    memcpy(host.data() + o_fin, fin_o.data(), fin_o.size() * 8);
    memcpy(host.data() + o_nrem, nrem_o.data(), nmem * 8);
    memcpy(host.data() + o_row0, row0_o.data(), nmem * 8);
    memcpy(host.data() + o_bp, bp.data(), nmem * sizeof(void *));
    memcpy(host.data() + o_mem, mem.data(), nmem * sizeof(ExpoMember<T>));
    FIT_CHECK(cudaMemcpyAsync(g->xtab.p, host.data(), total, cudaMemcpyHostToDevice, s));
    FIT_CHECK(cudaStreamSynchronize(s));   // the host table must outlive the copy

    ExpoArgs<T> a;
    memset(&a, 0, sizeof(a));
    a.nx = g->nx; a.ny = g->ny; a.nz = g->nz; a.pitch = g->pitch; a.ncp = ncp;
    a.cb = (const T *)g->coef.p;
    a.ch = (const T *)g->ch.p;
    a.kappa = expo_unit(g) / dt;
    a.mem = (const ExpoMember<T> *)(dt_base + o_mem);
    a.reg = (const double *)(dt_base + o_reg);
    a.sync = dt / (2.0 * expo_unit(g));
    a.m1 = m1;
    if ((rc = ensure(g->err, sizeof(int)))) return rc;
    a.err = (int *)g->err.p;
    a.extra_tx = opts ? std::max(0, opts->debug_extra_tx) : 0;
    a.nprb = probes ? nprb : 0;
    for (int p = 0; p < a.nprb; ++p) a.prb[p] = {prb[p].axis, prb[p].i, prb[p].j, prb[p].k};
    // z chunks: enough blocks to fill the GPU with the fewest members of a launch
    const long long cols = (long long)((g->nx + 31) / 32) * ((g->ny + 7) / 8);
    a.kz = 8;   // measured best on 256^3 (FP32: 8 planes 0.63 of HBM, 32 planes 0.53)
    while (a.kz > 2 && cols * ((g->nz + a.kz - 1) / a.kz) < 8 * 152) a.kz /= 2;
    if (opts && opts->tile_z > 0) a.kz = std::min(opts->tile_z, g->nz);
    a.nchunk = (g->nz + a.kz - 1) / a.kz;
    if ((long long)a.nchunk * nmem > 65535) return FIT_ERR_UNSUPPORTED;

    // FP32: fused pairs (TMA ring) unless opts->kernel = 1 asks for the plain launches.  FP64 is
    // bound by the FP64 pipes, where the plain launches measured faster (12.5 against 10.4
    // Gcell-applications/s on 256^3); opts->kernel = 2 selects the fused kernel there.
    bool fused = sizeof(T) == 4 ? !(opts && opts->kernel == 1) : (opts && opts->kernel == 2);
    TmaMaps maps;
    CUtensorMap cbmap;
    ExpoArgs<T> af;
    if (fused) {
        const int ftx = expo_pair_tile_x((int)sizeof(T)), fty = expo_pair_tile_y((int)sizeof(T));
        fused = encode_tma_maps(&maps, (int)sizeof(T), g->nx, g->ny, g->nz, g->pitch, g->xblocks.p, 3 * nmem,
                                g->coef.p, 3, ftx, fty) &&
                encode_window_map(&cbmap, (int)sizeof(T), g->nx, g->ny, g->nz, g->pitch, g->coef.p, 3, ftx + 8,
                                  fty + 2, 3);
        af = a;
        const long long fcols = (long long)((g->nx + ftx - 1) / ftx) * ((g->ny + fty - 1) / fty);
        af.kz = (opts && opts->tile_z > 0) ? std::min(opts->tile_z, g->nz) : 16;   // 16 measured best (256^3)
        while (af.kz > 4 && fcols * ((g->nz + af.kz - 1) / af.kz) < 4 * 152) af.kz /= 2;
        af.nchunk = (g->nz + af.kz - 1) / af.kz;
    }
    const int wait_limit = opts ? std::max(0, opts->debug_wait_limit) : 0;
    const double eb = (double)sizeof(T) * (double)ncell;   // bytes of one component
    const double coefc = 3.0 + (g->mu_array ? 3.0 : 0.0);
    long long nev = 0;
    auto run = [&](int mode, int active) -> int {
        a.mode = mode;
        a.nmem = active;
        if (profile) {
            while ((long long)g->ev.size() < 2 * (nev + 1)) {
                cudaEvent_t e;
                FIT_CHECK(cudaEventCreate(&e));
                g->ev.push_back(e);
            }
            FIT_CHECK(cudaEventRecord(g->ev[2 * nev], s));
        }
        FIT_CHECK(launch_expo<T>(a, g->mu_array, s));
        if (profile) {
            FIT_CHECK(cudaEventRecord(g->ev[2 * nev + 1], s));
            ++nev;
        }
        g->stats.kernel_launches += 1;
        if (mode == kExpoSync) {
            g->stats.expo_alg_bytes += eb * (9.0 * active + (g->mu_array ? 3.0 : 0.0));
            return FIT_OK;
        }
        const double fields = mode == kExpoInit ? 12.0 : mode == kExpoPair1 ? 24.0 : 18.0;
        g->stats.expo_launches += 1;
        g->stats.expo_applications += active;
        g->stats.expo_alg_bytes += eb * (fields * active + coefc);
        return FIT_OK;
    };
    // one fused pair j: y = X R_{j-1}, R_j = X y + eta_j^2 R_{j-1} (not after the last), P update
    auto run_fused = [&](int j, int active) -> int {
        af.pair = j;
        af.substep = a.substep;
        af.nmem = active;
        af.eta2 = j < J ? eta2[j - 1] : 0.0;
        const bool last = j == J;
        if (profile) {
            while ((long long)g->ev.size() < 2 * (nev + 1)) {
                cudaEvent_t e;
                FIT_CHECK(cudaEventCreate(&e));
                g->ev.push_back(e);
            }
            FIT_CHECK(cudaEventRecord(g->ev[2 * nev], s));
        }
        FIT_CHECK(launch_expo_pair_tma<T>(af, maps.state, cbmap, last, g->mu_array, wait_limit, s));
        if (profile) {
            FIT_CHECK(cudaEventRecord(g->ev[2 * nev + 1], s));
            ++nev;
        }
        g->stats.kernel_launches += 1;
        g->stats.expo_launches += 1;
        g->stats.expo_applications += (long long)active * (last ? 1 : 2);
        g->stats.expo_alg_bytes += eb * ((last ? 18.0 : 24.0) * active + coefc);
        if (probes) {
            FIT_CHECK(launch_expo_gather_fused<T>(af, s));
            g->stats.kernel_launches += 1;
        }
        return FIT_OK;
    };
    auto gather = [&](int mode, int active) -> int {
        if (!probes) return FIT_OK;
        a.mode = mode;
        a.nmem = active;
        FIT_CHECK(launch_expo_gather<T>(a, s));
        g->stats.kernel_launches += 1;
        return FIT_OK;
    };
    const size_t row = (size_t)g->nx * sizeof(T), prow = (size_t)g->pitch * sizeof(T);
    const size_t rows3 = 3 * (size_t)g->ny * g->nz;
    auto finalize = [&](int r) -> int {
        const T *P = mem[r].P;
        if (acc_e) {
            FIT_CHECK(accumulate_state<T>(3 * ncp, P, acc_e, s));
            g->stats.kernel_launches += 1;
        }
        if (acc_h) {
            FIT_CHECK(accumulate_state<T>(3 * ncp, P + 3 * ncp, acc_h, s));
            g->stats.kernel_launches += 1;
        }
        if (out_e) FIT_CHECK(cudaMemcpy2DAsync(out_e, row, P, prow, row, rows3, kind_from_dev(out_e), s));
        if (out_h) FIT_CHECK(cudaMemcpy2DAsync(out_h, row, P + 3 * ncp, prow, row, rows3, kind_from_dev(out_h), s));
        return FIT_OK;
    };

    if (sync_first && (rc = run(kExpoSync, nmem))) return rc;
    int active = nmem;
    for (long long sub = 0; sub < mem[0].nsub; ++sub) {
        while (active > 0 && mem[active - 1].nsub <= sub) --active;
        a.substep = (int)sub;
        if ((rc = run(kExpoInit, active)) || (rc = gather(kExpoInit, active))) return rc;
        for (int j = 1; j <= J; ++j) {
            a.pair = j;
            if (fused) {
                if ((rc = run_fused(j, active))) return rc;
                continue;
            }
            if ((rc = run(kExpoPair1, active)) || (rc = gather(kExpoPair1, active))) return rc;
            if (j < J) {
                a.eta2 = eta2[j - 1];
                if ((rc = run(kExpoPair2, active))) return rc;
            }
        }
        for (int r = active - 1; r >= 0; --r)
            if (mem[r].nsub == sub + 1 && (rc = finalize(r))) return rc;
    }
    if (probes) {
        long long maxr = 0;
        for (int t = 0; t < nmem; ++t) maxr = std::max(maxr, nrem[t]);
        FIT_CHECK(launch_expo_dense(nmem, (const double *const *)(dt_base + o_bp), (const long long *)(dt_base + o_nrem),
                                    (const long long *)(dt_base + o_row0), maxr, q, m1, nprb,
                                    (const double *)(dt_base + o_D), (double *)g->xpm.p, probe_rows * nprb, s));
        FIT_CHECK(add_members(nmem, probe_rows * nprb, (const double *)g->xpm.p, probe_rows * nprb, probe_dev, s));
        g->stats.kernel_launches += 2;
    }
    if (profile && nev > 0) {
        FIT_CHECK(cudaStreamSynchronize(s));
        double ms = 0.0;
        for (long long t = 0; t < nev; ++t) {
            float v = 0.f;
            FIT_CHECK(cudaEventElapsedTime(&v, g->ev[2 * t], g->ev[2 * t + 1]));
            ms += v;
        }
        g->stats.expo_ms += ms;
    }
    return FIT_OK;
}

// compact (3, nz, ny, nx) T -> pitched block components [0, 3) or [3, 6), masked later
template <typename T>
int load_compact(fit_grid *g, T *dst3, const void *src, cudaStream_t s) {
    if (!src) return FIT_OK;
    const size_t row = (size_t)g->nx * sizeof(T), prow = (size_t)g->pitch * sizeof(T);
    FIT_CHECK(cudaMemcpy2DAsync(dst3, prow, src, row, row, 3 * (size_t)g->ny * g->nz, kind_to_dev(src), s));
    return FIT_OK;
}

template <typename T>
int expo_propagate_impl(fit_grid *g, double dt, long nsteps, const fit_probe *prb, int nprb, double *probe_out,
                        void *e_io, void *h_io, const fit_run_opts *opts, cudaStream_t s) {
    int rc;
    ExpoParams X;
    if ((rc = expo_params(g, dt, opts, &X))) return rc;
    g->stats = fit_run_stats{0, 0, 0, 0.0, 0.0, 0, 0, 0.0, 0.0};
    const size_t n6 = 6 * (size_t)g->ncp;
    if ((rc = ensure(g->xblocks, 3 * n6 * sizeof(T)))) return rc;
    if ((rc = ensure(g->err, sizeof(int)))) return rc;
    FIT_CHECK(cudaMemsetAsync(g->err.p, 0, sizeof(int), s));
    T *P = (T *)g->xblocks.p;
    FIT_CHECK(cudaMemsetAsync(P, 0, n6 * sizeof(T), s));
    if ((rc = load_compact<T>(g, P, e_io, s)) || (rc = load_compact<T>(g, P + 3 * g->ncp, h_io, s))) return rc;
    FIT_CHECK(mask_state<T>(g->nx, g->ny, g->nz, g->pitch, P, P + 3 * g->ncp, s));
    g->stats.kernel_launches += 1;
    const bool host_out = (probe_out && !is_device(probe_out)) || (e_io && !is_device(e_io)) ||
                          (h_io && !is_device(h_io));
    double *pdev = nullptr;
    if (probe_out && nprb > 0) {
        if (is_device(probe_out)) pdev = probe_out;
        else {
            if ((rc = ensure(g->probe_ws, sizeof(double) * (size_t)nsteps * nprb))) return rc;
            pdev = (double *)g->probe_ws.p;
        }
        FIT_CHECK(cudaMemsetAsync(pdev, 0, sizeof(double) * (size_t)nsteps * nprb, s));
    }
    std::vector<ExpoSpec> specs(1, ExpoSpec{nsteps, 0, false});
    rc = expo_members<T>(g, dt, X, specs, false, prb, nprb, pdev, nsteps, nullptr, nullptr, e_io, h_io, opts, s);
    if (rc) return rc;
    if (pdev && pdev != probe_out)
        FIT_CHECK(cudaMemcpyAsync(probe_out, pdev, sizeof(double) * (size_t)nsteps * nprb, cudaMemcpyDeviceToHost, s));
    return finish(g, s, host_out);
}

template <typename T>
int paraexp_expo_impl(fit_grid *g, double dt, int K, const long *win, const fit_source *src, int nsrc,
                      const fit_probe *prb, int nprb, double *probe_out, double *e_final, double *h_final,
                      const void *e0, const void *h0, const fit_run_opts *opts, cudaStream_t s) {
    int rc;
    ExpoParams X;
    if ((rc = expo_params(g, dt, opts, &X))) return rc;
    const int scheme = opts->sigma_scheme;
    const long long W0 = win[0], WK = win[K], nt = WK - W0;
    const bool u0 = e0 || h0;
    const int nexp = (K - 1) + (u0 ? 1 : 0);
    const size_t n6 = 6 * (size_t)g->ncp, n3 = 3 * (size_t)g->ncp;
    if ((rc = ensure(g->xblocks, (3 * (size_t)nexp + 1) * n6 * sizeof(T)))) return rc;
    T *blocks = (T *)g->xblocks.p;
    T *lastv = blocks + 3 * n6 * (size_t)nexp;   // v_K's final state
    const bool host_out = (probe_out && !is_device(probe_out)) || (e_final && !is_device(e_final)) ||
                          (h_final && !is_device(h_final));
    double *pdev = nullptr;
    if (probe_out && nprb > 0 && nt > 0) {
        if (is_device(probe_out)) pdev = probe_out;
        else {
            if ((rc = ensure(g->probe_ws, sizeof(double) * (size_t)nt * nprb))) return rc;
            pdev = (double *)g->probe_ws.p;
        }
    }
    double *ae = nullptr, *ah = nullptr;
    if (e_final || h_final) {
        if ((rc = ensure(g->acc, 2 * n3 * sizeof(double)))) return rc;
        ae = (double *)g->acc.p;
        ah = ae + n3;
    }
    // v_j: leapfrog over window j only; final states into the members' P blocks
    std::vector<MemberSpec> specs;
    std::vector<T *> keep;
    for (int j = 1; j <= K; ++j) {
        specs.push_back({win[j - 1], win[j] - win[j - 1], win[j - 1], win[j], nullptr, nullptr});
        keep.push_back(j < K ? blocks + 3 * n6 * (size_t)(j - 1) : lastv);
    }
    rc = run_members<T>(g, dt, scheme, specs, W0, nt, src, nsrc, prb, nprb, W0, nt, pdev, nullptr, 0, nullptr,
                        nullptr, nullptr, nullptr, opts, s, keep.data());
    if (rc) return rc;
    if (ae) {
        FIT_CHECK(cudaMemsetAsync(ae, 0, 2 * n3 * sizeof(double), s));
        FIT_CHECK(accumulate_state<T>((long long)n3, lastv, ae, s));
        FIT_CHECK(accumulate_state<T>((long long)n3, lastv + n3, ah, s));
        g->stats.kernel_launches += 2;
    }
    std::vector<ExpoSpec> xs;
    for (int j = 1; j < K; ++j) xs.push_back({WK - win[j], win[j] - W0, true});
    if (u0) {   // w_1 from (e^{W_0}, h^{W_0 - 1/2})
        T *P = blocks + 3 * n6 * (size_t)(K - 1);
        FIT_CHECK(cudaMemsetAsync(P, 0, n6 * sizeof(T), s));
        if ((rc = load_compact<T>(g, P, e0, s)) || (rc = load_compact<T>(g, P + n3, h0, s))) return rc;
        FIT_CHECK(mask_state<T>(g->nx, g->ny, g->nz, g->pitch, P, P + n3, s));
        g->stats.kernel_launches += 1;
        xs.push_back({nt, 0, true});
    }
    rc = expo_members<T>(g, dt, X, xs, true, prb, nprb, pdev, nt, ae, ah, nullptr, nullptr, opts, s);
    if (rc) return rc;
    if (pdev && pdev != probe_out)
        FIT_CHECK(cudaMemcpyAsync(probe_out, pdev, sizeof(double) * (size_t)nt * nprb, cudaMemcpyDeviceToHost, s));
    const size_t row = (size_t)g->nx * sizeof(double), prow = (size_t)g->pitch * sizeof(double);
    const size_t rows3 = 3 * (size_t)g->ny * g->nz;
    if (e_final) FIT_CHECK(cudaMemcpy2DAsync(e_final, row, ae, prow, row, rows3, kind_from_dev(e_final), s));
    if (h_final) FIT_CHECK(cudaMemcpy2DAsync(h_final, row, ah, prow, row, rows3, kind_from_dev(h_final), s));
    return finish(g, s, host_out);
}

template int paraexp_expo_impl<float>(fit_grid *, double, int, const long *, const fit_source *, int,
                                      const fit_probe *, int, double *, double *, double *, const void *,
                                      const void *, const fit_run_opts *, cudaStream_t);
template int paraexp_expo_impl<double>(fit_grid *, double, int, const long *, const fit_source *, int,
                                       const fit_probe *, int, double *, double *, double *, const void *,
                                       const void *, const fit_run_opts *, cudaStream_t);

}  // namespace fitgb

extern "C" {

int fit_spectral_bound(const fit_grid *g, double *beta) {
    if (!g || !beta) return FIT_ERR_ARG;
    *beta = 2.0 / expo_unit(g);
    return FIT_OK;
}

int fit_expo_propagate(fit_grid *g, double dt, long nsteps, const fit_probe *prb, int nprb, double *probe_out,
                       void *e_io, void *h_io, const fit_run_opts *opts, void *stream) {
    if (!g || nsteps < 0 || !opts || !(dt > 0.0) || !std::isfinite(dt)) return FIT_ERR_ARG;
    if (any_foreign({probe_out, e_io, h_io})) return FIT_ERR_ARG;
    if (opts->homogeneous != FIT_HOMOG_LEJA && opts->homogeneous != FIT_HOMOG_TAYLOR) return FIT_ERR_ARG;
    int rc;
    if ((rc = check_sources_probes(g, nullptr, 0, prb, nprb))) return rc;
    if (g->prec == 48 || g->prec == 40 || g->lossy) return FIT_ERR_UNSUPPORTED;
    if (nsteps == 0) return FIT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (g->prec == 64)
        return expo_propagate_impl<double>(g, dt, nsteps, prb, nprb, probe_out, e_io, h_io, opts, s);
    return expo_propagate_impl<float>(g, dt, nsteps, prb, nprb, probe_out, e_io, h_io, opts, s);
}

}  // extern "C"
