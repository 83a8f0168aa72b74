// api.cu -- the C ABI of include/fitgb.h: grid objects, coefficient cache,
// workspaces, and the member engine that drives the fused step kernel for
// plain leapfrog runs and for ParaExp.
//
// ParaExp engine (Sec. III, Algorithm 1): every window problem is a member
// (start step, source window).  Members are advanced iteration-aligned --
// at iteration `it` member m is at absolute step start_m + it -- so one
// launch moves every active member one step and the coefficient tile it
// reads serves all of them.  Members are ordered by decreasing length, so
// the active set is always a prefix of the member table.  A member's final
// state is added into the FP64 (or Kahan-FP32) superposition right after its
// last step, shortest member first; its probe rows go to a buffer of its own
// and are summed in member order at the end, so the result does not depend
// on scheduling.
#include <atomic>

#include "grid.h"

using namespace fitgb;

namespace fitgb {

namespace {
std::atomic<long long> g_fail_alloc{-1};   // allocations left before the injected failure (-1: off)
}

cudaError_t dev_alloc(void **p, size_t bytes) {
    long long left = g_fail_alloc.load();
    while (left >= 0) {
        if (g_fail_alloc.compare_exchange_weak(left, left - 1)) {
            if (left == 0) {   // this is the allocation chosen to fail
                *p = nullptr;
                return cudaErrorMemoryAllocation;
            }
            break;
        }
    }
    return cudaMalloc(p, bytes);
}

// Run `specs` members, iteration-aligned; see the file comment.
//   probe_dev: (probe rows) x nprb device buffer to receive the probe sum, or null
//   energy_dev: device buffer (rows) for member 0's energy, or null
//   acc_e, acc_h: padded FP64 superposition targets (3 components each), or null
//   final_e, final_h: copy member 0's final state here (compact layout), or null
template <typename T>
int run_members(fit_grid *g, double dt, int scheme, const std::vector<MemberSpec> &specs_in,
                long long amp_base, long long amp_len, const fit_source *src, int nsrc, const fit_probe *prb,
                int nprb, long long probe_base, long long probe_rows, double *probe_dev, double *energy_dev,
                int sum_mode, double *acc_e, double *acc_h, void *final_e, void *final_h,
                const fit_run_opts *opts, cudaStream_t s, T *const *keep_final) {
    const long long ncell = g->ncell;   // real cells (algorithmic counts)
    const long long ncp = g->ncp;       // padded component stride (device arrays)
    const bool comp = g->prec == 48;    // hi/lo float pairs: 12-component state blocks
    const bool resf = g->prec == 40;    // floats + bfloat16 residual words: 9-component state blocks
    const size_t n6 = (comp ? 12 : (resf ? 9 : 6)) * (size_t)ncp;
    const size_t row = (size_t)g->nx * sizeof(T), prow = (size_t)g->pitch * sizeof(T);
    const size_t rows3 = 3 * (size_t)g->ny * g->nz;
    int rc;
    if (nsrc > kMaxSrc || nprb > kMaxPrb) return FIT_ERR_UNSUPPORTED;
    g->stats = fit_run_stats{0, 0, 0, 0.0, 0.0, 0, 0, 0.0, 0.0};
    if ((rc = ensure_coeffs<T>(g, dt, scheme, energy_dev != nullptr, s))) return rc;
    const bool profile = opts && opts->profile;
    long long nev = 0;   // events recorded (pairs around step launches)
    // algorithmic bytes of one step launch: fields of every member once in and
    // once out, plus the coefficient arrays once
    const double fld_bytes = (comp ? 24.0 : (resf ? 18.0 : 12.0)) * sizeof(T) * (double)ncell;
    const double coef_bytes = ((g->lossy ? 6.0 : 3.0) + (g->mu_array ? 3.0 : 0.0) +
                               (energy_dev ? (3.0 + (g->mu_array ? 3.0 : 0.0)) : 0.0)) * sizeof(T) * (double)ncell;

    // order members by decreasing length (stable: equal lengths keep caller order)
    std::vector<int> order(specs_in.size());
    for (size_t m = 0; m < order.size(); ++m) order[m] = (int)m;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return specs_in[a].nit > specs_in[b].nit; });
    const int nm_total = (int)order.size();
    int mpp = (opts && opts->members_per_pass > 0) ? std::min(opts->members_per_pass, nm_total) : nm_total;
    if (!(opts && opts->members_per_pass > 0) && nm_total > 1) {
        // All members at once, within two limits.  (1) The member states advanced by one
        // launch stay within kLaunchStateBytes: on GB300 a launch whose member states span
        // more runs slower per cell-update (512^3 with residual fields: 27 members, 261 GB:
        // 62.5 Gcell/s; 16: 71.5; 8: 73.7; 6: 74.1; plain FP32: 32 members, 206 GB: 113.8,
        // 16: 117.3), while grids whose K states are smaller keep every member in one launch
        // (256^3: 16 members, 19 GB, at the best rate).  (2) They fit in the device memory
        // left (a too-small state buffer is freed before the new one is taken, so it counts
        // as free), less a margin for the call's other workspaces.
        constexpr size_t kLaunchStateBytes = size_t(96) << 30;
        const size_t per = 2 * n6 * sizeof(T);
        mpp = (int)std::max<size_t>(1, std::min<size_t>((size_t)nm_total, kLaunchStateBytes / per));
        size_t free_b = 0, total_b = 0;
        if (g->state.n < per * (size_t)mpp) {
            if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
                const size_t avail = free_b + g->state.n;
                const size_t margin = (size_t(1) << 30) + total_b / 64 +
                                      (sum_mode == 1 && acc_e ? 2 * n6 * sizeof(float) : 0);
                if (avail < margin + per * (size_t)mpp)
                    mpp = avail > margin + per ? (int)std::min<size_t>((avail - margin) / per, (size_t)mpp) : 1;
            } else {
                cudaGetLastError();
            }
        }
    }

    // workspaces
    if ((rc = ensure(g->state, 2 * n6 * sizeof(T) * (size_t)mpp))) return rc;
    const bool probes = probe_dev && nprb > 0 && probe_rows > 0;
    if (probes && (rc = ensure(g->pm, sizeof(double) * (size_t)probe_rows * nprb * nm_total))) return rc;
    if (nsrc > 0) {
        if ((rc = ensure(g->amp, sizeof(double) * (size_t)amp_len * nsrc))) return rc;
        if ((rc = ensure(g->srcdev, sizeof(fit_source) * nsrc))) return rc;
        FIT_CHECK(cudaMemcpyAsync(g->srcdev.p, src, sizeof(fit_source) * nsrc, cudaMemcpyHostToDevice, s));
        FIT_CHECK(source_table((const fit_source *)g->srcdev.p, nsrc, amp_base, amp_len, dt, (double *)g->amp.p, s));
        g->stats.kernel_launches += 1;
    }
    if ((rc = ensure(g->memdev, sizeof(Member) * (size_t)mpp))) return rc;
    if ((rc = ensure(g->err, sizeof(int)))) return rc;
    FIT_CHECK(cudaMemsetAsync(g->err.p, 0, sizeof(int), s));
    if (probes) FIT_CHECK(cudaMemsetAsync(g->pm.p, 0, sizeof(double) * (size_t)probe_rows * nprb * nm_total, s));
    if (energy_dev) FIT_CHECK(cudaMemsetAsync(energy_dev, 0, sizeof(double) * (size_t)specs_in[0].nit, s));
    const bool kahan = sum_mode == 1 && acc_e && !comp && !resf;
    if (kahan) {
        if ((rc = ensure(g->kahan, 2 * n6 * sizeof(float)))) return rc;
        FIT_CHECK(cudaMemsetAsync(g->kahan.p, 0, 2 * n6 * sizeof(float), s));
    }
    if (acc_e) FIT_CHECK(cudaMemsetAsync(acc_e, 0, 3 * ncp * sizeof(double), s));
    if (acc_h) FIT_CHECK(cudaMemsetAsync(acc_h, 0, 3 * ncp * sizeof(double), s));

    StepArgs<T> a;
    memset(&a, 0, sizeof(a));
    Tile tile = pick_tile(g, opts);
    a.nx = g->nx; a.ny = g->ny; a.nz = g->nz; a.pitch = g->pitch; a.ncell = ncp;
    a.tiles_x = (g->nx + tile.tx - 1) / tile.tx;
    a.tiles_y = (g->ny + tile.ty - 1) / tile.ty;
    a.kz = tile.kz;
    a.nchunk = (g->nz + tile.kz - 1) / tile.kz;
    a.cb = (const T *)g->coef.p;
    a.ca = g->lossy ? (const T *)g->coef.p + 3 * ncp : nullptr;
    a.ch = (const T *)g->ch.p;
    a.meps = energy_dev ? (const T *)g->meps.p : nullptr;
    a.mmu = energy_dev ? (const T *)g->mmu.p : nullptr;
    a.mem = (const Member *)g->memdev.p;
    a.amp = (const double *)g->amp.p;
    a.amp_base = amp_base;
    a.amp_len = amp_len;
    a.nsrc = nsrc;
    for (int q = 0; q < nsrc; ++q) a.src[q] = {src[q].axis, src[q].i, src[q].j, src[q].k};
    a.nprb = probes ? nprb : 0;
    for (int q = 0; q < nprb; ++q) a.prb[q] = {prb[q].axis, prb[q].i, prb[q].j, prb[q].k};
    a.err = (int *)g->err.p;
    a.wait_limit = opts ? std::max(0, opts->debug_wait_limit) : 0;
    a.extra_tx = opts ? std::max(0, opts->debug_extra_tx) : 0;
    TmaMaps maps;
    if (resf) {
        if (!res_tile_supported(tile.tx, tile.ty)) tile.tx = 64, tile.ty = 4;
        if (!encode_tma_maps(&maps, (int)sizeof(T), g->nx, g->ny, g->nz, g->pitch, g->state.p, 2 * mpp, g->coef.p,
                             g->lossy ? 6 : 3, tile.tx, tile.ty, 9))
            return FIT_ERR_UNSUPPORTED;
    } else if (comp) {
        if (!comp_tile_supported(tile.tx, tile.ty)) tile.tx = 32, tile.ty = 8;
        if (!encode_tma_maps(&maps, (int)sizeof(T), g->nx, g->ny, g->nz, g->pitch, g->state.p, 2 * mpp, g->coef.p,
                             g->lossy ? 6 : 3, tile.tx, tile.ty, 12))
            return FIT_ERR_UNSUPPORTED;
    } else if (tile.kernel == 2 &&
               !encode_tma_maps(&maps, (int)sizeof(T), g->nx, g->ny, g->nz, g->pitch, g->state.p, 2 * mpp,
                                g->coef.p, g->lossy ? 6 : 3, tile.tx, tile.ty)) {
        tile.kernel = 1;
        if (!tile_supported(tile.tx, tile.ty)) tile.tx = 32, tile.ty = 8;
    }

    // member 0's final state -> (final_e, final_h): compact rows of T, or FP64
    // joined from the hi/lo pairs of a compensated grid
    auto copy_out = [&](const T *fin) -> int {
        for (int part = 0; part < 2; ++part) {
            void *dst = part ? final_h : final_e;
            if (!dst) continue;
            if (!comp && !resf) {
                FIT_CHECK(cudaMemcpy2DAsync(dst, row, fin + 3 * part * ncp, prow, row, rows3, kind_from_dev(dst), s));
                continue;
            }
            double *dout = (double *)dst;
            const bool host = !is_device(dst);
            if (host) {
                int r2;
                if ((r2 = ensure(g->stage, 3 * (size_t)ncell * sizeof(double)))) return r2;
                dout = (double *)g->stage.p;
            }
            if (resf)
                FIT_CHECK(join_res(g->nx, g->ny, g->nz, g->pitch, (const float *)fin, part, dout, s));
            else
                FIT_CHECK(join_pairs(g->nx, g->ny, g->nz, g->pitch, (const float *)(fin + 3 * part * ncp),
                                     (const float *)(fin + (6 + 3 * part) * ncp), dout, s));
            if (host)
                FIT_CHECK(cudaMemcpyAsync(dst, dout, 3 * (size_t)ncell * sizeof(double), cudaMemcpyDeviceToHost, s));
        }
        return FIT_OK;
    };

    // two steps per launch (FP32, TMA, no energy): the temporal-blocking kernel
    bool two = false;
    TmaMaps maps2;
    CUtensorMap coefwin;
    Tile tile2 = {32, 8, tile.kz, 2, 3};
    if (opts && opts->steps_per_launch == 2 && sizeof(T) == 4 && !comp && !resf && !energy_dev &&
        tile.kernel == 2) {
        if (opts->tile_x > 0 && opts->tile_y > 0 && step2_tile_supported(opts->tile_x, opts->tile_y))
            tile2.tx = opts->tile_x, tile2.ty = opts->tile_y;
        two = encode_tma_maps(&maps2, 4, g->nx, g->ny, g->nz, g->pitch, g->state.p, 2 * mpp, g->coef.p,
                              g->lossy ? 6 : 3, tile2.tx, tile2.ty + 2) &&
              encode_window_map(&coefwin, 4, g->nx, g->ny, g->nz, g->pitch, g->coef.p, g->lossy ? 6 : 3,
                                tile2.tx + 8, tile2.ty + 4, g->lossy ? 6 : 3);
    }
    StepArgs<T> a2 = a;
    if (two) {
        a2.tiles_x = (g->nx + tile2.tx - 1) / tile2.tx;
        a2.tiles_y = (g->ny + tile2.ty - 1) / tile2.ty;
        a2.kz = (opts && opts->tile_z > 0) ? opts->tile_z : 64;
        const long long cols2 = (long long)a2.tiles_x * a2.tiles_y;
        while (a2.kz > 8 && cols2 * ((g->nz + a2.kz - 1) / a2.kz) < 2 * 152) a2.kz /= 2;
        a2.nchunk = (g->nz + a2.kz - 1) / a2.kz;
    }

    // z chunks (unless the caller fixed them): from the step kernel's CTAs per SM, asked
    // of the launch call itself, for the largest group here and again for every launch
    // whose number of active members differs from the previous one's
    const Tile chunk_tile = tile;   // the tile's default chunk as the longest
    long long chunk_slots = 0;
    int chunk_nsm = 152;
    {
        int per_sm = 0, nsm = 0, dev = 0;
        cudaError_t qe = cudaGetDevice(&dev);
        if (qe == cudaSuccess) qe = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (qe == cudaSuccess && !two && !tile.kz_fixed) {
            StepArgs<T> q = a;
            q.occ_out = &per_sm;
            if (resf)
                qe = launch_step_res((const StepArgs<float> &)q, maps, tile, g->lossy, g->mu_array, energy_dev != nullptr,
                                     s);
            else if (comp)
                qe = launch_step_comp((const StepArgs<float> &)q, maps, tile, g->lossy, g->mu_array,
                                      energy_dev != nullptr, s);
            else if (tile.kernel == 2)
                qe = launch_step_tma<T>(q, maps, tile, g->lossy, g->mu_array, energy_dev != nullptr, s);
            else
                qe = launch_step<T>(q, tile, g->lossy, g->mu_array, energy_dev != nullptr, s);
        }
        if (qe != cudaSuccess) {
            cudaGetLastError();
            per_sm = 0;
        }
        chunk_slots = (long long)per_sm * nsm;
        chunk_nsm = nsm > 0 ? nsm : 152;
        tile.kz = chunk_length(g->nx, g->ny, g->nz, chunk_tile, mpp, chunk_slots, chunk_nsm);
        a.kz = tile.kz;
        a.nchunk = (g->nz + tile.kz - 1) / tile.kz;
    }
    int chunk_members = mpp;   // the member count a.kz was chosen for

    // Passes over groups of members from the end of the table (shortest members) to
    // its start, the first group taking the remainder, so that the long members that
    // set the launch count share their launches with full groups.  Inside a group
    // members finish shortest first, so the superposition adds members in decreasing
    // table order whatever members_per_pass is.
    const int npass = (nm_total + mpp - 1) / mpp;
    auto group = [&](int pass) { return pass == 0 ? nm_total - (npass - 1) * mpp : mpp; };
    for (int pass = 0, g_end = nm_total; g_end > 0; g_end -= group(pass++)) {
        const int cnt = group(pass);
        const int first = g_end - cnt;
        std::vector<Member> mem(cnt);
        for (int q = 0; q < cnt; ++q) {
            const MemberSpec &sp = specs_in[order[first + q]];
            T *base = (T *)g->state.p + 2 * n6 * (size_t)q;
            mem[q].st[0] = base;
            mem[q].st[1] = base + n6;
            mem[q].blk[0] = 2 * q;
            mem[q].blk[1] = 2 * q + 1;
            mem[q].start = sp.start;
            mem[q].end = sp.start + sp.nit;
            mem[q].src_lo = sp.src_lo;
            mem[q].src_hi = sp.src_hi;
            mem[q].probe = probes ? (double *)g->pm.p + (size_t)order[first + q] * probe_rows * nprb : nullptr;
            mem[q].probe_base = probe_base;
            mem[q].energy = (energy_dev && order[first + q] == 0) ? energy_dev : nullptr;
            mem[q].energy_base = sp.start;
            // initial state into buffer 0
            FIT_CHECK(cudaMemsetAsync(base, 0, n6 * sizeof(T), s));
            if (resf && (sp.e0 || sp.h0)) {   // FP64 compact input -> floats + residual words (masked)
                const double *din[2] = {(const double *)sp.e0, (const double *)sp.h0};
                const size_t n3d = 3 * (size_t)ncell * sizeof(double);
                for (int part = 0; part < 2; ++part) {
                    if (!din[part] || is_device(din[part])) continue;
                    if ((rc = ensure(g->stage, 2 * n3d))) return rc;
                    double *dst = (double *)g->stage.p + part * 3 * (size_t)ncell;
                    FIT_CHECK(cudaMemcpyAsync(dst, din[part], n3d, cudaMemcpyHostToDevice, s));
                    din[part] = dst;
                }
                FIT_CHECK(split_res(g->nx, g->ny, g->nz, g->pitch, din[0], din[1], (float *)base, s));
                g->stats.kernel_launches += 1;
            } else if (comp) {   // FP64 compact input -> hi/lo pairs (masked to the degrees of freedom)
                for (int part = 0; part < 2; ++part) {
                    const void *src0 = part ? sp.h0 : sp.e0;
                    if (!src0) continue;
                    const double *din = (const double *)src0;
                    if (!is_device(src0)) {
                        if ((rc = ensure(g->stage, 3 * (size_t)ncell * sizeof(double)))) return rc;
                        FIT_CHECK(cudaMemcpyAsync(g->stage.p, src0, 3 * (size_t)ncell * sizeof(double),
                                                  cudaMemcpyHostToDevice, s));
                        din = (const double *)g->stage.p;
                    }
                    FIT_CHECK(split_pairs(g->nx, g->ny, g->nz, g->pitch, din, (float *)(base + 3 * part * ncp),
                                          (float *)(base + (6 + 3 * part) * ncp), part, s));
                    g->stats.kernel_launches += 1;
                }
            } else {
                if (sp.e0)
                    FIT_CHECK(cudaMemcpy2DAsync(base, prow, sp.e0, row, row, rows3, kind_to_dev(sp.e0), s));
                if (sp.h0)
                    FIT_CHECK(cudaMemcpy2DAsync(base + 3 * ncp, prow, sp.h0, row, row, rows3, kind_to_dev(sp.h0), s));
            }
            if (!comp && !resf && (sp.e0 || sp.h0)) {
                FIT_CHECK(mask_state<T>(g->nx, g->ny, g->nz, g->pitch, base, base + 3 * ncp, s));
                g->stats.kernel_launches += 1;
            }
        }
        FIT_CHECK(cudaMemcpyAsync(g->memdev.p, mem.data(), sizeof(Member) * cnt, cudaMemcpyHostToDevice, s));
        // the host table must outlive the async copy
        FIT_CHECK(cudaStreamSynchronize(s));

        const long long nit_max = specs_in[order[first]].nit;
        int active = cnt;
        // a member that took its last step in the launch just issued, whose final
        // state is `fin`: superposition, copy-out, keep
        auto finish_member = [&](int q, const T *fin) -> int {
            if (acc_e) {
                if (kahan) {
                    float *ks = (float *)g->kahan.p;
                    FIT_CHECK(accumulate_state_kahan<T>((long long)n6, fin, ks, ks + n6, s));
                } else {
                    FIT_CHECK(accumulate_state<T>(3 * ncp, fin, acc_e, s));
                    if (acc_h) FIT_CHECK(accumulate_state<T>(3 * ncp, fin + 3 * ncp, acc_h, s));
                }
                g->stats.kernel_launches += 1;
            }
            if (order[first + q] == 0) {
                int r2 = copy_out(fin);
                if (r2) return r2;
            }
            if (keep_final && keep_final[order[first + q]])
                FIT_CHECK(cudaMemcpyAsync(keep_final[order[first + q]], fin, n6 * sizeof(T), cudaMemcpyDeviceToDevice,
                                          s));
            return FIT_OK;
        };
        for (long long it = 0, L = 0; two && it < nit_max; it += 2, ++L) {
            while (active > 0 && specs_in[order[first + active - 1]].nit <= it) --active;
            a2.nmem = active;
            a2.it = (int)it;
            a2.parity = (int)(L & 1);
            if (profile) {
                while ((long long)g->ev.size() < 2 * (nev + 1)) {
                    cudaEvent_t e;
                    FIT_CHECK(cudaEventCreate(&e));
                    g->ev.push_back(e);
                }
                FIT_CHECK(cudaEventRecord(g->ev[2 * nev], s));
            }
            FIT_CHECK(launch_step2_tma((const StepArgs<float> &)a2, maps2.state, coefwin, tile2.tx, tile2.ty, g->lossy,
                                       g->mu_array, s));
            if (profile) {
                FIT_CHECK(cudaEventRecord(g->ev[2 * nev + 1], s));
                ++nev;
            }
            g->stats.step_launches += 1;
            g->stats.kernel_launches += 1;
            // algorithmic bytes are counted per step as for the one-step kernel
            int two_steps = 0;
            for (int q = 0; q < active; ++q) {
                const long long left = specs_in[order[first + q]].nit - it;
                const int st = left >= 2 ? 2 : 1;
                g->stats.cell_updates += (long long)st * ncell;
                g->stats.alg_bytes += fld_bytes * st;
                if (st == 2) two_steps = 1;
            }
            g->stats.alg_bytes += coef_bytes * (two_steps ? 2 : 1);
            for (int q = active - 1; q >= 0; --q) {
                const long long left = specs_in[order[first + q]].nit - it;
                if (left > 2) continue;
                int r2 = finish_member(q, (const T *)mem[q].st[(L + 1) & 1]);
                if (r2) return r2;
            }
        }
        for (long long it = 0; !two && it < nit_max; ++it) {
            while (active > 0 && specs_in[order[first + active - 1]].nit <= it) --active;
            a.nmem = active;
            if (active != chunk_members && chunk_slots > 0 && !two) {
                a.kz = chunk_length(g->nx, g->ny, g->nz, chunk_tile, active, chunk_slots, chunk_nsm);
                a.nchunk = (g->nz + a.kz - 1) / a.kz;
                chunk_members = active;
            }
            a.it = (int)it;
            a.parity = (int)(it & 1);
            if (profile) {
                while ((long long)g->ev.size() < 2 * (nev + 1)) {
                    cudaEvent_t e;
                    FIT_CHECK(cudaEventCreate(&e));
                    g->ev.push_back(e);
                }
                FIT_CHECK(cudaEventRecord(g->ev[2 * nev], s));
            }
            if (resf)
                FIT_CHECK(launch_step_res((const StepArgs<float> &)a, maps, tile, g->lossy, g->mu_array,
                                          energy_dev != nullptr, s));
            else if (comp)
                FIT_CHECK(launch_step_comp((const StepArgs<float> &)a, maps, tile, g->lossy, g->mu_array,
                                           energy_dev != nullptr, s));
            else if (tile.kernel == 2)
                FIT_CHECK(launch_step_tma<T>(a, maps, tile, g->lossy, g->mu_array, energy_dev != nullptr, s));
            else
                FIT_CHECK(launch_step<T>(a, tile, g->lossy, g->mu_array, energy_dev != nullptr, s));
            if (profile) {
                FIT_CHECK(cudaEventRecord(g->ev[2 * nev + 1], s));
                ++nev;
            }
            g->stats.step_launches += 1;
            g->stats.kernel_launches += 1;
            g->stats.cell_updates += (long long)active * ncell;
            g->stats.alg_bytes += fld_bytes * active + coef_bytes;
            // members that just took their last step, shortest first (table end first)
            for (int q = active - 1; q >= 0; --q) {
                const MemberSpec &sp = specs_in[order[first + q]];
                if (sp.nit != it + 1) continue;
                const T *fin = (const T *)mem[q].st[(it + 1) & 1];
                if (acc_e) {
                    if (kahan) {
                        float *ks = (float *)g->kahan.p;
                        FIT_CHECK(accumulate_state_kahan<T>((long long)n6, fin, ks, ks + n6, s));
                        g->stats.kernel_launches += 1;
                    } else if (resf) {
                        FIT_CHECK(accumulate_res(ncp, (const float *)fin, 0, acc_e, s));
                        g->stats.kernel_launches += 1;
                        if (acc_h) {
                            FIT_CHECK(accumulate_res(ncp, (const float *)fin, 1, acc_h, s));
                            g->stats.kernel_launches += 1;
                        }
                    } else if (comp) {
                        FIT_CHECK(accumulate_pairs(3 * ncp, (const float *)fin, (const float *)(fin + 6 * ncp),
                                                   acc_e, s));
                        g->stats.kernel_launches += 1;
                        if (acc_h) {
                            FIT_CHECK(accumulate_pairs(3 * ncp, (const float *)(fin + 3 * ncp),
                                                       (const float *)(fin + 9 * ncp), acc_h, s));
                            g->stats.kernel_launches += 1;
                        }
                    } else {
                        FIT_CHECK(accumulate_state<T>(3 * ncp, fin, acc_e, s));
                        g->stats.kernel_launches += 1;
                        if (acc_h) {
                            FIT_CHECK(accumulate_state<T>(3 * ncp, fin + 3 * ncp, acc_h, s));
                            g->stats.kernel_launches += 1;
                        }
                    }
                }
                if (order[first + q] == 0 && (rc = copy_out(fin))) return rc;
                if (keep_final && keep_final[order[first + q]])
                    FIT_CHECK(cudaMemcpyAsync(keep_final[order[first + q]], fin, n6 * sizeof(T),
                                              cudaMemcpyDeviceToDevice, s));
            }
        }
        // zero-length members: their final state is the initial one
        for (int q = 0; q < cnt; ++q) {
            const MemberSpec &sp = specs_in[order[first + q]];
            if (sp.nit > 0) continue;
            const T *fin = (const T *)mem[q].st[0];
            if (acc_e && resf) {
                FIT_CHECK(accumulate_res(ncp, (const float *)fin, 0, acc_e, s));
                if (acc_h) FIT_CHECK(accumulate_res(ncp, (const float *)fin, 1, acc_h, s));
            } else if (acc_e && comp) {
                FIT_CHECK(accumulate_pairs(3 * ncp, (const float *)fin, (const float *)(fin + 6 * ncp), acc_e, s));
                if (acc_h)
                    FIT_CHECK(accumulate_pairs(3 * ncp, (const float *)(fin + 3 * ncp), (const float *)(fin + 9 * ncp),
                                               acc_h, s));
            } else if (acc_e && !kahan) {
                FIT_CHECK(accumulate_state<T>(3 * ncp, fin, acc_e, s));
                if (acc_h) FIT_CHECK(accumulate_state<T>(3 * ncp, fin + 3 * ncp, acc_h, s));
            } else if (kahan) {
                float *ks = (float *)g->kahan.p;
                FIT_CHECK(accumulate_state_kahan<T>((long long)n6, fin, ks, ks + n6, s));
            }
            if (order[first + q] == 0 && (rc = copy_out(fin))) return rc;
        }
    }
    if (kahan) {
        float *ks = (float *)g->kahan.p;
        FIT_CHECK(kahan_finish(3 * ncp, ks, ks + n6, acc_e, s));
        if (acc_h) FIT_CHECK(kahan_finish(3 * ncp, ks + 3 * ncp, ks + n6 + 3 * ncp, acc_h, s));
    }
    if (kahan) g->stats.kernel_launches += acc_h ? 2 : 1;
    if (probes) {
        FIT_CHECK(sum_members(nm_total, probe_rows * nprb, (const double *)g->pm.p, probe_rows * nprb, probe_dev, s));
        g->stats.kernel_launches += 1;
    }
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
    return FIT_OK;
}


template int run_members<float>(fit_grid *, double, int, const std::vector<MemberSpec> &, long long, long long,
                                const fit_source *, int, const fit_probe *, int, long long, long long, double *,
                                double *, int, double *, double *, void *, void *, const fit_run_opts *,
                                cudaStream_t, float *const *);
template int run_members<double>(fit_grid *, double, int, const std::vector<MemberSpec> &, long long, long long,
                                 const fit_source *, int, const fit_probe *, int, long long, long long, double *,
                                 double *, int, double *, double *, void *, void *, const fit_run_opts *,
                                 cudaStream_t, double *const *);

}  // namespace fitgb

namespace {

template <typename T>
int leapfrog_impl(fit_grid *g, double dt, long nsteps, long step0, const fit_source *src, int nsrc,
                  const fit_probe *prb, int nprb, double *probe_out, double *energy_out, void *e_io, void *h_io,
                  const fit_run_opts *opts, cudaStream_t s) {
    int rc;
    const int scheme = opts ? opts->sigma_scheme : 0;
    const bool host_out = (probe_out && !is_device(probe_out)) || (energy_out && !is_device(energy_out)) ||
                          (e_io && !is_device(e_io)) || (h_io && !is_device(h_io));
    double *pdev = nullptr, *edev = nullptr;
    if (probe_out && nprb > 0) {
        if (is_device(probe_out)) pdev = probe_out;
        else {
            if ((rc = ensure(g->probe_ws, sizeof(double) * (size_t)nsteps * nprb))) return rc;
            pdev = (double *)g->probe_ws.p;
        }
    }
    if (energy_out) {
        if (is_device(energy_out)) edev = energy_out;
        else {
            if ((rc = ensure(g->energy, sizeof(double) * (size_t)nsteps))) return rc;
            edev = (double *)g->energy.p;
        }
    }
    std::vector<MemberSpec> specs(1);
    specs[0] = {step0, nsteps, -(1LL << 62), (1LL << 62), e_io, h_io};
    rc = run_members<T>(g, dt, scheme, specs, step0, nsteps, src, nsrc, prb, nprb, step0, nsteps, pdev, edev, 0,
                        nullptr, nullptr, e_io, h_io, opts, s);
    if (rc) return rc;
    if (pdev && pdev != probe_out)
        FIT_CHECK(cudaMemcpyAsync(probe_out, pdev, sizeof(double) * (size_t)nsteps * nprb, cudaMemcpyDeviceToHost, s));
    if (edev && edev != energy_out)
        FIT_CHECK(cudaMemcpyAsync(energy_out, edev, sizeof(double) * (size_t)nsteps, cudaMemcpyDeviceToHost, s));
    return finish(g, s, host_out);
}

template <typename T>
int paraexp_impl(fit_grid *g, double dt, int K, const long *win, const fit_source *src, int nsrc,
                 const fit_probe *prb, int nprb, double *probe_out, double *e_final, double *h_final,
                 const void *e0, const void *h0, const fit_run_opts *opts, cudaStream_t s) {
    int rc;
    const int scheme = opts ? opts->sigma_scheme : 0;
    const long long W0 = win[0], WK = win[K], nt = WK - W0;
    std::vector<MemberSpec> specs;
    if (e0 || h0) specs.push_back({W0, nt, 0, 0, e0, h0});   // w_1: homogeneous, from u0
    for (int j = 1; j <= K; ++j) specs.push_back({win[j - 1], WK - win[j - 1], win[j - 1], win[j], nullptr, nullptr});
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
    const size_t n3 = 3 * (size_t)g->ncp;
    if (e_final || h_final) {
        if ((rc = ensure(g->acc, 2 * n3 * sizeof(double)))) return rc;
        ae = (double *)g->acc.p;
        ah = ae + n3;
    }
    const int sum_mode = opts ? opts->sum_mode : 0;
    rc = run_members<T>(g, dt, scheme, specs, W0, nt, src, nsrc, prb, nprb, W0, nt, pdev, nullptr, sum_mode, ae, ah,
                        nullptr, nullptr, opts, s);
    if (rc) return rc;
    if (pdev && pdev != probe_out)
        FIT_CHECK(cudaMemcpyAsync(probe_out, pdev, sizeof(double) * (size_t)nt * nprb, cudaMemcpyDeviceToHost, s));
    const size_t row = (size_t)g->nx * sizeof(double), prow = (size_t)g->pitch * sizeof(double);
    const size_t rows3 = 3 * (size_t)g->ny * g->nz;
    if (e_final) FIT_CHECK(cudaMemcpy2DAsync(e_final, row, ae, prow, row, rows3, kind_from_dev(e_final), s));
    if (h_final) FIT_CHECK(cudaMemcpy2DAsync(h_final, row, ah, prow, row, rows3, kind_from_dev(h_final), s));
    return finish(g, s, host_out);
}

}  // namespace

extern "C" {

const char *fit_version(void) { return "fitgb 0.1 (sm_103a)"; }

const char *fit_strerror(int st) {
    switch (st) {
    case FIT_OK: return "ok";
    case FIT_ERR_ARG: return "invalid argument";
    case FIT_ERR_CFL: return "time step above the CFL estimate";
    case FIT_ERR_OOM: return "device out of memory";
    case FIT_ERR_CUDA: return "CUDA runtime error";
    case FIT_ERR_TIMEOUT: return "device wait timed out";
    case FIT_ERR_NONFINITE: return "non-finite or non-positive material";
    case FIT_ERR_UNSUPPORTED: return "unsupported request";
    default: return "unknown status";
    }
}

int fit_grid_create(int nx, int ny, int nz, double dx, double dy, double dz, const float *eps_r,
                    const float *mu_r, const float *sigma, int precision, unsigned flags, fit_grid **out) {
    if (!out) return FIT_ERR_ARG;
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1 || !eps_r) return FIT_ERR_ARG;
    if (flags & ~FIT_FLAG_COEF_FLOAT) return FIT_ERR_ARG;
    if (any_foreign({eps_r, mu_r, sigma})) return FIT_ERR_ARG;
    if (!(dx > 0) || !(dy > 0) || !(dz > 0) || !std::isfinite(dx) || !std::isfinite(dy) || !std::isfinite(dz))
        return FIT_ERR_ARG;
    if (precision != 32 && precision != 64 && precision != 48 && precision != 40) return FIT_ERR_ARG;
    const long long ncell = (long long)nx * ny * nz;
    if (ncell > (1LL << 34)) return FIT_ERR_ARG;
    fit_grid *g = new (std::nothrow) fit_grid();
    if (!g) return FIT_ERR_OOM;
    g->nx = nx; g->ny = ny; g->nz = nz;
    g->d[0] = dx; g->d[1] = dy; g->d[2] = dz;
    g->prec = precision;
    g->flags = flags;
    g->ncell = ncell;
    g->pitch = pitch_of(nx);
    g->ncp = (long long)g->pitch * ny * nz;
    const size_t bytes = sizeof(float) * (size_t)ncell;
    cudaStream_t s = 0;
    auto fail = [&](int rc) {
        fit_grid_destroy(g);
        return rc;
    };
    cudaError_t ae;
    if ((ae = dev_alloc((void **)&g->eps, bytes)) != cudaSuccess) { cudaGetLastError(); return fail(map_err(ae)); }
    if (cudaMemcpy(g->eps, eps_r, bytes, kind_to_dev(eps_r)) != cudaSuccess) return fail(FIT_ERR_CUDA);
    if (mu_r) {
        if ((ae = dev_alloc((void **)&g->mu, bytes)) != cudaSuccess) { cudaGetLastError(); return fail(map_err(ae)); }
        if (cudaMemcpy(g->mu, mu_r, bytes, kind_to_dev(mu_r)) != cudaSuccess) return fail(FIT_ERR_CUDA);
    }
    if (sigma) {
        if ((ae = dev_alloc((void **)&g->sig, bytes)) != cudaSuccess) { cudaGetLastError(); return fail(map_err(ae)); }
        if (cudaMemcpy(g->sig, sigma, bytes, kind_to_dev(sigma)) != cudaSuccess) return fail(FIT_ERR_CUDA);
    }
    if (ensure(g->scratch, 64)) return fail(FIT_ERR_OOM);
    MaterialFlags mf;
    if (check_materials(g->eps, g->mu, g->sig, ncell, &mf, g->scratch.p, s) != cudaSuccess) return fail(FIT_ERR_CUDA);
    if (mf.bad_eps || mf.bad_mu || mf.bad_sigma) return fail(FIT_ERR_NONFINITE);
    g->mu_array = mf.mu_nonuniform != 0;
    g->lossy = mf.lossy != 0;
    g->eps_mu_min = mf.eps_mu_min;
    *out = g;
    return FIT_OK;
}

int fit_grid_create_graded(int nx, int ny, int nz, const double *dx, const double *dy, const double *dz,
                           const float *eps_r, const float *mu_r, const float *sigma, int precision, unsigned flags,
                           fit_grid **out) {
    if (!out) return FIT_ERR_ARG;
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1 || !dx || !dy || !dz) return FIT_ERR_ARG;
    const double *ds[3] = {dx, dy, dz};
    const int n[3] = {nx, ny, nz};
    std::vector<double> spc;
    double mean[3] = {0, 0, 0};
    for (int a = 0; a < 3; ++a)
        for (int i = 0; i < n[a]; ++i) {
            const double v = ds[a][i];
            if (!(v > 0.0) || !std::isfinite(v)) return FIT_ERR_ARG;
            spc.push_back(v);
            mean[a] += v / n[a];
        }
    fit_grid *g = nullptr;
    int rc = fit_grid_create(nx, ny, nz, mean[0], mean[1], mean[2], eps_r, mu_r, sigma, precision, flags, &g);
    if (rc) return rc;
    if (ensure(g->spc, spc.size() * sizeof(double)) ||
        cudaMemcpy(g->spc.p, spc.data(), spc.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
        fit_grid_destroy(g);
        return FIT_ERR_OOM;
    }
    g->graded = true;
    g->spc_host = spc;
    g->mu_array = true;   // ch varies per face
    if (graded_cfl_and_bound(nx, ny, nz, (const double *)g->spc.p, g->eps, g->mu, g->scratch.p, &g->cfl_graded,
                             &g->rowsum, 0) != cudaSuccess) {
        fit_grid_destroy(g);
        return FIT_ERR_CUDA;
    }
    *out = g;
    return FIT_OK;
}

void fit_grid_destroy(fit_grid *g) {
    if (!g) return;
    cudaDeviceSynchronize();
    if (g->eps) cudaFree(g->eps);
    if (g->mu) cudaFree(g->mu);
    if (g->sig) cudaFree(g->sig);
    Buf *bufs[] = {&g->coef, &g->ch, &g->meps, &g->mmu, &g->state, &g->pm, &g->amp, &g->srcdev,
                   &g->memdev, &g->acc, &g->kahan, &g->stage, &g->energy, &g->scratch, &g->probe_ws, &g->err,
                   &g->ckpt, &g->ring, &g->lam, &g->gacc, &g->aprobe, &g->aamp, &g->adjmem, &g->scalar,
                   &g->grad_ws, &g->xblocks, &g->xtab, &g->xbasis, &g->xpm, &g->spc, &g->gblk, &g->dhist};
    for (Buf *b : bufs) release(*b);
    for (cudaEvent_t e : g->ev) cudaEventDestroy(e);
    delete g;
}

int fit_cfl_dt(const fit_grid *g, double *dt_out) {
    if (!g || !dt_out) return FIT_ERR_ARG;
    *dt_out = cfl_of(g);
    return FIT_OK;
}

int fit_grid_info(const fit_grid *g, int *nx, int *ny, int *nz, int *precision, int *lossy) {
    if (!g) return FIT_ERR_ARG;
    if (nx) *nx = g->nx;
    if (ny) *ny = g->ny;
    if (nz) *nz = g->nz;
    if (precision) *precision = g->prec;
    if (lossy) *lossy = g->lossy ? 1 : 0;
    return FIT_OK;
}

int fit_leapfrog_run(fit_grid *g, double dt, long nsteps, long step0, const fit_source *src, int nsrc,
                     const fit_probe *prb, int nprb, double *probe_out, double *energy_out, void *e_io, void *h_io,
                     const fit_run_opts *opts, void *stream) {
    if (!g || nsteps < 0) return FIT_ERR_ARG;
    if (any_foreign({probe_out, energy_out, e_io, h_io})) return FIT_ERR_ARG;
    int rc;
    if ((rc = check_dt(g, dt, opts))) return rc;
    if ((rc = check_sources_probes(g, src, nsrc, prb, nprb))) return rc;
    if (opts && (opts->sigma_scheme < 0 || opts->sigma_scheme > 1)) return FIT_ERR_ARG;
    if (nsteps == 0) return FIT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (g->prec == 64)
        return leapfrog_impl<double>(g, dt, nsteps, step0, src, nsrc, prb, nprb, probe_out, energy_out, e_io, h_io,
                                     opts, s);
    if ((g->prec == 48 || g->prec == 40) && opts && opts->kernel == 1) return FIT_ERR_UNSUPPORTED;
    return leapfrog_impl<float>(g, dt, nsteps, step0, src, nsrc, prb, nprb, probe_out, energy_out, e_io, h_io, opts,
                                s);
}

int paraexp_run(fit_grid *g, double dt, int K, const long *win, const fit_source *src, int nsrc,
                const fit_probe *prb, int nprb, double *probe_out, double *e_final, double *h_final,
                const void *e0, const void *h0, const fit_run_opts *opts, void *stream) {
    if (!g || K < 1 || !win) return FIT_ERR_ARG;
    if (any_foreign({probe_out, e_final, h_final, e0, h0})) return FIT_ERR_ARG;
    for (int j = 1; j <= K; ++j)
        if (win[j] <= win[j - 1]) return FIT_ERR_ARG;
    int rc;
    if ((rc = check_dt(g, dt, opts))) return rc;
    if ((rc = check_sources_probes(g, src, nsrc, prb, nprb))) return rc;
    if (opts && (opts->sigma_scheme < 0 || opts->sigma_scheme > 1 || opts->sum_mode < 0 || opts->sum_mode > 1))
        return FIT_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (opts && opts->homogeneous != FIT_HOMOG_LEAPFROG) {
        if (opts->homogeneous != FIT_HOMOG_LEJA && opts->homogeneous != FIT_HOMOG_TAYLOR) return FIT_ERR_ARG;
        if (opts->sum_mode != 0) return FIT_ERR_ARG;
        if (g->prec == 48 || g->prec == 40 || g->lossy) return FIT_ERR_UNSUPPORTED;
        if (g->prec == 64)
            return paraexp_expo_impl<double>(g, dt, K, win, src, nsrc, prb, nprb, probe_out, e_final, h_final, e0,
                                             h0, opts, s);
        return paraexp_expo_impl<float>(g, dt, K, win, src, nsrc, prb, nprb, probe_out, e_final, h_final, e0, h0,
                                        opts, s);
    }
    if (g->prec == 64)
        return paraexp_impl<double>(g, dt, K, win, src, nsrc, prb, nprb, probe_out, e_final, h_final, e0, h0, opts, s);
    if ((g->prec == 48 || g->prec == 40) && opts && (opts->kernel == 1 || opts->sum_mode == 1))
        return FIT_ERR_UNSUPPORTED;
    return paraexp_impl<float>(g, dt, K, win, src, nsrc, prb, nprb, probe_out, e_final, h_final, e0, h0, opts, s);
}

int fit_last_stats(const fit_grid *g, fit_run_stats *out) {
    if (!g || !out) return FIT_ERR_ARG;
    *out = g->stats;
    return FIT_OK;
}

int fit_debug_fail_alloc(long long after) {
    g_fail_alloc.store(after < 0 ? -1 : after);
    return FIT_OK;
}

int fit_debug_chunk_length(int nx, int ny, int nz, int tile_x, int tile_y, int kz_max, int nmem, long long slots) {
    if (nx < 1 || ny < 1 || nz < 1 || tile_x < 1 || tile_y < 1 || kz_max < 1 || nmem < 1) return FIT_ERR_ARG;
    Tile t{tile_x, tile_y, kz_max, 2};
    return chunk_length(nx, ny, nz, t, nmem, slots, 152);
}

int fit_sync(fit_grid *g, void *stream) {
    if (!g) return FIT_ERR_ARG;
    return finish(g, (cudaStream_t)stream, true);
}

}  // extern "C"
