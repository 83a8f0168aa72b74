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
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

using namespace fitgb;

namespace {

struct Buf {
    void *p = nullptr;
    size_t n = 0;
};

}  // namespace

struct fit_grid {
    int nx = 0, ny = 0, nz = 0;
    double d[3] = {0, 0, 0};
    int prec = 32;
    long long ncell = 0;   // nx*ny*nz
    int pitch = 0;         // padded row length (multiple of 4)
    long long ncp = 0;     // pitch*ny*nz: padded component stride
    float *eps = nullptr, *mu = nullptr, *sig = nullptr;
    bool mu_array = false, lossy = false;
    double eps_mu_min = 1.0;
    unsigned flags = 0;
    // graded grids: per-axis cell sizes on the device, eq. (cfl) with local sizes, ||A||_1
    bool graded = false;
    Buf spc;
    double cfl_graded = 0.0, rowsum = 0.0;
    // coefficient cache
    bool c_valid = false, c_has_energy = false;
    double c_dt = 0.0;
    int c_scheme = -1;
    Buf coef, ch, meps, mmu;   // coef: cb (3 components) then ca (3, lossy only)
    // workspaces
    Buf state, pm, amp, srcdev, memdev, acc, kahan, stage, energy, scratch, probe_ws, err;
    Buf ckpt, ring, lam, gacc, gblk, aprobe, aamp, adjmem, scalar, grad_ws;   // adjoint workspaces
    Buf xblocks, xtab, xbasis, xpm;   // exponential propagators: state blocks, tables, probe basis, probe rows
    int deferred = 0;
    Tile tile = {32, 8, 32, 2};
    bool tile_fixed = false;
    fit_run_stats stats = {0, 0, 0, 0.0, 0.0, 0, 0, 0.0, 0.0};
    std::vector<cudaEvent_t> ev;   // pool for per-launch timing (opts->profile)
};

namespace {

int map_err(cudaError_t e) {
    if (e == cudaSuccess) return FIT_OK;
    if (e == cudaErrorMemoryAllocation) return FIT_ERR_OOM;
    return FIT_ERR_CUDA;
}

#define FIT_CHECK(call)                                          \
    do {                                                         \
        cudaError_t _e = (call);                                 \
        if (_e != cudaSuccess) {                                 \
            return map_err(_e);                                  \
        }                                                        \
    } while (0)

int ensure(Buf &b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.n >= bytes) return FIT_OK;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.n = 0;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return FIT_ERR_OOM;
    }
    b.n = bytes;
    return FIT_OK;
}

void release(Buf &b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.n = 0;
}

bool is_device(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

cudaMemcpyKind kind_to_dev(const void *src) {
    return is_device(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
}
cudaMemcpyKind kind_from_dev(const void *dst) {
    return is_device(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
}

double cfl_of(const fit_grid *g) {
    if (g->graded) return g->cfl_graded;
    const double inv = 1.0 / (g->d[0] * g->d[0]) + 1.0 / (g->d[1] * g->d[1]) + 1.0 / (g->d[2] * g->d[2]);
    return std::sqrt(kEps0 * kMu0 * (double)g->eps_mu_min / inv);
}


bool edge_in_box(const fit_grid *g, int axis, int i, int j, int k) {
    if (axis < 0 || axis > 2) return false;
    if (i < 0 || j < 0 || k < 0 || i >= g->nx || j >= g->ny || k >= g->nz) return false;
    return true;
}

bool edge_is_dof(const fit_grid *g, int axis, int i, int j, int k) {
    if (!edge_in_box(g, axis, i, j, k)) return false;
    const int q[3] = {i, j, k};
    const int b = (axis + 1) % 3, c = (axis + 2) % 3;
    return q[b] > 0 && q[c] > 0;
}

// ensure the coefficients for (dt, scheme) exist on the device
template <typename T>
int ensure_coeffs(fit_grid *g, double dt, int scheme, bool need_energy, cudaStream_t s) {
    if (g->c_valid && g->c_dt == dt && g->c_scheme == scheme && (!need_energy || g->c_has_energy)) return FIT_OK;
    const size_t n3 = 3 * (size_t)g->ncp * sizeof(T);
    const size_t nch = g->mu_array ? n3 : 3 * sizeof(T);
    int rc;
    if ((rc = ensure(g->coef, g->lossy ? 2 * n3 : n3))) return rc;
    if ((rc = ensure(g->ch, nch))) return rc;
    const bool energy = need_energy || g->c_has_energy;
    if (energy) {
        if ((rc = ensure(g->meps, n3))) return rc;
        if ((rc = ensure(g->mmu, nch))) return rc;
    }
    T *cb = (T *)g->coef.p;
    T *ca = g->lossy ? cb + 3 * g->ncp : nullptr;
    if (g->graded)
        FIT_CHECK(build_coeffs_graded<T>(g->nx, g->ny, g->nz, g->pitch, (const double *)g->spc.p, g->eps, g->mu, g->sig,
                                         dt, scheme, ca, cb, (T *)g->ch.p, energy ? (T *)g->meps.p : nullptr,
                                         energy ? (T *)g->mmu.p : nullptr, s, (g->flags & FIT_FLAG_COEF_FLOAT) != 0));
    else
    FIT_CHECK(build_coeffs<T>(g->nx, g->ny, g->nz, g->pitch, g->d, g->eps, g->mu, g->sig, dt, scheme, g->mu_array,
                              ca, cb, (T *)g->ch.p, energy ? (T *)g->meps.p : nullptr,
                              energy ? (T *)g->mmu.p : nullptr, s, (g->flags & FIT_FLAG_COEF_FLOAT) != 0));
    g->stats.kernel_launches += 1;
    g->c_valid = true;
    g->c_dt = dt;
    g->c_scheme = scheme;
    g->c_has_energy = energy;
    return FIT_OK;
}

struct MemberSpec {
    long long start, nit, src_lo, src_hi;
    const void *e0, *h0;   // initial state (grid precision) or null
};

Tile pick_tile(const fit_grid *g, const fit_run_opts *o) {
    Tile t = g->tile;
    // FP32 default: 64 x 4 tiles, a 3-plane ring (4 CTAs per SM), 64-plane chunks
    if (g->prec == 32 && !g->tile_fixed) t = Tile{64, 4, 64, 2, 3};
    if (o && o->kernel > 0) t.kernel = o->kernel;
    if (o && o->tile_x > 0 && o->tile_y > 0) {
        t.tx = o->tile_x;
        t.ty = o->tile_y;
        t.stages = 0;   // that tile's default ring depth unless stages is given
    }
    if (g->prec == 48) {
        if (!comp_tile_supported(t.tx, t.ty)) t.tx = 32, t.ty = 8;
        t.kernel = 2;
    } else if (t.kernel == 2 && !tma_tile_supported(t.tx, t.ty, g->prec == 64 ? 8 : 4)) {
        t.kernel = 1;
    }
    if (t.kernel == 1 && !tile_supported(t.tx, t.ty)) {
        t.tx = 32;
        t.ty = 8;
    }
    if (o && o->tile_z > 0) t.kz = o->tile_z;
    if (o && (o->stages == 3 || o->stages == 4)) t.stages = o->stages;
    if (t.kz <= 0) t.kz = 32;
    // small grids: more z chunks so the GPU fills up
    const long long cols = (long long)((g->nx + t.tx - 1) / t.tx) * ((g->ny + t.ty - 1) / t.ty);
    while (t.kz > 8 && cols * ((g->nz + t.kz - 1) / t.kz) < 4 * 152) t.kz /= 2;
    return t;
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
                const fit_run_opts *opts, cudaStream_t s, T *const *keep_final = nullptr) {
    const long long ncell = g->ncell;   // real cells (algorithmic counts)
    const long long ncp = g->ncp;       // padded component stride (device arrays)
    const bool comp = g->prec == 48;    // hi/lo float pairs: 12-component state blocks
    const size_t n6 = (comp ? 12 : 6) * (size_t)ncp;
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
    const double fld_bytes = (comp ? 24.0 : 12.0) * sizeof(T) * (double)ncell;
    const double coef_bytes = ((g->lossy ? 6.0 : 3.0) + (g->mu_array ? 3.0 : 0.0) +
                               (energy_dev ? (3.0 + (g->mu_array ? 3.0 : 0.0)) : 0.0)) * sizeof(T) * (double)ncell;

    // order members by decreasing length (stable: equal lengths keep caller order)
    std::vector<int> order(specs_in.size());
    for (size_t m = 0; m < order.size(); ++m) order[m] = (int)m;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return specs_in[a].nit > specs_in[b].nit; });
    const int nm_total = (int)order.size();
    const int mpp = (opts && opts->members_per_pass > 0) ? std::min(opts->members_per_pass, nm_total) : nm_total;

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
    const bool kahan = sum_mode == 1 && acc_e && !comp;
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
    if (comp) {
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
            if (!comp) {
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
    if (opts && opts->steps_per_launch == 2 && sizeof(T) == 4 && !comp && !energy_dev && tile.kernel == 2) {
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

    // Groups run from the end of the table (shortest members) to its start, and
    // inside a group members finish shortest first, so the superposition adds
    // members in decreasing table order whatever members_per_pass is.
    for (int g_end = nm_total; g_end > 0; g_end -= mpp) {
        const int first = std::max(0, g_end - mpp);
        const int cnt = g_end - first;
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
            if (comp) {   // FP64 compact input -> hi/lo pairs (masked to the degrees of freedom)
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
            if (!comp && (sp.e0 || sp.h0)) {
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
            if (comp)
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
            if (acc_e && comp) {
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

int check_sources_probes(const fit_grid *g, const fit_source *src, int nsrc, const fit_probe *prb, int nprb) {
    if (nsrc < 0 || nprb < 0) return FIT_ERR_ARG;
    if (nsrc > 0 && !src) return FIT_ERR_ARG;
    if (nprb > 0 && !prb) return FIT_ERR_ARG;
    for (int s = 0; s < nsrc; ++s) {
        if (!edge_is_dof(g, src[s].axis, src[s].i, src[s].j, src[s].k)) return FIT_ERR_ARG;
        if (src[s].waveform < 0 || src[s].waveform > 2) return FIT_ERR_ARG;
        if ((src[s].waveform != FIT_WAVE_SINE) && !(src[s].width > 0.0)) return FIT_ERR_ARG;
    }
    for (int p = 0; p < nprb; ++p)
        if (!edge_in_box(g, prb[p].axis, prb[p].i, prb[p].j, prb[p].k)) return FIT_ERR_ARG;
    if (nsrc > kMaxSrc || nprb > kMaxPrb) return FIT_ERR_UNSUPPORTED;
    return FIT_OK;
}

int check_dt(const fit_grid *g, double dt, const fit_run_opts *o) {
    if (!(dt > 0.0) || !std::isfinite(dt)) return FIT_ERR_ARG;
    if (!(o && o->force_dt) && dt > cfl_of(g) * (1.0 + 1e-12)) return FIT_ERR_CFL;
    return FIT_OK;
}

int finish(fit_grid *g, cudaStream_t s, bool host_outputs) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return map_err(e);
    if (host_outputs) {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return map_err(e);
        int herr = 0;
        if (g->err.p) {
            cudaMemcpy(&herr, g->err.p, sizeof(int), cudaMemcpyDeviceToHost);
            if (herr) {
                cudaMemset(g->err.p, 0, sizeof(int));
                return (herr & kErrTimeout) ? FIT_ERR_TIMEOUT : FIT_ERR_ARG;
            }
        }
    }
    return FIT_OK;
}

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
    if (C <= 0) C = std::max(1, (int)std::ceil(std::sqrt((double)N)));
    if (C > N) C = (int)N;
    const long long nseg = (N + C - 1) / C;
    const long long ncp = g->ncp;
    const size_t n6 = 6 * (size_t)ncp;
    if ((rc = ensure(g->ckpt, (size_t)nseg * n6 * sizeof(T)))) return rc;
    if ((rc = ensure(g->ring, (size_t)(C + 1) * n6 * sizeof(T)))) return rc;
    if ((rc = ensure(g->lam, 2 * n6 * sizeof(T)))) return rc;
    if ((rc = ensure(g->gacc, 3 * (size_t)ncp * sizeof(double)))) return rc;
    // FP32 fields: the gradient of each block of kGradBlock adjoint steps is summed in FP32 and
    // then added into the FP64 total (block boundaries fixed in the adjoint step index, so the
    // result does not depend on the checkpoint interval)
    constexpr int kGradBlock = 64;
    const bool fp32_blocks = sizeof(T) == 4;
    if (fp32_blocks && (rc = ensure(g->gblk, 3 * (size_t)ncp * sizeof(float)))) return rc;
    if ((rc = ensure(g->aprobe, (size_t)N * nprb * sizeof(double)))) return rc;
    if ((rc = ensure(g->aamp, (size_t)N * nprb * sizeof(double)))) return rc;
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
    FIT_CHECK(cudaMemsetAsync(lam, 0, 2 * n6 * sizeof(T), s));
    FIT_CHECK(cudaMemsetAsync(gacc, 0, 3 * (size_t)ncp * sizeof(double), s));
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
          encode_tma_maps(&lam_maps, (int)sizeof(T), g->nx, g->ny, g->nz, g->pitch, lam, 2, g->coef.p,
                          g->lossy ? 6 : 3, tile.tx, tile.ty))) {
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
    auto step = [&](const TmaMaps &maps) -> cudaError_t {
        g->stats.step_launches += 1;
        g->stats.kernel_launches += 1;
        g->stats.cell_updates += g->ncell;
        if (tile.kernel == 2) return launch_step_tma<T>(a, maps, tile, g->lossy, g->mu_array, false, s);
        return launch_step<T>(a, tile, g->lossy, g->mu_array, false, s);
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
        if (n % C == 0)
            FIT_CHECK(cudaMemcpyAsync(ckpt + (size_t)(n / C) * n6, ring + (size_t)(n & 1) * n6, n6 * sizeof(T),
                                      cudaMemcpyDeviceToDevice, s));
        a.it = (int)n;
        a.parity = (int)(n & 1);
        FIT_CHECK(step(ring_maps));
    }
    a.nprb = 0;
    double *Jdev = (double *)g->scalar.p;
    FIT_CHECK(probe_functional(prb, nprb, g->d, aprobe, N, Jdev, s));
    // adjoint state at N and the adjoint sources
    FIT_CHECK(adjoint_init<T>(prb, nprb, g->d, aprobe + (size_t)(N - 1) * nprb, (const T *)g->coef.p, lam, g->pitch,
                              g->ny, ncp, s));
    FIT_CHECK(adjoint_sources(prb, nprb, g->d, aprobe, N, aamp, s));
    g->stats.kernel_launches += 3;
    const double K[3] = {-kEps0 * (g->d[1] * g->d[2] / g->d[0]) / dt, -kEps0 * (g->d[2] * g->d[0] / g->d[1]) / dt,
                         -kEps0 * (g->d[0] * g->d[1] / g->d[2]) / dt};

    for (long long sg = nseg - 1; sg >= 0; --sg) {
        const long long A = sg * C, B = std::min<long long>(A + C, N);
        FIT_CHECK(cudaMemcpyAsync(ring, ckpt + (size_t)sg * n6, n6 * sizeof(T), cudaMemcpyDeviceToDevice, s));
        set_forward_sources();
        for (long long q = 0; q < B - A; ++q) {   // ring slot q -> q+1: step A+q
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
            FIT_CHECK(step(lam_maps));
            const T *mu_in = lam + (size_t)(t & 1) * n6;
            if (fp32_blocks) {
                FIT_CHECK(grad_accumulate_block(ncp, (const float *)mu_in, (const float *)(ring + (size_t)(n + 1 - A) * n6),
                                                (const float *)(ring + (size_t)(n - A) * n6), K, (float *)g->gblk.p, s));
                g->stats.kernel_launches += 1;
                if ((t + 1) % kGradBlock == 0 || t == N - 1) {
                    FIT_CHECK(grad_flush(ncp, (float *)g->gblk.p, gacc, s));
                    g->stats.kernel_launches += 1;
                }
            } else {
                FIT_CHECK(grad_accumulate<T>(ncp, mu_in, ring + (size_t)(n + 1 - A) * n6, ring + (size_t)(n - A) * n6,
                                             K, gacc, s));
                g->stats.kernel_launches += 1;
            }
        }
    }
    // per-cell gradient and J
    double *gout = grad_out;
    const bool grad_host = grad_out && !is_device(grad_out);
    if (grad_host || !grad_out) {
        if ((rc = ensure(g->grad_ws, sizeof(double) * (size_t)g->ncell))) return rc;
        gout = (double *)g->grad_ws.p;
    }
    FIT_CHECK(grad_scatter(g->nx, g->ny, g->nz, g->pitch, ncp, gacc, gout, s));
    g->stats.kernel_launches += 1;
    if (grad_host)
        FIT_CHECK(cudaMemcpyAsync(grad_out, gout, sizeof(double) * (size_t)g->ncell, cudaMemcpyDeviceToHost, s));
    if (J_out) FIT_CHECK(cudaMemcpyAsync(J_out, Jdev, sizeof(double), kind_from_dev(J_out), s));
    const bool host_out = grad_host || (J_out && !is_device(J_out));
    return finish(g, s, host_out);
}

// ---------------------------------------------------------------------------
// Batched ParaExp over many grids (FP32): every member of every grid is a work
// item of one persistent launch per iteration; see batched_tma_kernel.
// ---------------------------------------------------------------------------

std::mutex g_tune_mu;
std::map<std::string, Tile> g_tune_cache;   // batch signature -> tile, kz

struct BatchHost {
    const fit_paraexp_problem *p = nullptr;
    std::vector<MemberSpec> specs;
    std::vector<int> order;       // member table slot -> spec index (longest first)
    long long W0 = 0, nt = 0;
    double *pdev = nullptr;       // summed probe rows (device)
    double *ae = nullptr, *ah = nullptr;
    bool probes = false;
};

struct DevBuf {   // a temporary device allocation of one batched call
    void *p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};

// Fill grid descriptors, tensor maps and the work list for a tile shape.
int batch_layout(std::vector<BatchHost> &H, Tile tile, bool lossy, std::vector<GridDesc<float>> &gds,
                 std::vector<TmaMaps> &maps, std::vector<WorkItem> &items) {
    const int ng = (int)H.size();
    gds.assign(ng, GridDesc<float>());
    maps.assign(ng, TmaMaps());
    items.clear();
    for (int gi = 0; gi < ng; ++gi) {
        fit_grid *g = H[gi].p->grid;
        GridDesc<float> &d = gds[gi];
        memset(&d, 0, sizeof(d));
        d.nx = g->nx; d.ny = g->ny; d.nz = g->nz; d.pitch = g->pitch; d.ncell = g->ncp;
        d.tiles_x = (g->nx + tile.tx - 1) / tile.tx;
        d.tiles_y = (g->ny + tile.ty - 1) / tile.ty;
        d.kz = std::max(1, std::min(tile.kz, g->nz));
        d.nchunk = (g->nz + d.kz - 1) / d.kz;
        d.ch = (const float *)g->ch.p;
        d.muarr = g->mu_array ? 1 : 0;
        d.mem = (const Member *)g->memdev.p;
        d.amp = (const double *)g->amp.p;
        d.amp_base = H[gi].W0;
        d.nsrc = H[gi].p->nsrc;
        d.nprb = H[gi].probes ? H[gi].p->nprb : 0;
        for (int q = 0; q < d.nsrc; ++q) {
            const fit_source &r = H[gi].p->src[q];
            d.src[q] = {r.axis, r.i, r.j, r.k};
        }
        for (int q = 0; q < d.nprb; ++q) {
            const fit_probe &r = H[gi].p->prb[q];
            d.prb[q] = {r.axis, r.i, r.j, r.k};
        }
        const int K = (int)H[gi].specs.size();
        if (!encode_tma_maps(&maps[gi], 4, g->nx, g->ny, g->nz, g->pitch, g->state.p, 2 * K, g->coef.p,
                             lossy ? 6 : 3, tile.tx, tile.ty))
            return FIT_ERR_UNSUPPORTED;
        for (int t = 0; t < d.tiles_x * d.tiles_y; ++t)
            for (int c = 0; c < d.nchunk; ++c)
                for (int q = 0; q < K; ++q) items.push_back({gi, q, t, c});
    }
    return FIT_OK;
}

int batched_group(const std::vector<const fit_paraexp_problem *> &probs, bool lossy, const fit_run_opts *opts,
                  cudaStream_t s) {
    const int ng = (int)probs.size();
    const int scheme = opts ? opts->sigma_scheme : 0;
    int rc;
    std::vector<BatchHost> H(ng);
    long long nit_max = 0;
    for (int gi = 0; gi < ng; ++gi) {
        const fit_paraexp_problem &q = *probs[gi];
        fit_grid *g = q.grid;
        BatchHost &h = H[gi];
        h.p = &q;
        g->stats = fit_run_stats{0, 0, 0, 0.0, 0.0, 0, 0, 0.0, 0.0};
        if ((rc = ensure_coeffs<float>(g, q.dt, scheme, false, s))) return rc;
        h.W0 = q.win[0];
        h.nt = q.win[q.K] - q.win[0];
        for (int j = 1; j <= q.K; ++j)
            h.specs.push_back({q.win[j - 1], q.win[q.K] - q.win[j - 1], q.win[j - 1], q.win[j], nullptr, nullptr});
        h.order.resize(q.K);
        for (int m = 0; m < q.K; ++m) h.order[m] = m;
        std::stable_sort(h.order.begin(), h.order.end(),
                         [&](int a, int b) { return h.specs[a].nit > h.specs[b].nit; });
        nit_max = std::max(nit_max, h.specs[h.order[0]].nit);
        const size_t n6 = 6 * (size_t)g->ncp;
        if ((rc = ensure(g->state, 2 * n6 * sizeof(float) * (size_t)q.K))) return rc;
        FIT_CHECK(cudaMemsetAsync(g->state.p, 0, 2 * n6 * sizeof(float) * (size_t)q.K, s));
        h.probes = q.probe_out && q.nprb > 0 && h.nt > 0;
        if (h.probes) {
            const size_t pm = sizeof(double) * (size_t)h.nt * q.nprb * q.K;
            if ((rc = ensure(g->pm, pm))) return rc;
            FIT_CHECK(cudaMemsetAsync(g->pm.p, 0, pm, s));
            if (is_device(q.probe_out)) h.pdev = q.probe_out;
            else {
                if ((rc = ensure(g->probe_ws, sizeof(double) * (size_t)h.nt * q.nprb))) return rc;
                h.pdev = (double *)g->probe_ws.p;
            }
        }
        if (q.nsrc > 0) {
            if ((rc = ensure(g->amp, sizeof(double) * (size_t)h.nt * q.nsrc))) return rc;
            if ((rc = ensure(g->srcdev, sizeof(fit_source) * q.nsrc))) return rc;
            FIT_CHECK(cudaMemcpyAsync(g->srcdev.p, q.src, sizeof(fit_source) * q.nsrc, cudaMemcpyHostToDevice, s));
            FIT_CHECK(source_table((const fit_source *)g->srcdev.p, q.nsrc, h.W0, h.nt, q.dt, (double *)g->amp.p, s));
        }
        if (q.e_final || q.h_final) {
            if ((rc = ensure(g->acc, 2 * 3 * (size_t)g->ncp * sizeof(double)))) return rc;
            h.ae = (double *)g->acc.p;
            h.ah = h.ae + 3 * (size_t)g->ncp;
            FIT_CHECK(cudaMemsetAsync(g->acc.p, 0, 2 * 3 * (size_t)g->ncp * sizeof(double), s));
        }
        if ((rc = ensure(g->err, sizeof(int)))) return rc;
        FIT_CHECK(cudaMemsetAsync(g->err.p, 0, sizeof(int), s));
        if ((rc = ensure(g->memdev, sizeof(Member) * (size_t)q.K))) return rc;
        std::vector<Member> mem(q.K);
        for (int m = 0; m < q.K; ++m) {
            const MemberSpec &sp = h.specs[h.order[m]];
            memset(&mem[m], 0, sizeof(Member));
            float *base = (float *)g->state.p + 2 * n6 * (size_t)m;
            mem[m].st[0] = base;
            mem[m].st[1] = base + n6;
            mem[m].blk[0] = 2 * m;
            mem[m].blk[1] = 2 * m + 1;
            mem[m].start = sp.start;
            mem[m].end = sp.start + sp.nit;
            mem[m].src_lo = sp.src_lo;
            mem[m].src_hi = sp.src_hi;
            mem[m].probe = h.probes ? (double *)g->pm.p + (size_t)h.order[m] * h.nt * q.nprb : nullptr;
            mem[m].probe_base = h.W0;
        }
        FIT_CHECK(cudaMemcpyAsync(g->memdev.p, mem.data(), sizeof(Member) * q.K, cudaMemcpyHostToDevice, s));
        FIT_CHECK(cudaStreamSynchronize(s));   // the host table is released at scope end
    }

    // tile shape: caller's, tuned, or the default
    Tile tile = {32, 8, 32, 2};
    if (opts && opts->tile_x > 0 && opts->tile_y > 0 && batched_tile_supported(opts->tile_x, opts->tile_y)) {
        tile.tx = opts->tile_x;
        tile.ty = opts->tile_y;
    }
    if (opts && opts->tile_z > 0) tile.kz = opts->tile_z;
    if (opts && (opts->stages == 3 || opts->stages == 4)) tile.stages = opts->stages;
    int nsm = 152;
    {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            nsm = 152;
        }
    }
    std::vector<GridDesc<float>> gds;
    std::vector<TmaMaps> maps;
    std::vector<WorkItem> items;
    DevBuf d_grids, d_maps, d_items, d_counter;
    const size_t gd_bytes = sizeof(GridDesc<float>) * ng, map_bytes = sizeof(CUtensorMap) * 2 * ng;
    if (cudaMalloc(&d_grids.p, gd_bytes) != cudaSuccess || cudaMalloc(&d_maps.p, map_bytes) != cudaSuccess ||
        cudaMalloc(&d_counter.p, sizeof(int) * (size_t)std::max<long long>(nit_max, 8)) != cudaSuccess) {
        cudaGetLastError();
        return FIT_ERR_OOM;
    }
    size_t items_cap = 0;
    int *err = (int *)probs[0]->grid->err.p;
    auto upload = [&](const Tile &t) -> int {
        int r = batch_layout(H, t, lossy, gds, maps, items);
        if (r) return r;
        if (items.size() > items_cap) {
            if (d_items.p) cudaFree(d_items.p);
            d_items.p = nullptr;
            if (cudaMalloc(&d_items.p, sizeof(WorkItem) * items.size()) != cudaSuccess) {
                cudaGetLastError();
                return FIT_ERR_OOM;
            }
            items_cap = items.size();
        }
        std::vector<CUtensorMap> flat(2 * ng);
        for (int gi = 0; gi < ng; ++gi) {
            flat[2 * gi] = maps[gi].state;
            flat[2 * gi + 1] = maps[gi].coef;
        }
        if (cudaMemcpy(d_grids.p, gds.data(), gd_bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(d_maps.p, flat.data(), map_bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(d_items.p, items.data(), sizeof(WorkItem) * items.size(), cudaMemcpyHostToDevice) !=
                cudaSuccess)
            return FIT_ERR_CUDA;
        return FIT_OK;
    };
    auto make_args = [&](long long it) {
        BatchArgs<float> b;
        b.grids = (const GridDesc<float> *)d_grids.p;
        b.maps = (const CUtensorMap *)d_maps.p;
        b.items = (const WorkItem *)d_items.p;
        b.nitems = (int)items.size();
        b.it = (int)it;
        b.parity = (int)(it & 1);
        b.counter = (int *)d_counter.p + it;
        b.err = err;
        return b;
    };

    // autotune: time a few iterations of each candidate, once per batch signature
    if (opts && opts->autotune && !(opts->tile_x > 0)) {
        std::string sig = lossy ? "L" : "N";
        for (int gi = 0; gi < ng; ++gi) {
            const fit_grid *g = H[gi].p->grid;
            sig += ":" + std::to_string(g->nx) + "x" + std::to_string(g->ny) + "x" + std::to_string(g->nz) + "k" +
                   std::to_string(H[gi].p->K);
        }
        bool hit = false;
        {
            std::lock_guard<std::mutex> lock(g_tune_mu);
            auto f = g_tune_cache.find(sig);
            if (f != g_tune_cache.end()) {
                tile = f->second;
                hit = true;
            }
        }
        if (!hit) {
            const Tile cands[] = {{32, 8, 32, 2, 4}, {32, 8, 16, 2, 4}, {32, 8, 8, 2, 4},  {32, 8, 32, 2, 3},
                                  {32, 8, 16, 2, 3}, {64, 4, 32, 2, 4}, {64, 4, 16, 2, 4}, {64, 4, 32, 2, 3},
                                  {32, 4, 32, 2, 4}, {32, 4, 16, 2, 4}, {32, 16, 32, 2, 3}};
            const int trials = (int)std::min<long long>(3, nit_max);
            float best = 1e30f;
            Tile best_t = tile;
            cudaEvent_t e0, e1;
            FIT_CHECK(cudaEventCreate(&e0));
            FIT_CHECK(cudaEventCreate(&e1));
            for (const Tile &c : cands) {
                if ((rc = upload(c))) continue;
                const int ctas = batched_ctas_per_sm_f32(c, lossy) * nsm;
                FIT_CHECK(cudaMemsetAsync(d_counter.p, 0, sizeof(int) * (size_t)std::max<long long>(nit_max, 8), s));
                FIT_CHECK(cudaEventRecord(e0, s));
                for (int it = 0; it < trials; ++it) FIT_CHECK(launch_batched_f32(make_args(it), c, lossy, ctas, s));
                FIT_CHECK(cudaEventRecord(e1, s));
                FIT_CHECK(cudaEventSynchronize(e1));
                float ms = 0.f;
                FIT_CHECK(cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best) {
                    best = ms;
                    best_t = c;
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            tile = best_t;
            std::lock_guard<std::mutex> lock(g_tune_mu);
            g_tune_cache[sig] = tile;
            // the trial steps wrote into the states and probe rows: start over from zero
            for (int gi = 0; gi < ng; ++gi) {
                fit_grid *g = H[gi].p->grid;
                const size_t n6 = 6 * (size_t)g->ncp;
                FIT_CHECK(cudaMemsetAsync(g->state.p, 0, 2 * n6 * sizeof(float) * H[gi].specs.size(), s));
                if (H[gi].probes)
                    FIT_CHECK(cudaMemsetAsync(g->pm.p, 0,
                                              sizeof(double) * (size_t)H[gi].nt * H[gi].p->nprb * H[gi].specs.size(),
                                              s));
            }
        }
    }
    if ((rc = upload(tile))) return rc;
    const int ctas = batched_ctas_per_sm_f32(tile, lossy) * nsm;
    FIT_CHECK(cudaMemsetAsync(d_counter.p, 0, sizeof(int) * (size_t)std::max<long long>(nit_max, 8), s));

    // the iteration loop, optionally captured as one CUDA graph
    const bool graph = opts && opts->use_graph;
    cudaStream_t cs = s;
    cudaGraph_t gr = nullptr;
    cudaGraphExec_t ge = nullptr;
    if (graph) {
        FIT_CHECK(cudaStreamSynchronize(s));
        FIT_CHECK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        FIT_CHECK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    }
    auto loop = [&]() -> cudaError_t {
        cudaError_t e;
        for (long long it = 0; it < nit_max; ++it) {
            if ((e = launch_batched_f32(make_args(it), tile, lossy, ctas, cs)) != cudaSuccess) return e;
            for (int gi = 0; gi < ng; ++gi) {
                BatchHost &h = H[gi];
                fit_grid *g = h.p->grid;
                g->stats.step_launches += 1;
                for (int m = (int)h.specs.size() - 1; m >= 0; --m) {   // shortest first
                    const MemberSpec &sp = h.specs[h.order[m]];
                    if (sp.start + it < sp.start + sp.nit) g->stats.cell_updates += g->ncell;
                    if (sp.nit != it + 1 || !h.ae) continue;
                    const size_t n6 = 6 * (size_t)g->ncp;
                    const float *fin = (const float *)g->state.p + 2 * n6 * (size_t)m + ((it + 1) & 1) * n6;
                    if ((e = accumulate_state<float>(3 * g->ncp, fin, h.ae, cs)) != cudaSuccess) return e;
                    if ((e = accumulate_state<float>(3 * g->ncp, fin + 3 * g->ncp, h.ah, cs)) != cudaSuccess)
                        return e;
                }
            }
        }
        return cudaSuccess;
    };
    cudaError_t le = loop();
    if (graph) {
        cudaError_t ee = cudaStreamEndCapture(cs, &gr);
        if (le == cudaSuccess) le = ee;
        if (le == cudaSuccess) le = cudaGraphInstantiate(&ge, gr, 0);
        if (le == cudaSuccess) le = cudaGraphLaunch(ge, s);
        if (le == cudaSuccess) le = cudaStreamSynchronize(s);
        if (ge) cudaGraphExecDestroy(ge);
        if (gr) cudaGraphDestroy(gr);
        cudaStreamDestroy(cs);
    }
    FIT_CHECK(le);
    // probe sums and final fields of each grid
    for (int gi = 0; gi < ng; ++gi) {
        BatchHost &h = H[gi];
        fit_grid *g = h.p->grid;
        const fit_paraexp_problem &q = *h.p;
        if (h.probes) {
            FIT_CHECK(sum_members((int)h.specs.size(), h.nt * q.nprb, (const double *)g->pm.p, h.nt * q.nprb, h.pdev, s));
            if (h.pdev != q.probe_out)
                FIT_CHECK(cudaMemcpyAsync(q.probe_out, h.pdev, sizeof(double) * (size_t)h.nt * q.nprb,
                                          cudaMemcpyDeviceToHost, s));
        }
        const size_t row = (size_t)g->nx * sizeof(double), prow = (size_t)g->pitch * sizeof(double);
        const size_t rows3 = 3 * (size_t)g->ny * g->nz;
        if (q.e_final)
            FIT_CHECK(cudaMemcpy2DAsync(q.e_final, row, h.ae, prow, row, rows3, kind_from_dev(q.e_final), s));
        if (q.h_final)
            FIT_CHECK(cudaMemcpy2DAsync(q.h_final, row, h.ah, prow, row, rows3, kind_from_dev(q.h_final), s));
        g->stats.kernel_launches = g->stats.step_launches;   // shared launches, counted per grid
    }
    // temporary tables are freed when this call returns: wait for the work
    FIT_CHECK(cudaStreamSynchronize(s));
    int rc2 = FIT_OK;
    for (int gi = 0; gi < ng && !rc2; ++gi) rc2 = finish(H[gi].p->grid, s, true);
    return rc2;
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
    if (!(dx > 0) || !(dy > 0) || !(dz > 0) || !std::isfinite(dx) || !std::isfinite(dy) || !std::isfinite(dz))
        return FIT_ERR_ARG;
    if (precision != 32 && precision != 64 && precision != 48) return FIT_ERR_ARG;
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
    if (cudaMalloc(&g->eps, bytes) != cudaSuccess) { cudaGetLastError(); return fail(FIT_ERR_OOM); }
    if (cudaMemcpy(g->eps, eps_r, bytes, kind_to_dev(eps_r)) != cudaSuccess) return fail(FIT_ERR_CUDA);
    if (mu_r) {
        if (cudaMalloc(&g->mu, bytes) != cudaSuccess) { cudaGetLastError(); return fail(FIT_ERR_OOM); }
        if (cudaMemcpy(g->mu, mu_r, bytes, kind_to_dev(mu_r)) != cudaSuccess) return fail(FIT_ERR_CUDA);
    }
    if (sigma) {
        if (cudaMalloc(&g->sig, bytes) != cudaSuccess) { cudaGetLastError(); return fail(FIT_ERR_OOM); }
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
    g->mu_array = true;   // ch varies per face
    if (graded_cfl_and_bound(nx, ny, nz, (const double *)g->spc.p, g->eps, g->mu, g->scratch.p, &g->cfl_graded,
                             &g->rowsum, 0) != cudaSuccess) {
        fit_grid_destroy(g);
        return FIT_ERR_CUDA;
    }
    *out = g;
    return FIT_OK;
}

int fit_spectral_bound(const fit_grid *g, double *beta) {
    if (!g || !beta) return FIT_ERR_ARG;
    *beta = 2.0 / expo_unit(g);
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
                   &g->grad_ws, &g->xblocks, &g->xtab, &g->xbasis, &g->xpm, &g->spc, &g->gblk};
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
    int rc;
    if ((rc = check_dt(g, dt, opts))) return rc;
    if ((rc = check_sources_probes(g, src, nsrc, prb, nprb))) return rc;
    if (opts && (opts->sigma_scheme < 0 || opts->sigma_scheme > 1)) return FIT_ERR_ARG;
    if (nsteps == 0) return FIT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (g->prec == 64)
        return leapfrog_impl<double>(g, dt, nsteps, step0, src, nsrc, prb, nprb, probe_out, energy_out, e_io, h_io,
                                     opts, s);
    if (g->prec == 48 && opts && opts->kernel == 1) return FIT_ERR_UNSUPPORTED;
    return leapfrog_impl<float>(g, dt, nsteps, step0, src, nsrc, prb, nprb, probe_out, energy_out, e_io, h_io, opts,
                                s);
}

int paraexp_run(fit_grid *g, double dt, int K, const long *win, const fit_source *src, int nsrc,
                const fit_probe *prb, int nprb, double *probe_out, double *e_final, double *h_final,
                const void *e0, const void *h0, const fit_run_opts *opts, void *stream) {
    if (!g || K < 1 || !win) return FIT_ERR_ARG;
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
        if (g->prec == 48 || g->lossy) return FIT_ERR_UNSUPPORTED;
        if (g->prec == 64)
            return paraexp_expo_impl<double>(g, dt, K, win, src, nsrc, prb, nprb, probe_out, e_final, h_final, e0,
                                             h0, opts, s);
        return paraexp_expo_impl<float>(g, dt, K, win, src, nsrc, prb, nprb, probe_out, e_final, h_final, e0, h0,
                                        opts, s);
    }
    if (g->prec == 64)
        return paraexp_impl<double>(g, dt, K, win, src, nsrc, prb, nprb, probe_out, e_final, h_final, e0, h0, opts, s);
    if (g->prec == 48 && opts && (opts->kernel == 1 || opts->sum_mode == 1)) return FIT_ERR_UNSUPPORTED;
    return paraexp_impl<float>(g, dt, K, win, src, nsrc, prb, nprb, probe_out, e_final, h_final, e0, h0, opts, s);
}

int paraexp_run_batched(const fit_paraexp_problem *probs, int nprobs, const fit_run_opts *opts, void *stream) {
    if (!probs || nprobs < 0) return FIT_ERR_ARG;
    if (opts && (opts->sigma_scheme < 0 || opts->sigma_scheme > 1)) return FIT_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    // validate everything first; a grid may appear in one problem only
    for (int p = 0; p < nprobs; ++p) {
        const fit_paraexp_problem &q = probs[p];
        if (!q.grid || q.K < 1 || !q.win) return FIT_ERR_ARG;
        for (int j = 1; j <= q.K; ++j)
            if (q.win[j] <= q.win[j - 1]) return FIT_ERR_ARG;
        int rc;
        if ((rc = check_dt(q.grid, q.dt, opts))) return rc;
        if ((rc = check_sources_probes(q.grid, q.src, q.nsrc, q.prb, q.nprb))) return rc;
        for (int r = 0; r < p; ++r)
            if (probs[r].grid == q.grid) return FIT_ERR_ARG;
    }
    // the persistent batched launch advances leapfrog members; exponential homogeneous problems
    // (and the plain per-window comparison modes) run the problems one after another
    const bool fused = !(opts && (opts->members_per_pass > 0 || opts->sum_mode != 0 || opts->kernel == 1 ||
                                  opts->homogeneous != FIT_HOMOG_LEAPFROG || opts->steps_per_launch == 2));
    std::vector<const fit_paraexp_problem *> lossless, lossy;
    for (int p = 0; p < nprobs; ++p) {
        const fit_paraexp_problem &q = probs[p];
        if (!fused || q.grid->prec != 32) {   // one problem after another
            int rc = paraexp_run(q.grid, q.dt, q.K, q.win, q.src, q.nsrc, q.prb, q.nprb, q.probe_out, q.e_final,
                                 q.h_final, nullptr, nullptr, opts, stream);
            if (rc) return rc;
            continue;
        }
        (q.grid->lossy ? lossy : lossless).push_back(&q);
    }
    int rc;
    if (!lossless.empty() && (rc = batched_group(lossless, false, opts, s))) return rc;
    if (!lossy.empty() && (rc = batched_group(lossy, true, opts, s))) return rc;
    return FIT_OK;
}

int fit_adjoint_grad(fit_grid *g, double dt, long nsteps, const fit_source *src, int nsrc, const fit_probe *prb,
                     int nprb, int ckpt_every, double *J_out, double *grad_eps_r, const fit_run_opts *opts,
                     void *stream) {
    if (!g || nsteps < 1 || ckpt_every < 0) return FIT_ERR_ARG;
    int rc;
    if ((rc = check_dt(g, dt, opts))) return rc;
    if ((rc = check_sources_probes(g, src, nsrc, prb, nprb))) return rc;
    if (opts && (opts->sigma_scheme < 0 || opts->sigma_scheme > 1)) return FIT_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (g->graded) return FIT_ERR_UNSUPPORTED;
    if (g->prec == 64)
        return adjoint_impl<double>(g, dt, nsteps, src, nsrc, prb, nprb, ckpt_every, J_out, grad_eps_r, opts, s);
    if (g->prec == 48 || g->graded) return FIT_ERR_UNSUPPORTED;
    return adjoint_impl<float>(g, dt, nsteps, src, nsrc, prb, nprb, ckpt_every, J_out, grad_eps_r, opts, s);
}

int fit_expo_propagate(fit_grid *g, double dt, long nsteps, const fit_probe *prb, int nprb, double *probe_out,
                       void *e_io, void *h_io, const fit_run_opts *opts, void *stream) {
    if (!g || nsteps < 0 || !opts || !(dt > 0.0) || !std::isfinite(dt)) return FIT_ERR_ARG;
    if (opts->homogeneous != FIT_HOMOG_LEJA && opts->homogeneous != FIT_HOMOG_TAYLOR) return FIT_ERR_ARG;
    int rc;
    if ((rc = check_sources_probes(g, nullptr, 0, prb, nprb))) return rc;
    if (g->prec == 48 || g->lossy) return FIT_ERR_UNSUPPORTED;
    if (nsteps == 0) return FIT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (g->prec == 64)
        return expo_propagate_impl<double>(g, dt, nsteps, prb, nprb, probe_out, e_io, h_io, opts, s);
    return expo_propagate_impl<float>(g, dt, nsteps, prb, nprb, probe_out, e_io, h_io, opts, s);
}

int fit_last_stats(const fit_grid *g, fit_run_stats *out) {
    if (!g || !out) return FIT_ERR_ARG;
    *out = g->stats;
    return FIT_OK;
}

int fit_sync(fit_grid *g, void *stream) {
    if (!g) return FIT_ERR_ARG;
    return finish(g, (cudaStream_t)stream, true);
}

}  // extern "C"
