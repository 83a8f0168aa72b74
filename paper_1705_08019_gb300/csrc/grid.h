// grid.h -- the grid object behind the opaque fit_grid of include/fitgb.h and
// the host helpers its translation units share: device workspaces, pointer
// kinds, error mapping, the coefficient cache, tile choice, argument checks
// and the member engine's interface (api.cu), the exponential propagators
// (expo_api.cu), the adjoint (adjoint_api.cu) and the batched launch
// (batched_api.cu).
#pragma once

#include <algorithm>
#include <cmath>
#include <cstring>
#include <initializer_list>
#include <new>
#include <vector>

#include "internal.h"

struct Buf {   // a device allocation owned by a grid
    void *p = nullptr;
    size_t n = 0;
};

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
    std::vector<double> spc_host;   // the same sizes on the host
    double cfl_graded = 0.0, rowsum = 0.0;
    // coefficient cache
    bool c_valid = false, c_has_energy = false;
    double c_dt = 0.0;
    int c_scheme = -1;
    Buf coef, ch, meps, mmu;   // coef: cb (3 components) then ca (3, lossy only)
    // workspaces
    Buf state, pm, amp, srcdev, memdev, acc, kahan, stage, energy, scratch, probe_ws, err;
    Buf ckpt, ring, lam, gacc, gblk, aprobe, aamp, adjmem, scalar, grad_ws, dhist;   // adjoint workspaces
    Buf xblocks, xtab, xbasis, xpm;   // exponential propagators: state blocks, tables, probe basis, probe rows
    int deferred = 0;
    fitgb::Tile tile = {32, 8, 32, 2};
    bool tile_fixed = false;
    fit_run_stats stats = {0, 0, 0, 0.0, 0.0, 0, 0, 0.0, 0.0};
    std::vector<cudaEvent_t> ev;   // pool for per-launch timing (opts->profile)
};

namespace fitgb {

inline int map_err(cudaError_t e) {
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

// Every device allocation of the library goes through dev_alloc.  The test
// hook fit_debug_fail_alloc makes one chosen allocation fail as if the device
// were out of memory, without calling cudaMalloc.
cudaError_t dev_alloc(void **p, size_t bytes);

inline int ensure(Buf &b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.n >= bytes) return FIT_OK;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.n = 0;
    cudaError_t e = dev_alloc(&b.p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return FIT_ERR_OOM;
    }
    b.n = bytes;
    return FIT_OK;
}

inline void release(Buf &b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.n = 0;
}

inline bool is_device(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// true if p is device memory of a GPU other than the current one: the
// library's kernels cannot dereference it, so entry points reject it
inline bool foreign_device(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type != cudaMemoryTypeDevice) return false;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return at.device != dev;
}

inline bool any_foreign(std::initializer_list<const void *> ps) {
    for (const void *p : ps)
        if (foreign_device(p)) return true;
    return false;
}

inline cudaMemcpyKind kind_to_dev(const void *src) {
    return is_device(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
}
inline cudaMemcpyKind kind_from_dev(const void *dst) {
    return is_device(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
}

inline double cfl_of(const fit_grid *g) {
    if (g->graded) return g->cfl_graded;
    const double inv = 1.0 / (g->d[0] * g->d[0]) + 1.0 / (g->d[1] * g->d[1]) + 1.0 / (g->d[2] * g->d[2]);
    return std::sqrt(kEps0 * kMu0 * (double)g->eps_mu_min / inv);
}


inline bool edge_in_box(const fit_grid *g, int axis, int i, int j, int k) {
    if (axis < 0 || axis > 2) return false;
    if (i < 0 || j < 0 || k < 0 || i >= g->nx || j >= g->ny || k >= g->nz) return false;
    return true;
}

inline bool edge_is_dof(const fit_grid *g, int axis, int i, int j, int k) {
    if (!edge_in_box(g, axis, i, j, k)) return false;
    const int q[3] = {i, j, k};
    const int b = (axis + 1) % 3, c = (axis + 2) % 3;
    return q[b] > 0 && q[c] > 0;
}

// ensure the coefficients for (dt, scheme) exist on the device
template <typename T>
inline int ensure_coeffs(fit_grid *g, double dt, int scheme, bool need_energy, cudaStream_t s) {
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

inline Tile pick_tile(const fit_grid *g, const fit_run_opts *o) {
    Tile t = g->tile;
    // FP32 default: 64 x 4 tiles, a 3-plane ring (4 CTAs per SM), 64-plane chunks
    if ((g->prec == 32 || g->prec == 40) && !g->tile_fixed) t = Tile{64, 4, 64, 2, 3};
    if (o && o->kernel > 0) t.kernel = o->kernel;
    if (t.kernel == 3) {   // the TMA pipeline with one cell per thread
        t.kernel = 2;
        t.single = true;
    }
    if (o && o->tile_x > 0 && o->tile_y > 0) {
        t.tx = o->tile_x;
        t.ty = o->tile_y;
        t.stages = 0;   // that tile's default ring depth unless stages is given
    }
    if (g->prec == 48) {
        if (!comp_tile_supported(t.tx, t.ty)) t.tx = 32, t.ty = 8;
        t.kernel = 2;
    } else if (g->prec == 40) {
        if (!res_tile_supported(t.tx, t.ty)) t.tx = 64, t.ty = 4;
        t.kernel = 2;
    } else if (t.kernel == 2 && !tma_tile_supported(t.tx, t.ty, g->prec == 64 ? 8 : 4)) {
        t.kernel = 1;
    }
    if (t.kernel == 1 && !tile_supported(t.tx, t.ty)) {
        t.tx = 32;
        t.ty = 8;
    }
    if (o && (o->stages == 3 || o->stages == 4)) t.stages = o->stages;
    if (o && o->tile_z > 0) {   // the caller's chunk length, as given
        t.kz = o->tile_z;
        t.kz_fixed = true;
    }
    if (t.kz <= 0) t.kz = 32;
    return t;
}

// The z chunk length of a single-grid step launch over nmem members, at most
// t.kz.  One CTA streams one chunk of one tile column, loading its planes plus
// up to two beyond it (the plane below, whose h it recomputes, and the plane
// above).  With `slots` CTAs resident on the GPU at once, a launch of B CTAs
// runs in about ceil(B / slots) rounds, each as long as one CTA's planes; the
// length that minimizes rounds x (kz + 2) is taken, the longest on ties.  On
// GB300 this orders the measured launch times of single-member 128^3 and 256^3
// grids correctly, where a chunk that leaves a last, partly filled round costs
// up to a quarter of the step.  slots <= 0 (occupancy unknown): the chunk is
// halved down to 8 planes while the launch has fewer CTAs than 4 per SM.
inline int chunk_length(int nx, int ny, int nz, const Tile &t, int nmem, long long slots, int nsm) {
    const long long cols = (long long)((nx + t.tx - 1) / t.tx) * ((ny + t.ty - 1) / t.ty);
    int kz = std::max(1, std::min(t.kz, nz));
    if (t.kz_fixed) return t.kz;
    if (slots <= 0) {
        while (kz > 8 && cols * nmem * ((nz + kz - 1) / kz) < 4LL * nsm) kz /= 2;
        return kz;
    }
    long long best = -1;
    int best_kz = kz;
    for (int k = kz; k >= 1; --k) {
        const long long blocks = cols * nmem * ((nz + k - 1) / k);
        const long long cost = ((blocks + slots - 1) / slots) * (k + 2);
        if (best < 0 || cost < best) {
            best = cost;
            best_kz = k;
        }
    }
    return best_kz;
}


inline int check_sources_probes(const fit_grid *g, const fit_source *src, int nsrc, const fit_probe *prb, int nprb) {
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

inline int check_dt(const fit_grid *g, double dt, const fit_run_opts *o) {
    if (!(dt > 0.0) || !std::isfinite(dt)) return FIT_ERR_ARG;
    if (!(o && o->force_dt) && dt > cfl_of(g) * (1.0 + 1e-12)) return FIT_ERR_CFL;
    return FIT_OK;
}

inline int finish(fit_grid *g, cudaStream_t s, bool host_outputs) {
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


// api.cu: the ParaExp member engine (explicitly instantiated for float and double)
template <typename T>
int run_members(fit_grid *g, double dt, int scheme, const std::vector<MemberSpec> &specs_in,
                long long amp_base, long long amp_len, const fit_source *src, int nsrc, const fit_probe *prb,
                int nprb, long long probe_base, long long probe_rows, double *probe_dev, double *energy_dev,
                int sum_mode, double *acc_e, double *acc_h, void *final_e, void *final_h,
                const fit_run_opts *opts, cudaStream_t s, T *const *keep_final = nullptr);

// expo_api.cu: ParaExp with exponential homogeneous problems (float and double)
template <typename T>
int paraexp_expo_impl(fit_grid *g, double dt, int K, const long *win, const fit_source *src, int nsrc,
                      const fit_probe *prb, int nprb, double *probe_out, double *e_final, double *h_final,
                      const void *e0, const void *h0, const fit_run_opts *opts, cudaStream_t s);

}  // namespace fitgb
