// batched_api.cu -- paraexp_run_batched: many ParaExp problems of uneven
// size in one persistent, graph-captured, autotuned launch per iteration
// (kernel batched_tma_kernel in step_tma.cuh).
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>

#include "grid.h"

using namespace fitgb;

namespace {

// ---------------------------------------------------------------------------
// Batched ParaExp over many grids (FP32): every member of every grid is a work
// item of one persistent launch per iteration; see batched_tma_kernel.
// ---------------------------------------------------------------------------

std::mutex g_tune_mu;
std::map<std::string, Tile> g_tune_cache;   // batch signature -> tile, kz

// Optional on-disk copy of the autotuner's choices, shared across processes:
// the file named by the environment variable FITGB_TUNE_CACHE holds one line
// per choice, "<device>|<signature> tx ty kz stages"; a later line for the
// same key wins, and lines that do not parse are ignored.
std::string tune_device_name() {
    int d = 0;
    cudaDeviceProp p;
    if (cudaGetDevice(&d) != cudaSuccess || cudaGetDeviceProperties(&p, d) != cudaSuccess) {
        cudaGetLastError();
        return "unknown";
    }
    std::string n = p.name;
    for (char &c : n)
        if (c == ' ' || c == '|') c = '_';
    return n;
}

bool tune_disk_lookup(const std::string &key, Tile *out) {
    const char *path = std::getenv("FITGB_TUNE_CACHE");
    if (!path || !*path) return false;
    std::ifstream f(path);
    if (!f) return false;
    std::string line;
    bool found = false;
    while (std::getline(f, line)) {
        std::istringstream in(line);
        std::string k;
        Tile t = {0, 0, 0, 2, 0};
        if (!(in >> k >> t.tx >> t.ty >> t.kz >> t.stages) || k != key) continue;
        if (!batched_tile_supported(t.tx, t.ty) || t.kz < 1 || (t.stages != 3 && t.stages != 4)) continue;
        *out = t;
        found = true;
    }
    return found;
}

void tune_disk_store(const std::string &key, const Tile &t) {
    const char *path = std::getenv("FITGB_TUNE_CACHE");
    if (!path || !*path) return;
    char line[512];
    const int n = std::snprintf(line, sizeof(line), "%s %d %d %d %d\n", key.c_str(), t.tx, t.ty, t.kz, t.stages);
    if (n <= 0 || n >= (int)sizeof(line)) return;
    if (FILE *f = std::fopen(path, "a")) {   // one short append per choice
        std::fwrite(line, 1, (size_t)n, f);
        std::fclose(f);
    }
}

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
    // items of a tile column's last, shorter chunk go to the end of the list, longest
    // first, so that the CTAs' last items of a launch are short and the launch ends
    // with little idle time; members of one (grid, tile, chunk) stay adjacent
    std::vector<std::pair<int, WorkItem>> tail;
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
        const int last_len = g->nz - (d.nchunk - 1) * d.kz;   // planes of the last chunk
        for (int t = 0; t < d.tiles_x * d.tiles_y; ++t)
            for (int c = 0; c < d.nchunk; ++c)
                for (int q = 0; q < K; ++q) {
                    if (c == d.nchunk - 1 && last_len < d.kz) tail.push_back({last_len, WorkItem{gi, q, t, c}});
                    else items.push_back({gi, q, t, c});
                }
    }
    std::stable_sort(tail.begin(), tail.end(),
                     [](const std::pair<int, WorkItem> &a, const std::pair<int, WorkItem> &b) { return a.first > b.first; });
    for (const auto &e : tail) items.push_back(e.second);
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
    const bool single = opts && opts->kernel == 3;   // one cell per thread instead of two
    tile.single = single;
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
    if (dev_alloc(&d_grids.p, gd_bytes) != cudaSuccess || dev_alloc(&d_maps.p, map_bytes) != cudaSuccess ||
        dev_alloc(&d_counter.p, sizeof(int) * (size_t)std::max<long long>(nit_max, 8)) != cudaSuccess) {
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
            if (dev_alloc(&d_items.p, sizeof(WorkItem) * items.size()) != cudaSuccess) {
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
        std::string sig = std::string(single ? "fp32s" : "fp32") + (lossy ? "L" : "N");
        for (int gi = 0; gi < ng; ++gi) {
            const fit_grid *g = H[gi].p->grid;
            sig += ":" + std::to_string(g->nx) + "x" + std::to_string(g->ny) + "x" + std::to_string(g->nz) + "k" +
                   std::to_string(H[gi].p->K);
        }
        const std::string key = tune_device_name() + "|" + sig;
        bool hit = false;
        {
            std::lock_guard<std::mutex> lock(g_tune_mu);
            auto f = g_tune_cache.find(key);
            if (f != g_tune_cache.end()) {
                tile = f->second;
                hit = true;
            } else if (tune_disk_lookup(key, &tile)) {
                tile.single = single;
                g_tune_cache[key] = tile;
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
            for (Tile c : cands) {
                c.single = single;
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
            g_tune_cache[key] = tile;
            tune_disk_store(key, tile);
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
                int active = 0;
                for (int m = (int)h.specs.size() - 1; m >= 0; --m) {   // shortest first
                    const MemberSpec &sp = h.specs[h.order[m]];
                    if (sp.start + it < sp.start + sp.nit) {
                        g->stats.cell_updates += g->ncell;
                        ++active;
                    }
                    if (sp.nit != it + 1 || !h.ae) continue;
                    const size_t n6 = 6 * (size_t)g->ncp;
                    const float *fin = (const float *)g->state.p + 2 * n6 * (size_t)m + ((it + 1) & 1) * n6;
                    if ((e = accumulate_state<float>(3 * g->ncp, fin, h.ae, cs)) != cudaSuccess) return e;
                    if ((e = accumulate_state<float>(3 * g->ncp, fin + 3 * g->ncp, h.ah, cs)) != cudaSuccess)
                        return e;
                }
                // algorithmic bytes: each active member's fields in and out, the coefficients once
                if (active > 0)
                    g->stats.alg_bytes += (48.0 * active + (g->lossy ? 24.0 : 12.0) + (g->mu_array ? 12.0 : 0.0)) *
                                          (double)g->ncell;
            }
        }
        return cudaSuccess;
    };
    // opts->profile: the device time of the iteration loop (the batched launches and the
    // superposition of finished members) by CUDA events on the stream, into every grid's stats
    const bool profile = opts && opts->profile;
    cudaEvent_t pe[2] = {nullptr, nullptr};
    if (profile) {
        FIT_CHECK(cudaEventCreate(&pe[0]));
        FIT_CHECK(cudaEventCreate(&pe[1]));
        if (!graph) FIT_CHECK(cudaEventRecord(pe[0], s));
    }
    cudaError_t le = loop();
    if (profile && !graph && le == cudaSuccess) le = cudaEventRecord(pe[1], s);
    if (graph) {
        cudaError_t ee = cudaStreamEndCapture(cs, &gr);
        if (le == cudaSuccess) le = ee;
        if (le == cudaSuccess) le = cudaGraphInstantiate(&ge, gr, 0);
        if (le == cudaSuccess && profile) le = cudaEventRecord(pe[0], s);
        if (le == cudaSuccess) le = cudaGraphLaunch(ge, s);
        if (le == cudaSuccess && profile) le = cudaEventRecord(pe[1], s);
        if (le == cudaSuccess) le = cudaStreamSynchronize(s);
        if (ge) cudaGraphExecDestroy(ge);
        if (gr) cudaGraphDestroy(gr);
        cudaStreamDestroy(cs);
    }
    if (profile) {
        float ms = 0.f;
        if (le == cudaSuccess) le = cudaEventSynchronize(pe[1]);
        if (le == cudaSuccess) le = cudaEventElapsedTime(&ms, pe[0], pe[1]);
        cudaEventDestroy(pe[0]);
        cudaEventDestroy(pe[1]);
        for (int gi = 0; gi < ng; ++gi) H[gi].p->grid->stats.step_ms = ms;
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

int paraexp_run_batched(const fit_paraexp_problem *probs, int nprobs, const fit_run_opts *opts, void *stream) {
    if (!probs || nprobs < 0) return FIT_ERR_ARG;
    if (opts && (opts->sigma_scheme < 0 || opts->sigma_scheme > 1)) return FIT_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    // validate everything first; a grid may appear in one problem only
    for (int p = 0; p < nprobs; ++p) {
        const fit_paraexp_problem &q = probs[p];
        if (!q.grid || q.K < 1 || !q.win) return FIT_ERR_ARG;
        if (any_foreign({q.probe_out, q.e_final, q.h_final})) return FIT_ERR_ARG;
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

}  // extern "C"
