// noalloc.cu -- fit_leapfrog_run_static: an FP32 leapfrog run that allocates
// no device memory.
//
// Some callers cannot call cudaMalloc: code that runs where a device
// allocation could block or fail at the wrong moment (inside a real-time
// loop, a plugin that must not grow the process's memory footprint, or a
// host that hands out a fixed memory budget up front).  They still pass their
// own input and output buffers, but every workspace this run needs -- the
// second state block of the ping-pong, the leapfrog coefficients, the member
// and source tables, the source amplitude table and the error word -- lives
// in one file-scope __device__ array of kStaticScratchBytes (about 30 MiB)
// that every GPU loading this library holds until the process exits.
//
// Its device address is looked up with cudaGetSymbolAddress at the start of
// every call, on the current device (host code cannot use the array's name
// as a device address, and a cached address would be stale after the
// caller's context is torn down and recreated); the first call on a device
// also makes the runtime load this library's device code there, so it should
// come before any stream capture.  All calls share the one array and it keeps the last
// call's contents: this file clears and rebuilds everything a run reads
// before using it, and calls whose work overlaps on the GPU (different
// streams, or different threads) race on it and must be serialized by the
// caller.
#include <cmath>
#include <cstring>

#include "internal.h"

namespace fitgb {
namespace {

constexpr long long kStaticCells = 393216;       // max pitch*ny*nz (e.g. 64 x 64 x 96)
constexpr long long kStaticAmpSteps = 32768;     // source table chunk (steps)
constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t b) { return (b + kAlign - 1) & ~(kAlign - 1); }
constexpr size_t kStateOff = 0;
constexpr size_t kStateBytes = 2 * 6 * kStaticCells * sizeof(float);
constexpr size_t kCoefOff = align_up(kStateOff + kStateBytes);
constexpr size_t kCoefBytes = 6 * kStaticCells * sizeof(float);
constexpr size_t kAmpOff = align_up(kCoefOff + kCoefBytes);
constexpr size_t kAmpBytes = kStaticAmpSteps * kMaxSrc * sizeof(double);
constexpr size_t kMemberOff = align_up(kAmpOff + kAmpBytes);
constexpr size_t kSrcOff = align_up(kMemberOff + sizeof(Member));
constexpr size_t kChOff = align_up(kSrcOff + kMaxSrc * sizeof(fit_source));
constexpr size_t kErrOff = align_up(kChOff + 3 * sizeof(float));
constexpr size_t kFlagsOff = align_up(kErrOff + sizeof(int));
constexpr size_t kStaticScratchBytes = align_up(kFlagsOff + 64);

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// The device address of the scratch array on the current device; null on failure.
unsigned char *scratch_on_current_device() {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return nullptr;
    }
    return static_cast<unsigned char *>(p);
}

// device memory of the current device, or managed memory
bool on_device(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

int status_of(cudaError_t e) {
    if (e == cudaSuccess) return FIT_OK;
    return FIT_ERR_CUDA;
}

}  // namespace
}  // namespace fitgb

using namespace fitgb;

extern "C" int fit_leapfrog_run_static(int nx, int ny, int nz, double dx, double dy, double dz,
                                       const float *eps_r, const float *sigma, double dt, long nsteps,
                                       long step0, const fit_source *src, int nsrc, const fit_probe *prb,
                                       int nprb, double *probe_out, float *e_io, float *h_io, void *stream) {
    if (nx < 1 || ny < 1 || nz < 1 || nsteps < 0) return FIT_ERR_ARG;
    if (!(dx > 0) || !(dy > 0) || !(dz > 0) || !(dt > 0)) return FIT_ERR_ARG;
    if (!std::isfinite(dx) || !std::isfinite(dy) || !std::isfinite(dz) || !std::isfinite(dt)) return FIT_ERR_ARG;
    const int pitch = pitch_of(nx);
    const long long ncp = (long long)pitch * ny * nz;
    if (ncp > kStaticCells) return FIT_ERR_ARG;   // beyond the fixed scratch
    if (nsrc < 0 || nsrc > kMaxSrc || nprb < 0 || nprb > kMaxPrb) return FIT_ERR_ARG;
    if ((nsrc > 0 && !src) || (nprb > 0 && !prb)) return FIT_ERR_ARG;
    if (!eps_r || !e_io || !h_io || !on_device(eps_r) || !on_device(e_io) || !on_device(h_io)) return FIT_ERR_ARG;
    if (sigma && !on_device(sigma)) return FIT_ERR_ARG;
    if (probe_out && nprb > 0 && !on_device(probe_out)) return FIT_ERR_ARG;
    for (int s = 0; s < nsrc; ++s) {
        const int q[3] = {src[s].i, src[s].j, src[s].k};
        const int a = src[s].axis;
        if (a < 0 || a > 2 || q[0] < 0 || q[1] < 0 || q[2] < 0 || q[0] >= nx || q[1] >= ny || q[2] >= nz)
            return FIT_ERR_ARG;
        if (q[(a + 1) % 3] == 0 || q[(a + 2) % 3] == 0) return FIT_ERR_ARG;   // source on a PEC wall
        if (src[s].waveform < 0 || src[s].waveform > 2) return FIT_ERR_ARG;
        if (src[s].waveform != FIT_WAVE_SINE && !(src[s].width > 0.0)) return FIT_ERR_ARG;
    }
    for (int p = 0; p < nprb; ++p) {
        const fit_probe &r = prb[p];
        if (r.axis < 0 || r.axis > 2 || r.i < 0 || r.j < 0 || r.k < 0 || r.i >= nx || r.j >= ny || r.k >= nz)
            return FIT_ERR_ARG;
    }
    unsigned char *scr = scratch_on_current_device();
    if (!scr) return FIT_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float *state = reinterpret_cast<float *>(scr + kStateOff);
    float *coef = reinterpret_cast<float *>(scr + kCoefOff);
    double *amp = reinterpret_cast<double *>(scr + kAmpOff);
    Member *mem = reinterpret_cast<Member *>(scr + kMemberOff);
    fit_source *src_dev = reinterpret_cast<fit_source *>(scr + kSrcOff);
    float *ch = reinterpret_cast<float *>(scr + kChOff);
    int *err = reinterpret_cast<int *>(scr + kErrOff);
    void *flags = scr + kFlagsOff;

    // materials: valid values, lossy or not, and the CFL estimate (eq. cfl)
    MaterialFlags mf;
    const long long ncell = (long long)nx * ny * nz;
    cudaError_t ce = check_materials(eps_r, nullptr, sigma, ncell, &mf, flags, s);
    if (ce != cudaSuccess) return status_of(ce);
    if (mf.bad_eps || mf.bad_sigma) return FIT_ERR_NONFINITE;
    const double inv = 1.0 / (dx * dx) + 1.0 / (dy * dy) + 1.0 / (dz * dz);
    if (dt > std::sqrt(kEps0 * kMu0 * mf.eps_mu_min / inv) * (1.0 + 1e-12)) return FIT_ERR_CFL;
    const bool lossy = mf.lossy != 0;
    if (nsteps == 0) return FIT_OK;

    // state block 0 <- (e_io, h_io), rows re-pitched; everything else zero
    const size_t n6 = 6 * (size_t)ncp;
    const size_t row = (size_t)nx * sizeof(float), prow = (size_t)pitch * sizeof(float);
    const size_t rows3 = 3 * (size_t)ny * nz;
    if ((ce = cudaMemsetAsync(state, 0, 2 * n6 * sizeof(float), s)) != cudaSuccess) return status_of(ce);
    if ((ce = cudaMemcpy2DAsync(state, prow, e_io, row, row, rows3, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return status_of(ce);
    if ((ce = cudaMemcpy2DAsync(state + 3 * ncp, prow, h_io, row, row, rows3, cudaMemcpyDeviceToDevice, s)) !=
        cudaSuccess)
        return status_of(ce);
    if ((ce = mask_state<float>(nx, ny, nz, pitch, state, state + 3 * ncp, s)) != cudaSuccess) return status_of(ce);
    if ((ce = cudaMemsetAsync(err, 0, sizeof(int), s)) != cudaSuccess) return status_of(ce);

    // coefficients (semi-implicit sigma, mu_r = 1)
    const double d[3] = {dx, dy, dz};
    if ((ce = build_coeffs<float>(nx, ny, nz, pitch, d, eps_r, nullptr, sigma, dt, 0, false,
                                  lossy ? coef + 3 * ncp : nullptr, coef, ch, nullptr, nullptr, s)) != cudaSuccess)
        return status_of(ce);

    // the single member and the sources
    Member m;
    memset(&m, 0, sizeof(m));
    m.st[0] = state;
    m.st[1] = state + n6;
    m.blk[0] = 0;
    m.blk[1] = 1;
    m.start = step0;
    m.end = (1LL << 62);
    m.src_lo = -(1LL << 62);
    m.src_hi = (1LL << 62);
    m.probe = (probe_out && nprb > 0) ? probe_out : nullptr;
    m.probe_base = step0;
    if ((ce = cudaMemcpyAsync(mem, &m, sizeof(Member), cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return status_of(ce);
    if (nsrc > 0 &&
        (ce = cudaMemcpyAsync(src_dev, src, sizeof(fit_source) * nsrc, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return status_of(ce);

    StepArgs<float> a;
    memset(&a, 0, sizeof(a));
    a.nx = nx; a.ny = ny; a.nz = nz; a.pitch = pitch; a.ncell = ncp;
    Tile tile = {32, 8, 32, 2};
    a.tiles_x = (nx + tile.tx - 1) / tile.tx;
    a.tiles_y = (ny + tile.ty - 1) / tile.ty;
    const long long cols = (long long)a.tiles_x * a.tiles_y;
    while (tile.kz > 8 && cols * ((nz + tile.kz - 1) / tile.kz) < 4 * 152) tile.kz /= 2;
    a.kz = tile.kz;
    a.nchunk = (nz + tile.kz - 1) / tile.kz;
    a.cb = coef;
    a.ca = lossy ? coef + 3 * ncp : nullptr;
    a.ch = ch;
    a.mem = mem;
    a.nmem = 1;
    a.amp = amp;
    a.nsrc = nsrc;
    for (int q = 0; q < nsrc; ++q) a.src[q] = {src[q].axis, src[q].i, src[q].j, src[q].k};
    a.nprb = m.probe ? nprb : 0;
    for (int q = 0; q < nprb; ++q) a.prb[q] = {prb[q].axis, prb[q].i, prb[q].j, prb[q].k};
    a.err = err;
    TmaMaps maps;
    const bool use_tma = encode_tma_maps(&maps, (int)sizeof(float), nx, ny, nz, pitch, state, 2, coef,
                                         lossy ? 6 : 3, tile.tx, tile.ty);
    if (!use_tma) tile.kernel = 1;

    for (long long c0 = 0; c0 < nsteps; c0 += kStaticAmpSteps) {
        const long long len = (nsteps - c0 < kStaticAmpSteps) ? nsteps - c0 : kStaticAmpSteps;
        a.amp_base = step0 + c0;
        a.amp_len = len;
        if (nsrc > 0 && (ce = source_table(src_dev, nsrc, a.amp_base, len, dt, amp, s)) != cudaSuccess)
            return status_of(ce);
        for (long long it = c0; it < c0 + len; ++it) {
            a.it = (int)it;
            a.parity = (int)(it & 1);
            ce = use_tma ? launch_step_tma<float>(a, maps, tile, lossy, false, false, s)
                         : launch_step<float>(a, tile, lossy, false, false, s);
            if (ce != cudaSuccess) return status_of(ce);
        }
    }
    // final state -> caller's buffers
    const float *fin = state + ((nsteps & 1) ? n6 : 0);
    if ((ce = cudaMemcpy2DAsync(e_io, row, fin, prow, row, rows3, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return status_of(ce);
    if ((ce = cudaMemcpy2DAsync(h_io, row, fin + 3 * ncp, prow, row, rows3, cudaMemcpyDeviceToDevice, s)) !=
        cudaSuccess)
        return status_of(ce);
    int herr = 0;
    if ((ce = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return status_of(ce);
    if ((ce = cudaStreamSynchronize(s)) != cudaSuccess) return status_of(ce);
    if (herr) return (herr & kErrTimeout) ? FIT_ERR_TIMEOUT : FIT_ERR_ARG;
    return FIT_OK;
}
