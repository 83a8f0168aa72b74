// step_tma.cuh -- the fused FIT leapfrog step (Sec. II-A of the paper) with a
// TMA pipeline: the GB300 path of the hot loop.
//
// One CTA owns a TX x TY column of cells of one member and streams it along z
// over a chunk of planes (2.5-D blocking).  Plane data arrives by TMA
// (cp.async.bulk.tensor) into an S-deep shared-memory ring, one stage per
// plane, completing on one mbarrier per stage:
//   e^n       of the plane, x in [i0-4, i0+TX+4), y in [j0-1, j0+TY+1)
//   h^{n-1/2} of the plane, same window
//   cb (and ca) of the plane's TX x TY cells
// The e/h window starts 4 cells left of the tile so that its x coordinate is
// 16-byte aligned, as TMA requires; cells outside the grid arrive as zeros
// (the tensor maps' out-of-bounds fill), which is exactly the PEC/ghost
// value, so no bounds test is needed on the loads.  Thread 0 keeps S planes
// in flight, so DRAM latency hides behind the compute of earlier planes.
//
// Per plane k every thread computes h^{n+1/2} = h^{n-1/2} - ch (C e^n) for its
// cell (and the first TX+TY threads also for the low-x column / low-y row
// next to the tile, whose values its neighbours' e updates need), then
// e^{n+1} = ca e^n + cb (C~h^{n+1/2} - j^{n+1/2}) using the shared h plane and
// the previous plane's h_x, h_y kept in registers.  Fields are written with
// coalesced stores into the member's other state block.  Every byte of e, h
// and the coefficients is read once from DRAM per step (halo re-reads come
// from L2) and every field value is written once.
//
// Sources, probes and the interleaved energy W^n (eq. energy) are fused as in
// the plain-load kernel.  Every mbarrier wait is bounded: on timeout the CTA
// records kErrTimeout, stops, waits (bounded) for its own copies in flight
// and returns.
#pragma once

#include "internal.h"

namespace fitgb {
namespace tma {

constexpr int kWaitLimit = 1 << 22;

__device__ __forceinline__ uint32_t saddr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void proxy_fence() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int limit = kWaitLimit) {
    for (int n = 0; n < limit; ++n)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_load_5d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1,
                                            int c2, int c3, int c4) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(saddr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(saddr(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1,
                                            int c2, int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(saddr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(saddr(bar))
        : "memory");
}

constexpr int align128(int b) { return (b + 127) & ~127; }

template <typename T>
struct Acc;
template <>
struct Acc<float> {   // Kahan-compensated FP32
    float s = 0.f, c = 0.f;
    __device__ void add(float x) {
        float y = x - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ double value() const { return (double)s - (double)c; }
};
template <>
struct Acc<double> {
    double s = 0.0;
    __device__ void add(double x) { s += x; }
    __device__ double value() const { return s; }
};

template <typename T, int TX, int TY, int S, bool LOSSY>
struct Geometry {
    static constexpr int NT = TX * TY;
    static constexpr int BX = TX + 8;   // e/h window width: 4 cells each side
    static constexpr int EY = TY + 2;   // e/h window height: 1 row each side
    static constexpr int NC = LOSSY ? 6 : 3;
    static constexpr int E_BYTES = 3 * EY * BX * (int)sizeof(T);
    static constexpr int C_BYTES = NC * TY * TX * (int)sizeof(T);
    static constexpr int H_OFF = align128(E_BYTES);
    static constexpr int C_OFF = H_OFF + align128(E_BYTES);
    static constexpr int STAGE = C_OFF + align128(C_BYTES);
    static constexpr uint32_t TX_BYTES = 2 * E_BYTES + C_BYTES;
    static constexpr int DYN_SMEM = S * STAGE + 128;   // + room to align the base to 128 B
};

// Everything one CTA needs to advance one tile column (i0, j0, z chunk) of
// one member of one grid by one step.
template <typename T>
struct TileJob {
    int nx, ny, nz, pitch;
    long long ncell;          // pitch*ny*nz
    int i0, j0, k0, k1;
    const T *ch;              // 3 values, or 3 pitched components (muarr)
    const T *meps, *mmu;      // energy only
    int muarr, energy;
    long long step;           // absolute step of the member
    int blk_in;               // state block read (TMA coordinate)
    T *out;                   // state block written
    bool src_on;              // sources active at this step
    const double *amp;
    long long amp_base;
    int nsrc;
    const EdgeRef *src;       // generic pointer (parameter or global space)
    int nprb;
    const EdgeRef *prb;
    double *probe;
    long long probe_base;
    double *energy_out;       // energy row of this step, or null
    int *err;
    int wait_limit;           // polls per wait (kWaitLimit when 0)
    int extra_tx;             // test hook, see StepArgs
    const T *ge1, *ge0;       // fused adjoint gradient (GRAD kernels), see StepArgs
    float *gb;
    float gk[3];
    float *gd;                // e^{n+1} - e^n output of the forward sweep (two-cell FP32 kernel), see StepArgs
};

// Shared memory of the tile pipeline (dynamic stage ring + these statics).
template <typename T, int TX, int TY, int S>
struct TileSmem {
    uint64_t bar[S];
    T sH[3][TY + 1][TX + 1];   // h^{n+1/2} of plane k with low halos
    EdgeRef src_ref[kMaxSrc], prb_ref[kMaxPrb];
    int src_idx[kMaxSrc], prb_idx[kMaxPrb];
    int nsrc, nprb;
    double red[TX * TY / 32];
};

// One tile column of one step.  `phase` holds the parity of each stage's
// mbarrier; it carries over between calls on the same CTA.  Returns false if
// a bounded wait gave up (kErrTimeout recorded, no copy left in flight).
template <typename T, int TX, int TY, int S, bool LOSSY, bool GRAD = false>
__device__ __forceinline__ bool tma_tile(const TileJob<T> &J, const CUtensorMap *tm_state,
                                         const CUtensorMap *tm_coef, unsigned char *dsm,
                                         TileSmem<T, TX, TY, S> &sm, uint32_t &phase) {
    using G = Geometry<T, TX, TY, S, LOSSY>;
    constexpr int NT = G::NT, BX = G::BX, EY = G::EY;
    static_assert(S >= 3, "the e plane k+1 is read while plane k+S is in flight");
    static_assert(TX + TY <= NT, "halo threads");
    const int tid = threadIdx.x;
    const int lx = tid % TX, ly = tid / TX;
    const int nx = J.nx, ny = J.ny, pitch = J.pitch;
    const long long ncell = J.ncell;
    const int i0 = J.i0, j0 = J.j0, k0 = J.k0, k1 = J.k1;
    const int i = i0 + lx, j = j0 + ly;
    const bool own = (i < nx) && (j < ny);
    const int kstart = (k0 > 0) ? k0 - 1 : k0;   // k0-1: prologue plane (h only)
    const int total = k1 - kstart + 1;            // planes kstart .. k1
    T *__restrict__ out = J.out;

    if (tid == 0) {
        int ns = 0, np = 0;
        for (int s = 0; s < J.nsrc && J.src_on; ++s) {
            const EdgeRef r = J.src[s];
            if (r.i >= i0 && r.i < i0 + TX && r.j >= j0 && r.j < j0 + TY && r.k >= k0 && r.k < k1) {
                sm.src_idx[ns] = s;
                sm.src_ref[ns] = r;
                ++ns;
            }
        }
        for (int p = 0; p < J.nprb && J.probe; ++p) {
            const EdgeRef r = J.prb[p];
            if (r.i >= i0 && r.i < i0 + TX && r.j >= j0 && r.j < j0 + TY && r.k >= k0 && r.k < k1) {
                sm.prb_idx[np] = p;
                sm.prb_ref[np] = r;
                ++np;
            }
        }
        sm.nsrc = ns;
        sm.nprb = np;
    }
    __syncthreads();

    auto issue = [&](int p) {   // thread 0: start the copies of plane kstart + p
        const int kk = kstart + p;
        unsigned char *st = dsm + (p % S) * G::STAGE;
        uint64_t *b = &sm.bar[p % S];
        mbar_expect_tx(b, G::TX_BYTES + (p == 0 ? (uint32_t)J.extra_tx : 0u));
        tma_load_5d(st, tm_state, b, i0 - 4, j0 - 1, kk, 0, J.blk_in);
        tma_load_5d(st + G::H_OFF, tm_state, b, i0 - 4, j0 - 1, kk, 3, J.blk_in);
        tma_load_4d(st + G::C_OFF, tm_coef, b, i0, j0, kk, 0);
    };
    // wait for plane p (its stage's parity flips with every use)
    const int limit = J.wait_limit > 0 ? J.wait_limit : kWaitLimit;
    auto wait_plane = [&](int p) -> bool {
        const int st = p % S;
        const bool ok = mbar_wait(&sm.bar[st], (phase >> st) & 1u, limit);
        if (ok) phase ^= (1u << st);
        return ok;
    };
    int issued = 0;
    if (tid == 0) {
        proxy_fence();
        for (; issued < min(S, total); ++issued) issue(issued);
    }

    T ch[3] = {T(0), T(0), T(0)};
    if (!J.muarr) {
        ch[0] = J.ch[0];
        ch[1] = J.ch[1];
        ch[2] = J.ch[2];
    }
    T mmu_c[3] = {T(0), T(0), T(0)};
    if (J.energy && !J.muarr) {
        mmu_c[0] = J.mmu[0];
        mmu_c[1] = J.mmu[1];
        mmu_c[2] = J.mmu[2];
    }
    const bool hx_col = tid < TY;                   // low-x halo column
    const bool hy_row = tid >= TY && tid < TY + TX; // low-y halo row
    T hxp = T(0), hyp = T(0);   // h_x, h_y at (i, j, k-1), step n+1/2
    Acc<T> wacc;
    int bad = wait_plane(0) ? 0 : 1;
    int waited = bad ? 0 : 1;   // planes whose copies are known complete
    bool aborted = false;

    for (int k = kstart; k < k1; ++k) {
        const int p = k - kstart;
        const bool pro = k < k0;
        const T *eC = reinterpret_cast<const T *>(dsm + (p % S) * G::STAGE);
        const T *hC = reinterpret_cast<const T *>(dsm + (p % S) * G::STAGE + G::H_OFF);
        const T *cC = reinterpret_cast<const T *>(dsm + (p % S) * G::STAGE + G::C_OFF);
        const T *eN = reinterpret_cast<const T *>(dsm + ((p + 1) % S) * G::STAGE);
        if (!bad) {
            if (wait_plane(p + 1)) waited = p + 2;
            else bad = 1;
        }
#define EV(buf, comp, y, x) (buf)[((comp) * EY + (y)) * BX + (x)]
        const int sx = lx + 4, sy = ly + 1;
        const long long c = ((long long)k * ny + j) * pitch + i;
        T chl0 = ch[0], chl1 = ch[1], chl2 = ch[2];
        if (J.muarr) {
            chl0 = own ? J.ch[c] : T(0);
            chl1 = own ? J.ch[ncell + c] : T(0);
            chl2 = own ? J.ch[2 * ncell + c] : T(0);
        }
        const T ex0 = EV(eC, 0, sy, sx), ey0 = EV(eC, 1, sy, sx), ez0 = EV(eC, 2, sy, sx);
        const T ho0 = EV(hC, 0, sy, sx), ho1 = EV(hC, 1, sy, sx), ho2 = EV(hC, 2, sy, sx);
        // (C e)_x = e_y(q) + e_z(q+y) - e_y(q+z) - e_z(q)
        const T cx = ey0 + EV(eC, 2, sy + 1, sx) - EV(eN, 1, sy, sx) - ez0;
        // (C e)_y = e_z(q) + e_x(q+z) - e_z(q+x) - e_x(q)
        const T cy = ez0 + EV(eN, 0, sy, sx) - EV(eC, 2, sy, sx + 1) - ex0;
        // (C e)_z = e_x(q) + e_y(q+x) - e_x(q+y) - e_y(q)
        const T cz = ex0 + EV(eC, 1, sy, sx + 1) - EV(eC, 0, sy + 1, sx) - ey0;
        const T hxn = ho0 - chl0 * cx;
        const T hyn = ho1 - chl1 * cy;
        const T hzn = ho2 - chl2 * cz;
        if (!pro) {
            sm.sH[0][sy][lx + 1] = hxn;
            sm.sH[1][sy][lx + 1] = hyn;
            sm.sH[2][sy][lx + 1] = hzn;
            if (hx_col) {   // cell (i0-1, j0+tid): window x = 3
                const int y = tid + 1;
                T c1 = ch[1], c2 = ch[2];
                if (J.muarr) {
                    const int hi = i0 - 1, hj = j0 + tid;
                    const bool in = hi >= 0 && hj < ny;
                    const long long hc = ((long long)k * ny + hj) * pitch + hi;
                    c1 = in ? J.ch[ncell + hc] : T(0);
                    c2 = in ? J.ch[2 * ncell + hc] : T(0);
                }
                const T cyh = EV(eC, 2, y, 3) + EV(eN, 0, y, 3) - EV(eC, 2, y, 4) - EV(eC, 0, y, 3);
                const T czh = EV(eC, 0, y, 3) + EV(eC, 1, y, 4) - EV(eC, 0, y + 1, 3) - EV(eC, 1, y, 3);
                sm.sH[1][y][0] = EV(hC, 1, y, 3) - c1 * cyh;
                sm.sH[2][y][0] = EV(hC, 2, y, 3) - c2 * czh;
            } else if (hy_row) {   // cell (i0+t, j0-1): window y = 0
                const int t = tid - TY, x = t + 4;
                T c0 = ch[0], c2 = ch[2];
                if (J.muarr) {
                    const int hi = i0 + t, hj = j0 - 1;
                    const bool in = hj >= 0 && hi < nx;
                    const long long hc = ((long long)k * ny + hj) * pitch + hi;
                    c0 = in ? J.ch[hc] : T(0);
                    c2 = in ? J.ch[2 * ncell + hc] : T(0);
                }
                const T cxh = EV(eC, 1, 0, x) + EV(eC, 2, 1, x) - EV(eN, 1, 0, x) - EV(eC, 2, 0, x);
                const T czh = EV(eC, 0, 0, x) + EV(eC, 1, 0, x + 1) - EV(eC, 0, 1, x) - EV(eC, 1, 0, x);
                sm.sH[0][0][t + 1] = EV(hC, 0, 0, x) - c0 * cxh;
                sm.sH[2][0][t + 1] = EV(hC, 2, 0, x) - c2 * czh;
            }
            if (own && !bad) {
                out[3 * ncell + c] = hxn;
                out[4 * ncell + c] = hyn;
                out[5 * ncell + c] = hzn;
            }
        }
#undef EV
        if (__syncthreads_or(bad)) {   // (B) h plane complete
            aborted = true;
            break;
        }
        if (!pro && own) {
            const int sxh = lx + 1;
            // (C~h)_x = h_z(q) - h_z(q-y) - h_y(q) + h_y(q-z)
            T tx = hzn - sm.sH[2][sy - 1][sxh] - hyn + hyp;
            // (C~h)_y = h_x(q) - h_x(q-z) - h_z(q) + h_z(q-x)
            T ty = hxn - hxp - hzn + sm.sH[2][sy][sxh - 1];
            // (C~h)_z = h_y(q) - h_y(q-x) - h_x(q) + h_x(q-y)
            T tz = hyn - sm.sH[1][sy][sxh - 1] - hxn + sm.sH[0][sy - 1][sxh];
            for (int q = 0; q < sm.nsrc; ++q) {
                const EdgeRef r = sm.src_ref[q];
                if (r.i == i && r.j == j && r.k == k) {
                    const T jv = (T)J.amp[(J.step - J.amp_base) * J.nsrc + sm.src_idx[q]];
                    if (r.axis == 0) tx -= jv;
                    else if (r.axis == 1) ty -= jv;
                    else tz -= jv;
                }
            }
            const int cc = ly * TX + lx;
            const T bx = cC[cc], by = cC[TY * TX + cc], bz = cC[2 * TY * TX + cc];
            T exn, eyn, ezn;
            if (LOSSY) {
                exn = cC[3 * TY * TX + cc] * ex0 + bx * tx;
                eyn = cC[4 * TY * TX + cc] * ey0 + by * ty;
                ezn = cC[5 * TY * TX + cc] * ez0 + bz * tz;
            } else {
                exn = ex0 + bx * tx;
                eyn = ey0 + by * ty;
                ezn = ez0 + bz * tz;
            }
            out[c] = exn;
            out[ncell + c] = eyn;
            out[2 * ncell + c] = ezn;
            if (GRAD) {   // the input e is the adjoint state mu^{n+1}
                J.gb[c] += J.gk[0] * (ex0 * (J.ge1[c] - J.ge0[c]));
                J.gb[ncell + c] += J.gk[1] * (ey0 * (J.ge1[ncell + c] - J.ge0[ncell + c]));
                J.gb[2 * ncell + c] += J.gk[2] * (ez0 * (J.ge1[2 * ncell + c] - J.ge0[2 * ncell + c]));
            }
            for (int q = 0; q < sm.nprb; ++q) {
                const EdgeRef r = sm.prb_ref[q];
                if (r.i == i && r.j == j && r.k == k) {
                    const T v = r.axis == 0 ? exn : (r.axis == 1 ? eyn : ezn);
                    J.probe[(J.step - J.probe_base) * J.nprb + sm.prb_idx[q]] = (double)v;
                }
            }
            if (J.energy) {
                const T me0 = J.meps[c], me1 = J.meps[ncell + c], me2 = J.meps[2 * ncell + c];
                T mu0 = mmu_c[0], mu1 = mmu_c[1], mu2 = mmu_c[2];
                if (J.muarr) {
                    mu0 = J.mmu[c];
                    mu1 = J.mmu[ncell + c];
                    mu2 = J.mmu[2 * ncell + c];
                }
                wacc.add(me0 * ex0 * ex0);
                wacc.add(me1 * ey0 * ey0);
                wacc.add(me2 * ez0 * ez0);
                wacc.add(mu0 * ho0 * hxn);
                wacc.add(mu1 * ho1 * hyn);
                wacc.add(mu2 * ho2 * hzn);
            }
        }
        hxp = hxn;
        hyp = hyn;
        __syncthreads();   // (C) stage p and the h plane are free again
        if (tid == 0 && issued < total) {
            proxy_fence();
            issue(issued);
            ++issued;
        }
    }

    if (aborted) {
        if (tid == 0) {
            atomicOr(J.err, kErrTimeout);
            // do not leave while copies into this CTA's shared memory are pending
            for (int p = waited; p < issued; ++p) wait_plane(p);
        }
        return false;
    }
    if (J.energy) {
        double v = wacc.value();
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if ((tid & 31) == 0) sm.red[tid >> 5] = v;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < NT / 32; ++w) t += sm.red[w];
            if (J.energy_out) atomicAdd(J.energy_out, t);
        }
        __syncthreads();
    }
    return true;
}

template <typename T, int TX, int TY, int S>
__device__ __forceinline__ unsigned char *aligned_dsm() {
    extern __shared__ __align__(128) unsigned char dsm_raw[];
    return reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(dsm_raw) + 127) &
                                             ~static_cast<uintptr_t>(127));
}

// Single grid: one CTA = one (member, tile, chunk), member fastest.
template <typename T, int TX, int TY, int S, bool LOSSY, bool GRAD = false>
__global__ void __launch_bounds__(TX *TY) step_tma_kernel(const __grid_constant__ StepArgs<T> a,
                                                          const __grid_constant__ CUtensorMap tm_state,
                                                          const __grid_constant__ CUtensorMap tm_coef, int muarr,
                                                          int energy) {
    __shared__ TileSmem<T, TX, TY, S> sm;
    unsigned char *dsm = aligned_dsm<T, TX, TY, S>();
    int rest = blockIdx.x;
    const int m = rest % a.nmem;
    rest /= a.nmem;
    const int tile_x = rest % a.tiles_x;
    rest /= a.tiles_x;
    const int tile_y = rest % a.tiles_y;
    const int chunk = rest / a.tiles_y;
    const Member mb = a.mem[m];
    TileJob<T> J;
    J.nx = a.nx; J.ny = a.ny; J.nz = a.nz; J.pitch = a.pitch; J.ncell = a.ncell;
    J.i0 = tile_x * TX;
    J.j0 = tile_y * TY;
    J.k0 = chunk * a.kz;
    J.k1 = min(a.nz, J.k0 + a.kz);
    J.ch = a.ch; J.meps = a.meps; J.mmu = a.mmu; J.muarr = muarr; J.energy = energy;
    J.step = mb.start + a.it;
    J.blk_in = a.parity ? mb.blk[1] : mb.blk[0];
    J.out = static_cast<T *>(a.parity ? mb.st[0] : mb.st[1]);
    J.src_on = J.step >= mb.src_lo && J.step < mb.src_hi;
    J.amp = a.amp; J.amp_base = a.amp_base; J.nsrc = a.nsrc; J.src = a.src;
    J.nprb = a.nprb; J.prb = a.prb; J.probe = mb.probe; J.probe_base = mb.probe_base;
    J.energy_out = (energy && mb.energy) ? mb.energy + (J.step - mb.energy_base) : nullptr;
    J.err = a.err;
    J.wait_limit = a.wait_limit;
    J.extra_tx = a.extra_tx;
    J.ge1 = a.ge1;
    J.ge0 = a.ge0;
    J.gb = a.gb;
    J.gk[0] = a.gk[0];
    J.gk[1] = a.gk[1];
    J.gk[2] = a.gk[2];
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&sm.bar[s], 1);
        mbar_init_fence();
    }
    __syncthreads();
    uint32_t phase = 0;
    tma_tile<T, TX, TY, S, LOSSY, GRAD>(J, &tm_state, &tm_coef, dsm, sm, phase);
}

// Many grids: persistent CTAs (about one per resident slot) take work items
// from an atomic counter until the list is exhausted.  Items are ordered by
// (grid, tile, chunk, member), members innermost, so the CTAs working on one
// tile of different members run side by side and share its coefficients in
// L2; a member past its last step is skipped.
template <typename T, int TX, int TY, int S, bool LOSSY>
__global__ void __launch_bounds__(TX *TY) batched_tma_kernel(const __grid_constant__ BatchArgs<T> b) {
    __shared__ TileSmem<T, TX, TY, S> sm;
    unsigned char *dsm = aligned_dsm<T, TX, TY, S>();
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&sm.bar[s], 1);
        mbar_init_fence();
    }
    __syncthreads();
    uint32_t phase = 0;
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(b.counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= b.nitems) break;
        const WorkItem w = b.items[item];
        const GridDesc<T> &gd = b.grids[w.grid];
        const Member mb = gd.mem[w.member];
        if (mb.start + b.it >= mb.end) continue;   // member finished: nothing to do
        const int tile_x = w.tile % gd.tiles_x;
        const int tile_y = w.tile / gd.tiles_x;
        TileJob<T> J;
        J.nx = gd.nx; J.ny = gd.ny; J.nz = gd.nz; J.pitch = gd.pitch; J.ncell = gd.ncell;
        J.i0 = tile_x * TX;
        J.j0 = tile_y * TY;
        J.k0 = w.chunk * gd.kz;
        J.k1 = min(gd.nz, J.k0 + gd.kz);
        J.ch = gd.ch; J.meps = nullptr; J.mmu = nullptr; J.muarr = gd.muarr; J.energy = 0;
        J.step = mb.start + b.it;
        J.blk_in = b.parity ? mb.blk[1] : mb.blk[0];
        J.out = static_cast<T *>(b.parity ? mb.st[0] : mb.st[1]);
        J.src_on = J.step >= mb.src_lo && J.step < mb.src_hi;
        J.amp = gd.amp; J.amp_base = gd.amp_base; J.nsrc = gd.nsrc; J.src = gd.src;
        J.nprb = gd.nprb; J.prb = gd.prb; J.probe = mb.probe; J.probe_base = mb.probe_base;
        J.energy_out = nullptr;
        J.err = b.err;
        J.wait_limit = 0;
        J.extra_tx = 0;
        if (!tma_tile<T, TX, TY, S, LOSSY>(J, &b.maps[2 * w.grid], &b.maps[2 * w.grid + 1], dsm, sm, phase))
            return;
    }
}

template <typename T, int TX, int TY, int S, bool LOSSY, bool GRAD = false>
cudaError_t launch_one(const StepArgs<T> &a, const TmaMaps &maps, bool muarr, bool energy, cudaStream_t s) {
    using G = Geometry<T, TX, TY, S, LOSSY>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(step_tma_kernel<T, TX, TY, S, LOSSY, GRAD>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, G::DYN_SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (a.occ_out) return report_occupancy(step_tma_kernel<T, TX, TY, S, LOSSY, GRAD>, TX * TY, G::DYN_SMEM, a.occ_out);
    const long long blocks = (long long)a.nmem * a.tiles_x * a.tiles_y * a.nchunk;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    step_tma_kernel<T, TX, TY, S, LOSSY, GRAD><<<(unsigned)blocks, TX * TY, G::DYN_SMEM, s>>>(
        a, maps.state, maps.coef, muarr ? 1 : 0, energy ? 1 : 0);
    return cudaGetLastError();
}

template <typename T, int TX, int TY, int S, bool LOSSY>
cudaError_t launch_batched_one(const BatchArgs<T> &b, int ctas, cudaStream_t s) {
    using G = Geometry<T, TX, TY, S, LOSSY>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(batched_tma_kernel<T, TX, TY, S, LOSSY>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, G::DYN_SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (b.nitems <= 0) return cudaSuccess;
    const int grid = ctas < b.nitems ? ctas : b.nitems;
    batched_tma_kernel<T, TX, TY, S, LOSSY><<<grid, TX * TY, G::DYN_SMEM, s>>>(b);
    return cudaGetLastError();
}

// resident CTAs per SM of a batched configuration (for the persistent grid size)
template <typename T, int TX, int TY, int S, bool LOSSY>
int batched_occupancy() {
    using G = Geometry<T, TX, TY, S, LOSSY>;
    int n = 0;
    cudaFuncSetAttribute(batched_tma_kernel<T, TX, TY, S, LOSSY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         G::DYN_SMEM);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batched_tma_kernel<T, TX, TY, S, LOSSY>, TX * TY,
                                                      G::DYN_SMEM) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

}  // namespace tma
}  // namespace fitgb
