// step.cu -- fused FIT leapfrog step (Sec. II-A of the paper) for one or
// many members in a single launch.
//
// One CTA owns a TX x TY column of cells of one member and streams it along
// z over a chunk of KZ planes (2.5-D blocking).  Per plane k it
//   1. stages e^n of plane k+1 (tile plus a one-cell halo on every side) in a
//      two-slot shared-memory ring -- plane k is already there;
//   2. computes h^{n+1/2} = h^{n-1/2} - ch (C e^n) for its cells and, again,
//      for the low-x column and low-y row next to the tile (their e^{n+1}
//      updates need h at i-1 and j-1; recomputing beats a second pass);
//   3. computes e^{n+1} = ca e^n + cb (C~ h^{n+1/2} - j^{n+1/2}) from the
//      shared h plane and the previous plane's h_x, h_y kept in registers.
// Each field value is read once from DRAM and written once per step; the
// halo re-reads hit L2.  Members advance from one buffer of their state pair
// into the other, so neighbouring CTAs never see a half-updated plane.
//
// The launch order puts the member index fastest: the CTAs that own the same
// tile of different members run side by side and read the same coefficients,
// which then come from L2 after the first of them.
//
// Sources, probes and the interleaved energy W^n (eq. energy) are fused:
// each CTA filters the few sources/probes that fall in its column once.
#include "internal.h"

namespace fitgb {
namespace {

template <typename T>
struct Acc;  // energy accumulator: Kahan-compensated in FP32, plain in FP64
template <>
struct Acc<float> {
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

template <typename T, int TX, int TY, bool LOSSY, bool MUARR, bool ENERGY>
__global__ void __launch_bounds__(TX *TY) step_kernel(const StepArgs<T> a) {
    constexpr int NT = TX * TY;
    constexpr int RX = TX + 2, RY = TY + 2;   // e region: tile plus halo
    __shared__ T sE[2][3][RY][RX];            // e^n, planes k and k+1
    __shared__ T sH[3][TY + 1][TX + 1];       // h^{n+1/2}, plane k, low halos
    __shared__ EdgeRef sSrcRef[kMaxSrc], sPrbRef[kMaxPrb];
    __shared__ int sSrc[kMaxSrc], sPrb[kMaxPrb];
    __shared__ int sNsrc, sNprb;
    __shared__ double sRed[NT / 32];

    const int tid = threadIdx.x;
    const int lx = tid % TX, ly = tid / TX;

    // CTA -> (member, tile, z chunk), member fastest
    int rest = blockIdx.x;
    const int m = rest % a.nmem;
    rest /= a.nmem;
    const int tile_x = rest % a.tiles_x;
    rest /= a.tiles_x;
    const int tile_y = rest % a.tiles_y;
    const int chunk = rest / a.tiles_y;

    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const long long ncell = a.ncell;
    const int pitch = a.pitch;
    const long long plane = (long long)pitch * ny;
    const int i0 = tile_x * TX, j0 = tile_y * TY;
    const int i = i0 + lx, j = j0 + ly;
    const bool own = (i < nx) && (j < ny);
    const int k0 = chunk * a.kz;
    const int k1 = min(nz, k0 + a.kz);

    const Member mb = a.mem[m];
    const long long step = mb.start + a.it;
    const T *__restrict__ in = static_cast<const T *>(a.parity ? mb.st[1] : mb.st[0]);
    T *__restrict__ out = static_cast<T *>(a.parity ? mb.st[0] : mb.st[1]);
    const T *__restrict__ iex = in;
    const T *__restrict__ iey = in + ncell;
    const T *__restrict__ iez = in + 2 * ncell;
    const T *__restrict__ ihx = in + 3 * ncell;
    const T *__restrict__ ihy = in + 4 * ncell;
    const T *__restrict__ ihz = in + 5 * ncell;

    // the sources and probes inside this CTA's column chunk (fixed-bound
    // loops keep the parameter arrays out of local memory)
    if (tid == 0) {
        int ns = 0, np = 0;
        const bool on = step >= mb.src_lo && step < mb.src_hi;
#pragma unroll
        for (int s = 0; s < kMaxSrc; ++s) {
            const EdgeRef r = a.src[s];
            if (on && s < a.nsrc && r.i >= i0 && r.i < i0 + TX && r.j >= j0 && r.j < j0 + TY && r.k >= k0 &&
                r.k < k1) {
                sSrc[ns] = s;
                sSrcRef[ns] = r;
                ++ns;
            }
        }
#pragma unroll
        for (int p = 0; p < kMaxPrb; ++p) {
            const EdgeRef r = a.prb[p];
            if (mb.probe && p < a.nprb && r.i >= i0 && r.i < i0 + TX && r.j >= j0 && r.j < j0 + TY &&
                r.k >= k0 && r.k < k1) {
                sPrb[np] = p;
                sPrbRef[np] = r;
                ++np;
            }
        }
        sNsrc = ns;
        sNprb = np;
    }

    T ch[3];
    if (!MUARR) {
        ch[0] = a.ch[0];
        ch[1] = a.ch[1];
        ch[2] = a.ch[2];
    }
    T mmu_c[3] = {T(0), T(0), T(0)};
    if (ENERGY && !MUARR) {
        mmu_c[0] = a.mmu[0];
        mmu_c[1] = a.mmu[1];
        mmu_c[2] = a.mmu[2];
    }

#define FIT_LOAD_PLANE(slot, kk)                                                            \
    do {                                                                                    \
        const bool kin_ = (kk) < nz;                                                        \
        for (int idx = tid; idx < RX * RY; idx += NT) {                                     \
            const int ii = idx % RX, jj = idx / RX;                                         \
            const int gi = i0 - 1 + ii, gj = j0 - 1 + jj;                                   \
            T vx = T(0), vy = T(0), vz = T(0);                                              \
            if (kin_ && gi >= 0 && gi < nx && gj >= 0 && gj < ny) {                         \
                const long long c_ = (long long)(kk) * plane + (long long)gj * pitch + gi;     \
                vx = iex[c_];                                                               \
                vy = iey[c_];                                                               \
                vz = iez[c_];                                                               \
            }                                                                               \
            sE[slot][0][jj][ii] = vx;                                                       \
            sE[slot][1][jj][ii] = vy;                                                       \
            sE[slot][2][jj][ii] = vz;                                                       \
        }                                                                                   \
    } while (0)

    const int kstart = (k0 > 0) ? k0 - 1 : k0;   // k0-1: prologue plane (h only)
    FIT_LOAD_PLANE(kstart & 1, kstart);

    T hxp = T(0), hyp = T(0);   // h_x, h_y at (i, j, k-1), step n+1/2
    Acc<T> wacc;

    // halo assignment: threads [0, TY) take the low-x column, [TY, TY+TX) the low-y row
    const bool hx_col = tid < TY;
    const bool hy_row = tid >= TY && tid < TY + TX;

    for (int k = kstart; k < k1; ++k) {
        const bool pro = k < k0;
        const int cur = k & 1, nxt = cur ^ 1;
        FIT_LOAD_PLANE(nxt, k + 1);

        const long long c = (long long)k * plane + (long long)j * pitch + i;
        T ho[3] = {T(0), T(0), T(0)};
        if (own) {
            ho[0] = ihx[c];
            ho[1] = ihy[c];
            ho[2] = ihz[c];
        }
        // old h on the halo cell this thread recomputes
        T hh0 = T(0), hh1 = T(0);
        int hi = -1, hj = -1;
        if (!pro) {
            if (hx_col) { hi = i0 - 1; hj = j0 + tid; }
            if (hy_row) { hi = i0 + tid - TY; hj = j0 - 1; }
            if (hi >= 0 && hj >= 0 && hi < nx && hj < ny) {
                const long long hc = (long long)k * plane + (long long)hj * pitch + hi;
                if (hx_col) { hh0 = ihy[hc]; hh1 = ihz[hc]; }   // h_y, h_z
                else        { hh0 = ihx[hc]; hh1 = ihz[hc]; }   // h_x, h_z
            } else {
                hi = -1;
            }
        }
        __syncthreads();   // (A) plane k+1 staged

        // ---- H half step, own cell: h -= ch * (C e)
        const int sx = lx + 1, sy = ly + 1;
        T chl[3];
        if (MUARR) {
            chl[0] = own ? a.ch[c] : T(0);
            chl[1] = own ? a.ch[ncell + c] : T(0);
            chl[2] = own ? a.ch[2 * ncell + c] : T(0);
        } else {
            chl[0] = ch[0]; chl[1] = ch[1]; chl[2] = ch[2];
        }
        const T ex0 = sE[cur][0][sy][sx], ey0 = sE[cur][1][sy][sx], ez0 = sE[cur][2][sy][sx];
        // (C e)_x = e_y(q) + e_z(q+y) - e_y(q+z) - e_z(q)
        const T cx = ey0 + sE[cur][2][sy + 1][sx] - sE[nxt][1][sy][sx] - ez0;
        // (C e)_y = e_z(q) + e_x(q+z) - e_z(q+x) - e_x(q)
        const T cy = ez0 + sE[nxt][0][sy][sx] - sE[cur][2][sy][sx + 1] - ex0;
        // (C e)_z = e_x(q) + e_y(q+x) - e_x(q+y) - e_y(q)
        const T cz = ex0 + sE[cur][1][sy][sx + 1] - sE[cur][0][sy + 1][sx] - ey0;
        const T hxn = ho[0] - chl[0] * cx;
        const T hyn = ho[1] - chl[1] * cy;
        const T hzn = ho[2] - chl[2] * cz;

        if (!pro) {
            sH[0][sy][sx] = hxn;
            sH[1][sy][sx] = hyn;
            sH[2][sy][sx] = hzn;
            if (hx_col || hy_row) {
                T v0 = T(0), v1 = T(0);
                if (hi >= 0) {
                    const int qx = hi - i0 + 1, qy = hj - j0 + 1;   // region coords
                    long long hc = (long long)k * plane + (long long)hj * pitch + hi;
                    if (hx_col) {
                        const T cyh = sE[cur][2][qy][qx] + sE[nxt][0][qy][qx] - sE[cur][2][qy][qx + 1]
                                      - sE[cur][0][qy][qx];
                        const T czh = sE[cur][0][qy][qx] + sE[cur][1][qy][qx + 1] - sE[cur][0][qy + 1][qx]
                                      - sE[cur][1][qy][qx];
                        const T c1 = MUARR ? a.ch[ncell + hc] : ch[1];
                        const T c2 = MUARR ? a.ch[2 * ncell + hc] : ch[2];
                        v0 = hh0 - c1 * cyh;
                        v1 = hh1 - c2 * czh;
                    } else {
                        const T cxh = sE[cur][1][qy][qx] + sE[cur][2][qy + 1][qx] - sE[nxt][1][qy][qx]
                                      - sE[cur][2][qy][qx];
                        const T czh = sE[cur][0][qy][qx] + sE[cur][1][qy][qx + 1] - sE[cur][0][qy + 1][qx]
                                      - sE[cur][1][qy][qx];
                        const T c0 = MUARR ? a.ch[hc] : ch[0];
                        const T c2 = MUARR ? a.ch[2 * ncell + hc] : ch[2];
                        v0 = hh0 - c0 * cxh;
                        v1 = hh1 - c2 * czh;
                    }
                }
                if (hx_col) {
                    sH[1][tid + 1][0] = v0;
                    sH[2][tid + 1][0] = v1;
                } else {
                    sH[0][0][tid - TY + 1] = v0;
                    sH[2][0][tid - TY + 1] = v1;
                }
            }
            if (own) {
                out[3 * ncell + c] = hxn;
                out[4 * ncell + c] = hyn;
                out[5 * ncell + c] = hzn;
            }
        }
        __syncthreads();   // (B) h plane complete

        if (!pro && own) {
            // ---- E half step: e = ca e + cb (C~h - j)
            // (C~h)_x = h_z(q) - h_z(q-y) - h_y(q) + h_y(q-z)
            T tx = hzn - sH[2][sy - 1][sx] - hyn + hyp;
            // (C~h)_y = h_x(q) - h_x(q-z) - h_z(q) + h_z(q-x)
            T ty = hxn - hxp - hzn + sH[2][sy][sx - 1];
            // (C~h)_z = h_y(q) - h_y(q-x) - h_x(q) + h_x(q-y)
            T tz = hyn - sH[1][sy][sx - 1] - hxn + sH[0][sy - 1][sx];
            for (int q = 0; q < sNsrc; ++q) {
                const int s = sSrc[q];
                const EdgeRef r = sSrcRef[q];
                if (r.i == i && r.j == j && r.k == k) {
                    const T jv = (T)a.amp[(step - a.amp_base) * a.nsrc + s];
                    if (r.axis == 0) tx -= jv;
                    else if (r.axis == 1) ty -= jv;
                    else tz -= jv;
                }
            }
            const T bx = a.cb[c], by = a.cb[ncell + c], bz = a.cb[2 * ncell + c];
            T exn, eyn, ezn;
            if (LOSSY) {
                exn = a.ca[c] * ex0 + bx * tx;
                eyn = a.ca[ncell + c] * ey0 + by * ty;
                ezn = a.ca[2 * ncell + c] * ez0 + bz * tz;
            } else {
                exn = ex0 + bx * tx;
                eyn = ey0 + by * ty;
                ezn = ez0 + bz * tz;
            }
            out[c] = exn;
            out[ncell + c] = eyn;
            out[2 * ncell + c] = ezn;
            for (int q = 0; q < sNprb; ++q) {
                const int p = sPrb[q];
                const EdgeRef r = sPrbRef[q];
                if (r.i == i && r.j == j && r.k == k) {
                    const T v = r.axis == 0 ? exn : (r.axis == 1 ? eyn : ezn);
                    mb.probe[(step - mb.probe_base) * a.nprb + p] = (double)v;
                }
            }
            if (ENERGY) {
                const T me0 = a.meps[c], me1 = a.meps[ncell + c], me2 = a.meps[2 * ncell + c];
                T mu0, mu1, mu2;
                if (MUARR) {
                    mu0 = a.mmu[c]; mu1 = a.mmu[ncell + c]; mu2 = a.mmu[2 * ncell + c];
                } else {
                    mu0 = mmu_c[0]; mu1 = mmu_c[1]; mu2 = mmu_c[2];
                }
                wacc.add(me0 * ex0 * ex0);
                wacc.add(me1 * ey0 * ey0);
                wacc.add(me2 * ez0 * ez0);
                wacc.add(mu0 * ho[0] * hxn);
                wacc.add(mu1 * ho[1] * hyn);
                wacc.add(mu2 * ho[2] * hzn);
            }
        }
        hxp = hxn;
        hyp = hyn;
    }
#undef FIT_LOAD_PLANE

    if (ENERGY) {
        double v = wacc.value();
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if ((tid & 31) == 0) sRed[tid >> 5] = v;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < NT / 32; ++w) t += sRed[w];
            if (mb.energy) atomicAdd(mb.energy + (step - mb.energy_base), t);
        }
    }
}

template <typename T, int TX, int TY>
cudaError_t launch_tile(const StepArgs<T> &a, bool lossy, bool muarr, bool energy, cudaStream_t s) {
    if (a.occ_out) return report_occupancy(step_kernel<T, TX, TY, true, false, false>, TX * TY, 0, a.occ_out);
    const long long blocks = (long long)a.nmem * a.tiles_x * a.tiles_y * a.nchunk;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)blocks), block(TX * TY);
#define FIT_LAUNCH(L, M, E) step_kernel<T, TX, TY, L, M, E><<<grid, block, 0, s>>>(a)
    if (lossy) {
        if (muarr) { if (energy) FIT_LAUNCH(true, true, true); else FIT_LAUNCH(true, true, false); }
        else       { if (energy) FIT_LAUNCH(true, false, true); else FIT_LAUNCH(true, false, false); }
    } else {
        if (muarr) { if (energy) FIT_LAUNCH(false, true, true); else FIT_LAUNCH(false, true, false); }
        else       { if (energy) FIT_LAUNCH(false, false, true); else FIT_LAUNCH(false, false, false); }
    }
#undef FIT_LAUNCH
    return cudaGetLastError();
}

}  // namespace

bool tile_supported(int tx, int ty) {
    return (tx == 32 && (ty == 4 || ty == 8 || ty == 16)) || (tx == 64 && (ty == 2 || ty == 4)) ||
           (tx == 16 && ty == 8);
}

template <typename T>
cudaError_t launch_step(const StepArgs<T> &a, Tile t, bool lossy, bool muarr, bool energy, cudaStream_t s) {
    if (t.tx == 32 && t.ty == 8) return launch_tile<T, 32, 8>(a, lossy, muarr, energy, s);
    if (t.tx == 32 && t.ty == 4) return launch_tile<T, 32, 4>(a, lossy, muarr, energy, s);
    if (t.tx == 32 && t.ty == 16) return launch_tile<T, 32, 16>(a, lossy, muarr, energy, s);
    if (t.tx == 64 && t.ty == 4) return launch_tile<T, 64, 4>(a, lossy, muarr, energy, s);
    if (t.tx == 64 && t.ty == 2) return launch_tile<T, 64, 2>(a, lossy, muarr, energy, s);
    if (t.tx == 16 && t.ty == 8) return launch_tile<T, 16, 8>(a, lossy, muarr, energy, s);
    return cudaErrorInvalidValue;
}

template cudaError_t launch_step<float>(const StepArgs<float> &, Tile, bool, bool, bool, cudaStream_t);
template cudaError_t launch_step<double>(const StepArgs<double> &, Tile, bool, bool, bool, cudaStream_t);

}  // namespace fitgb
