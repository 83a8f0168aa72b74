// step2_tma.cu -- two leapfrog steps (Sec. II-A) per launch with a TMA
// pipeline: temporal blocking of the FP32 step for member-batched runs.
//
// Each CTA owns a TX x TY column of one member and streams it along z; the
// member's state (e^n, h^{n-1/2}) is read once and (e^{n+2}, h^{n+3/2}) is
// written once, so a cell-update moves half the field bytes of the one-step
// kernel (coefficients are still read once per launch).  Plane data arrives
// by TMA into an S-deep ring: e, h of the plane on the window x in
// [i0-4, i0+TX+4), y in [j0-2, j0+TY+2) (x aligned to 16 bytes, out-of-grid
// cells zero), and the coefficients (cb, ca) on the same window.
//
// The first step is computed on a region that covers what the second step
// needs (the halo recompute of the 2.5-D scheme):
//   h1 = h^{n+1/2} on x in [i0-2, i0+TX], y in [j0-2, j0+TY]
//   e1 = e^{n+1}   on x in [i0-1, i0+TX], y in [j0-1, j0+TY]  (sources of
//        step n on every edge of that region)
//   h2 = h^{n+3/2} on the tile plus its low-x column and low-y row
//   e2 = e^{n+2}   on the tile (sources of step n+1)
// The second step lags one plane: iteration t (planes t and t+1 present)
// computes h1, e1 of plane t and h2, e2 of plane t-1.  h1 and e1 keep two
// planes in shared memory; h2 of plane t-2 (x, y components) and the tile's
// coefficients of plane t-1 stay in registers.  A chunk [k0, k1) starts at
// plane k0-2 (zeros below the grid) and reads up to plane k1+1.
//
// A member with a single step left takes only the first step and writes h1, e1
// of the tile.  Probes record e^{n+1} and e^{n+2}.  Waits are bounded as in
// step_tma.cuh: on timeout the CTA records kErrTimeout, waits (bounded) for its
// own copies and returns.
#include "internal.h"
#include "step_tma.cuh"

namespace fitgb {
namespace {

using tma::mbar_expect_tx;
using tma::mbar_init;
using tma::mbar_init_fence;
using tma::mbar_wait;
using tma::proxy_fence;
using tma::tma_load_4d;
using tma::tma_load_5d;

template <int TX, int TY, int S, bool LOSSY>
struct G2 {
    static constexpr int NT = TX * TY;
    static constexpr int BX = TX + 8, EY = TY + 4;    // window
    static constexpr int NC = LOSSY ? 6 : 3;
    static constexpr int W3 = 3 * EY * BX * 4;        // one 3-component window of floats
    static constexpr int H_OFF = tma::align128(W3);
    static constexpr int C_OFF = H_OFF + tma::align128(W3);
    static constexpr int STAGE = C_OFF + tma::align128(NC * EY * BX * 4);
    static constexpr uint32_t TX_BYTES = 2 * W3 + NC * EY * BX * 4;
    // regions (width x height) of the first step
    static constexpr int H1X = TX + 3, H1Y = TY + 3;  // origin (i0-2, j0-2)
    static constexpr int E1X = TX + 2, E1Y = TY + 2;  // origin (i0-1, j0-1)
    static constexpr int H2X = TX + 1, H2Y = TY + 1;  // origin (i0-1, j0-1)
    static constexpr int SMEM_PLANES = (2 * 3 * H1Y * H1X + 2 * 3 * E1Y * E1X + 3 * H2Y * H2X) * 4;
    static constexpr int DYN_SMEM = S * STAGE + 128 + tma::align128(SMEM_PLANES);
};

struct S2Small {
    EdgeRef src_ref[kMaxSrc], prb_ref[kMaxPrb];
    int src_idx[kMaxSrc], prb_idx[kMaxPrb];
    int nsrc, nprb;
};

template <int TX, int TY, int S, bool LOSSY>
__global__ void __launch_bounds__(TX *TY) step2_tma_kernel(const __grid_constant__ StepArgs<float> a,
                                                           const __grid_constant__ CUtensorMap tm_state,
                                                           const __grid_constant__ CUtensorMap tm_coef, int muarr) {
    using G = G2<TX, TY, S, LOSSY>;
    constexpr int NT = G::NT, BX = G::BX, EY = G::EY;
    constexpr int H1X = G::H1X, H1Y = G::H1Y, E1X = G::E1X, E1Y = G::E1Y, H2X = G::H2X, H2Y = G::H2Y;
    static_assert(S >= 3, "planes t and t+1 are read while t+2 is in flight");
    static_assert(2 * (TX + TY) <= NT, "halo threads");
    __shared__ uint64_t bar[S];
    __shared__ S2Small sm;
    unsigned char *dsm = tma::aligned_dsm<float, TX, TY, S>();
    float *planes = reinterpret_cast<float *>(dsm + S * G::STAGE);
    float *h1s = planes;                              // [2][3][H1Y][H1X]
    float *e1s = h1s + 2 * 3 * H1Y * H1X;             // [2][3][E1Y][E1X]
    float *h2s = e1s + 2 * 3 * E1Y * E1X;             // [3][H2Y][H2X]
#define H1(sl, c, y, x) h1s[(((sl) * 3 + (c)) * H1Y + (y)) * H1X + (x)]
#define E1(sl, c, y, x) e1s[(((sl) * 3 + (c)) * E1Y + (y)) * E1X + (x)]
#define H2(c, y, x) h2s[((c) * H2Y + (y)) * H2X + (x)]
#define WV(buf, c, y, x) (buf)[((c) * EY + (y)) * BX + (x)]

    int rest = blockIdx.x;
    const int m = rest % a.nmem;
    rest /= a.nmem;
    const int tile_x = rest % a.tiles_x;
    rest /= a.tiles_x;
    const int tile_y = rest % a.tiles_y;
    const int chunk = rest / a.tiles_y;
    const Member mb = a.mem[m];
    const int nx = a.nx, ny = a.ny, nz = a.nz, pitch = a.pitch;
    const long long ncell = a.ncell;
    const int i0 = tile_x * TX, j0 = tile_y * TY;
    const int k0 = chunk * a.kz, k1 = min(nz, k0 + a.kz);
    const long long step = mb.start + a.it;
    const int nsteps = (int)min(2LL, mb.end - step);
    const int blk_in = a.parity ? mb.blk[1] : mb.blk[0];
    float *__restrict__ out = static_cast<float *>(a.parity ? mb.st[0] : mb.st[1]);
    const bool src_on0 = step >= mb.src_lo && step < mb.src_hi;
    const bool src_on1 = step + 1 >= mb.src_lo && step + 1 < mb.src_hi;
    const int tid = threadIdx.x, lx = tid % TX, ly = tid / TX;
    const int i = i0 + lx, j = j0 + ly;
    const bool own = i < nx && j < ny;
    const float *chg = a.ch;

    // the first prologue iteration reads the plane-(t-1) slots before anything was written there
    for (int idx = tid; idx < G::SMEM_PLANES / 4; idx += NT) planes[idx] = 0.f;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
        mbar_init_fence();
        int ns = 0, np = 0;
        for (int s = 0; s < a.nsrc; ++s) {   // sources on the first step's e region (or the tile)
            const EdgeRef r = a.src[s];
            if (r.i >= i0 - 1 && r.i <= i0 + TX && r.j >= j0 - 1 && r.j <= j0 + TY && r.k >= k0 - 1 && r.k <= k1) {
                sm.src_idx[ns] = s;
                sm.src_ref[ns] = r;
                ++ns;
            }
        }
        for (int p = 0; p < a.nprb && mb.probe; ++p) {
            const EdgeRef r = a.prb[p];
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

    const int kstart = k0 - 2;
    const int total = k1 - kstart + 2;   // planes kstart .. k1+1
    auto issue = [&](int p) {
        const int kk = kstart + p;
        unsigned char *st = dsm + (p % S) * G::STAGE;
        uint64_t *b = &bar[p % S];
        mbar_expect_tx(b, G::TX_BYTES + (p == 0 ? (uint32_t)a.extra_tx : 0u));
        tma_load_5d(st, &tm_state, b, i0 - 4, j0 - 2, kk, 0, blk_in);
        tma_load_5d(st + G::H_OFF, &tm_state, b, i0 - 4, j0 - 2, kk, 3, blk_in);
        tma_load_4d(st + G::C_OFF, &tm_coef, b, i0 - 4, j0 - 2, kk, 0);
    };
    const int limit = a.wait_limit > 0 ? a.wait_limit : tma::kWaitLimit;
    uint32_t phase = 0;
    auto wait_plane = [&](int p) -> bool {
        const int st = p % S;
        const bool ok = mbar_wait(&bar[st], (phase >> st) & 1u, limit);
        if (ok) phase ^= (1u << st);
        return ok;
    };
    int issued = 0;
    if (tid == 0) {
        proxy_fence();
        for (; issued < min(S, total); ++issued) issue(issued);
    }
    int bad = wait_plane(0) ? 0 : 1;
    int waited = bad ? 0 : 1;
    bool aborted = false;

    const float chs0 = muarr ? 0.f : chg[0], chs1 = muarr ? 0.f : chg[1], chs2 = muarr ? 0.f : chg[2];
    auto ch_at = [&](int comp, int ci, int cj, int ck) -> float {
        if (!muarr) return comp == 0 ? chs0 : (comp == 1 ? chs1 : chs2);
        if (ci < 0 || cj < 0 || ck < 0 || ci >= nx || cj >= ny || ck >= nz) return 0.f;
        return chg[comp * ncell + ((long long)ck * ny + cj) * pitch + ci];
    };
    // source current of step `st` on edge (axis, ci, cj, ck) of plane ck
    auto jsrc = [&](int axis, int ci, int cj, int ck, long long st, bool on) -> float {
        float v = 0.f;
        if (!on) return v;
        for (int q = 0; q < sm.nsrc; ++q) {
            const EdgeRef r = sm.src_ref[q];
            if (r.axis == axis && r.i == ci && r.j == cj && r.k == ck)
                v += (float)a.amp[(st - a.amp_base) * a.nsrc + sm.src_idx[q]];
        }
        return v;
    };
    const bool lo_col = tid < TY, lo_row = tid >= TY && tid < TY + TX;
    float h2xp = 0.f, h2yp = 0.f;                 // h2 of plane t-2 at this cell (x, y)
    float cbp0 = 0.f, cbp1 = 0.f, cbp2 = 0.f, cap0 = 1.f, cap1 = 1.f, cap2 = 1.f;   // tile coefficients, plane t-1
    float cbc0 = 0.f, cbc1 = 0.f, cbc2 = 0.f, cac0 = 1.f, cac1 = 1.f, cac2 = 1.f;   // the same of plane t

    for (int t = kstart; t <= k1; ++t) {
        const int p = t - kstart;
        const float *eC = reinterpret_cast<const float *>(dsm + (p % S) * G::STAGE);
        const float *hC = reinterpret_cast<const float *>(dsm + (p % S) * G::STAGE + G::H_OFF);
        const float *cC = reinterpret_cast<const float *>(dsm + (p % S) * G::STAGE + G::C_OFF);
        const float *eN = reinterpret_cast<const float *>(dsm + ((p + 1) % S) * G::STAGE);
        if (!bad) {
            if (wait_plane(p + 1)) waited = p + 2;
            else bad = 1;
        }
        if (__syncthreads_or(bad)) {
            aborted = true;
            break;
        }
        const int sc = (t + 4) & 1, sp = sc ^ 1;   // slots of planes t and t-1
        // (1) h1 of plane t on [i0-2, i0+TX] x [j0-2, j0+TY]; window x = rx + 2, y = ry
        for (int idx = tid; idx < H1X * H1Y; idx += NT) {
            const int rx = idx % H1X, ry = idx / H1X;
            const int x = rx + 2, y = ry;
            const float ex = WV(eC, 0, y, x), ey = WV(eC, 1, y, x), ez = WV(eC, 2, y, x);
            const float cx = (ey + WV(eC, 2, y + 1, x)) - (WV(eN, 1, y, x) + ez);
            const float cy = (ez + WV(eN, 0, y, x)) - (WV(eC, 2, y, x + 1) + ex);
            const float cz = (ex + WV(eC, 1, y, x + 1)) - (WV(eC, 0, y + 1, x) + ey);
            const int ci = i0 - 2 + rx, cj = j0 - 2 + ry;
            H1(sc, 0, ry, rx) = WV(hC, 0, y, x) - ch_at(0, ci, cj, t) * cx;
            H1(sc, 1, ry, rx) = WV(hC, 1, y, x) - ch_at(1, ci, cj, t) * cy;
            H1(sc, 2, ry, rx) = WV(hC, 2, y, x) - ch_at(2, ci, cj, t) * cz;
        }
        __syncthreads();
        // (2) e1 of plane t on [i0-1, i0+TX] x [j0-1, j0+TY]; h1 index = e1 index + 1
        for (int idx = tid; idx < E1X * E1Y; idx += NT) {
            const int rx = idx % E1X, ry = idx / E1X;
            const int hx = rx + 1, hy = ry + 1;       // h1 region coordinates of this cell
            const int x = rx + 3, y = ry + 1;         // window coordinates
            const float tx = (H1(sc, 2, hy, hx) - H1(sc, 2, hy - 1, hx)) - (H1(sc, 1, hy, hx) - H1(sp, 1, hy, hx));
            const float ty = (H1(sc, 0, hy, hx) - H1(sp, 0, hy, hx)) - (H1(sc, 2, hy, hx) - H1(sc, 2, hy, hx - 1));
            const float tz = (H1(sc, 1, hy, hx) - H1(sc, 1, hy, hx - 1)) - (H1(sc, 0, hy, hx) - H1(sc, 0, hy - 1, hx));
            const int ci = i0 - 1 + rx, cj = j0 - 1 + ry;
            float jx = 0.f, jy = 0.f, jz = 0.f;
            if (sm.nsrc > 0) {
                jx = jsrc(0, ci, cj, t, step, src_on0);
                jy = jsrc(1, ci, cj, t, step, src_on0);
                jz = jsrc(2, ci, cj, t, step, src_on0);
            }
            const float e0x = WV(eC, 0, y, x), e0y = WV(eC, 1, y, x), e0z = WV(eC, 2, y, x);
            const float bx = WV(cC, 0, y, x), by = WV(cC, 1, y, x), bz = WV(cC, 2, y, x);
            float ax = 1.f, ay = 1.f, az = 1.f;
            if (LOSSY) {
                ax = WV(cC, 3, y, x);
                ay = WV(cC, 4, y, x);
                az = WV(cC, 5, y, x);
            }
            E1(sc, 0, ry, rx) = (LOSSY ? ax * e0x : e0x) + bx * (tx - jx);
            E1(sc, 1, ry, rx) = (LOSSY ? ay * e0y : e0y) + by * (ty - jy);
            E1(sc, 2, ry, rx) = (LOSSY ? az * e0z : e0z) + bz * (tz - jz);
        }
        // this cell's coefficients of plane t (for e2 of plane t at the next iteration)
        {
            const int x = lx + 4, y = ly + 2;
            cbc0 = WV(cC, 0, y, x); cbc1 = WV(cC, 1, y, x); cbc2 = WV(cC, 2, y, x);
            if (LOSSY) {
                cac0 = WV(cC, 3, y, x); cac1 = WV(cC, 4, y, x); cac2 = WV(cC, 5, y, x);
            }
        }
        __syncthreads();
        const long long c1 = ((long long)t * ny + j) * pitch + i;   // cell of plane t
        if (nsteps == 1) {
            // a member's last step: h1, e1 of the tile are its output
            if (t >= k0 && t < k1 && own && !bad) {
                out[c1] = E1(sc, 0, ly + 1, lx + 1);
                out[ncell + c1] = E1(sc, 1, ly + 1, lx + 1);
                out[2 * ncell + c1] = E1(sc, 2, ly + 1, lx + 1);
                out[3 * ncell + c1] = H1(sc, 0, ly + 2, lx + 2);
                out[4 * ncell + c1] = H1(sc, 1, ly + 2, lx + 2);
                out[5 * ncell + c1] = H1(sc, 2, ly + 2, lx + 2);
                for (int q = 0; q < sm.nprb; ++q) {
                    const EdgeRef r = sm.prb_ref[q];
                    if (r.i == i && r.j == j && r.k == t)
                        mb.probe[(step - mb.probe_base) * a.nprb + sm.prb_idx[q]] =
                            (double)E1(sc, r.axis, ly + 1, lx + 1);
                }
            }
        } else {
            const int tm = t - 1;   // plane of the second step
            // (3) h2 of plane t-1 on the tile and its low halos; e1 of plane t-1 in slot sp
            auto h2_at = [&](int ex_, int ey_, int ci, int cj, float &o0, float &o1, float &o2) {
                // e1 region coordinates (ex_, ey_) of the cell; h1 region = +1
                const float ex = E1(sp, 0, ey_, ex_), ey = E1(sp, 1, ey_, ex_), ez = E1(sp, 2, ey_, ex_);
                const float cx = (ey + E1(sp, 2, ey_ + 1, ex_)) - (E1(sc, 1, ey_, ex_) + ez);
                const float cy = (ez + E1(sc, 0, ey_, ex_)) - (E1(sp, 2, ey_, ex_ + 1) + ex);
                const float cz = (ex + E1(sp, 1, ey_, ex_ + 1)) - (E1(sp, 0, ey_ + 1, ex_) + ey);
                o0 = H1(sp, 0, ey_ + 1, ex_ + 1) - ch_at(0, ci, cj, tm) * cx;
                o1 = H1(sp, 1, ey_ + 1, ex_ + 1) - ch_at(1, ci, cj, tm) * cy;
                o2 = H1(sp, 2, ey_ + 1, ex_ + 1) - ch_at(2, ci, cj, tm) * cz;
            };
            float h2x, h2y, h2z;
            h2_at(lx + 1, ly + 1, i, j, h2x, h2y, h2z);
            H2(0, ly + 1, lx + 1) = h2x;
            H2(1, ly + 1, lx + 1) = h2y;
            H2(2, ly + 1, lx + 1) = h2z;
            {
                float o0, o1, o2;
                if (lo_col) {   // cell (i0-1, j0+tid): h2 y, z
                    h2_at(0, tid + 1, i0 - 1, j0 + tid, o0, o1, o2);
                    H2(1, tid + 1, 0) = o1;
                    H2(2, tid + 1, 0) = o2;
                } else if (lo_row) {   // cell (i0+t, j0-1): h2 x, z
                    const int q = tid - TY;
                    h2_at(q + 1, 0, i0 + q, j0 - 1, o0, o1, o2);
                    H2(0, 0, q + 1) = o0;
                    H2(2, 0, q + 1) = o2;
                }
            }
            __syncthreads();
            // (4) e2 of plane t-1 on the tile
            if (tm >= k0 && tm < k1 && own && !bad) {
                const long long c = ((long long)tm * ny + j) * pitch + i;
                const float tx = (h2z - H2(2, ly, lx + 1)) - (h2y - h2yp);
                const float ty = (h2x - h2xp) - (h2z - H2(2, ly + 1, lx));
                const float tz = (h2y - H2(1, ly + 1, lx)) - (h2x - H2(0, ly, lx + 1));
                float jx = 0.f, jy = 0.f, jz = 0.f;
                if (sm.nsrc > 0) {
                    jx = jsrc(0, i, j, tm, step + 1, src_on1);
                    jy = jsrc(1, i, j, tm, step + 1, src_on1);
                    jz = jsrc(2, i, j, tm, step + 1, src_on1);
                }
                const float e1x = E1(sp, 0, ly + 1, lx + 1), e1y = E1(sp, 1, ly + 1, lx + 1),
                            e1z = E1(sp, 2, ly + 1, lx + 1);
                const float e2x = (LOSSY ? cap0 * e1x : e1x) + cbp0 * (tx - jx);
                const float e2y = (LOSSY ? cap1 * e1y : e1y) + cbp1 * (ty - jy);
                const float e2z = (LOSSY ? cap2 * e1z : e1z) + cbp2 * (tz - jz);
                out[c] = e2x;
                out[ncell + c] = e2y;
                out[2 * ncell + c] = e2z;
                out[3 * ncell + c] = h2x;
                out[4 * ncell + c] = h2y;
                out[5 * ncell + c] = h2z;
                for (int q = 0; q < sm.nprb; ++q) {
                    const EdgeRef r = sm.prb_ref[q];
                    if (r.i == i && r.j == j && r.k == tm) {
                        double *row = mb.probe + (step - mb.probe_base) * a.nprb + sm.prb_idx[q];
                        row[0] = (double)E1(sp, r.axis, ly + 1, lx + 1);
                        row[a.nprb] = (double)(r.axis == 0 ? e2x : (r.axis == 1 ? e2y : e2z));
                    }
                }
            }
            h2xp = h2x;
            h2yp = h2y;
        }
        cbp0 = cbc0; cbp1 = cbc1; cbp2 = cbc2;
        cap0 = cac0; cap1 = cac1; cap2 = cac2;
        __syncthreads();   // stage p, the h1/e1 slots of plane t-1 and the h2 plane are free again
        if (tid == 0 && issued < total) {
            proxy_fence();
            issue(issued);
            ++issued;
        }
    }
#undef H1
#undef E1
#undef H2
#undef WV
    if (aborted && tid == 0) {
        atomicOr(a.err, kErrTimeout);
        for (int q = waited; q < issued; ++q) wait_plane(q);
    }
}

template <int TX, int TY, int S, bool LOSSY>
cudaError_t launch2(const StepArgs<float> &a, const CUtensorMap &st, const CUtensorMap &co, bool muarr,
                    cudaStream_t s) {
    using G = G2<TX, TY, S, LOSSY>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(step2_tma_kernel<TX, TY, S, LOSSY>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, G::DYN_SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const long long blocks = (long long)a.nmem * a.tiles_x * a.tiles_y * a.nchunk;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    step2_tma_kernel<TX, TY, S, LOSSY><<<(unsigned)blocks, TX * TY, G::DYN_SMEM, s>>>(a, st, co, muarr ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace

bool step2_tile_supported(int tx, int ty) { return (tx == 32 && ty == 8) || (tx == 32 && ty == 16); }

cudaError_t launch_step2_tma(const StepArgs<float> &a, const CUtensorMap &tm_state, const CUtensorMap &tm_coef,
                             int tx, int ty, bool lossy, bool muarr, cudaStream_t s) {
    if (tx == 32 && ty == 8)
        return lossy ? launch2<32, 8, 3, true>(a, tm_state, tm_coef, muarr, s)
                     : launch2<32, 8, 3, false>(a, tm_state, tm_coef, muarr, s);
    if (tx == 32 && ty == 16)
        return lossy ? launch2<32, 16, 3, true>(a, tm_state, tm_coef, muarr, s)
                     : launch2<32, 16, 3, false>(a, tm_state, tm_coef, muarr, s);
    return cudaErrorInvalidValue;
}

}  // namespace fitgb
