// step_tma2.cuh -- the fused FP32 leapfrog step of step_tma.cuh with two cells
// per thread (Sec. II-A of the paper).
//
// The TMA ring, the windows and the tile geometry are those of tma_tile: a CTA
// owns a TX x TY column of cells of one member and streams it along z, plane
// data arriving by TMA into an S-deep shared-memory ring with one mbarrier per
// stage, every wait bounded.  Thread (t, y) owns the x-adjacent cells
// A = (i0+2t, j) and B = A + u_x, so
//   * shared-memory reads and global stores are 8 bytes wide,
//   * B's low-x neighbour is A and A's high-x neighbour is B (registers),
//   * the per-plane overhead (waits, barriers, index and address arithmetic,
//     the source and probe checks) is paid once per two cells.
// The arithmetic of each cell is the same expression, in the same order, as in
// tma_tile, so both kernels give the same fields.  The first TX/2 threads also
// compute the low-y halo row (pairs), the last TY threads the low-x halo
// column (single cells).
#pragma once

#include "step_tma.cuh"

namespace fitgb {
namespace tma {

// optional epilogues of the two-cell step kernel (template parameter EXTRA)
constexpr int kExtraNone = 0;
constexpr int kExtraGrad = 1;   // adjoint step: accumulate the gradient (StepArgs gb, ge1, ge0, gk)
constexpr int kExtraDiff = 2;   // forward step: write e^{n+1} - e^n (StepArgs gd)

template <int TX, int TY, int S>
struct TileSmem2 {
    uint64_t bar[S];
    // h^{n+1/2} of plane k: row 0 = low-y halo row, column 1 = low-x halo
    // column, cell x at column x + 2 (pairs 8-byte aligned)
    __align__(16) float sH[3][TY + 1][TX + 2];
    EdgeRef src_ref[kMaxSrc], prb_ref[kMaxPrb];
    int src_idx[kMaxSrc], prb_idx[kMaxPrb];
    int nsrc, nprb;
    double red[TX / 2 * TY / 32 + 1];
};

// One tile column of one step with two cells per thread; see tma_tile for the
// contract (phase, return value, error handling).
template <int TX, int TY, int S, bool LOSSY, int EXTRA = 0>
__device__ __forceinline__ bool tma_tile2(const TileJob<float> &J, const CUtensorMap *tm_state,
                                          const CUtensorMap *tm_coef, unsigned char *dsm,
                                          TileSmem2<TX, TY, S> &sm, uint32_t &phase) {
    using G = Geometry<float, TX, TY, S, LOSSY>;
    constexpr int BX = G::BX, EY = G::EY;
    constexpr int PX = TX / 2, NT = PX * TY;
    static_assert(S >= 3, "the e plane k+1 is read while plane k+S is in flight");
    static_assert(TX % 2 == 0 && PX + TY <= NT, "pairs and halo threads");
    const int tid = threadIdx.x;
    const int tx = tid % PX, ty = tid / PX;
    const int nx = J.nx, ny = J.ny, pitch = J.pitch;
    const long long ncell = J.ncell;
    const int i0 = J.i0, j0 = J.j0, k0 = J.k0, k1 = J.k1;
    const int i = i0 + 2 * tx, j = j0 + ty;
    const bool ownA = (i < nx) && (j < ny), ownB = (i + 1 < nx) && (j < ny);
    const int kstart = (k0 > 0) ? k0 - 1 : k0;
    const int total = k1 - kstart + 1;
    float *__restrict__ out = J.out;

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
    const int nsrc_cta = sm.nsrc, nprb_cta = sm.nprb;

    auto issue = [&](int p) {   // thread 0: start the copies of plane kstart + p
        const int kk = kstart + p;
        unsigned char *st = dsm + (p % S) * G::STAGE;
        uint64_t *b = &sm.bar[p % S];
        mbar_expect_tx(b, G::TX_BYTES + (p == 0 ? (uint32_t)J.extra_tx : 0u));
        tma_load_5d(st, tm_state, b, i0 - 4, j0 - 1, kk, 0, J.blk_in);
        tma_load_5d(st + G::H_OFF, tm_state, b, i0 - 4, j0 - 1, kk, 3, J.blk_in);
        tma_load_4d(st + G::C_OFF, tm_coef, b, i0, j0, kk, 0);
    };
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

    float ch0 = 0.f, ch1 = 0.f, ch2 = 0.f;
    if (!J.muarr) {
        ch0 = J.ch[0];
        ch1 = J.ch[1];
        ch2 = J.ch[2];
    }
    float mu0 = 0.f, mu1 = 0.f, mu2 = 0.f;
    if (J.energy && !J.muarr) {
        mu0 = J.mmu[0];
        mu1 = J.mmu[1];
        mu2 = J.mmu[2];
    }
    const bool hy_row = tid < PX;                   // low-y halo row, pair tid
    // low-x halo column: the last TY threads, cell tid - (NT - TY) (another warp than the
    // halo row's whenever the tile has more than one warp, so no warp runs both branches)
    const bool hx_col = tid >= NT - TY;
    float2 hxp = make_float2(0.f, 0.f), hyp = hxp;  // h_x, h_y at (., j, k-1), step n+1/2
    Acc<float> wacc;
    int bad = wait_plane(0) ? 0 : 1;
    int waited = bad ? 0 : 1;   // planes whose copies are known complete
    bool aborted = false;
    const int sx = 4 + 2 * tx, sy = ty + 1, hx = 2 * tx + 2;

#define EV(buf, comp, y, x) (buf)[((comp) * EY + (y)) * BX + (x)]
#define F2(ptr) (*reinterpret_cast<const float2 *>(ptr))
    for (int k = kstart; k < k1; ++k) {
        const int p = k - kstart;
        const bool pro = k < k0;
        const float *eC = reinterpret_cast<const float *>(dsm + (p % S) * G::STAGE);
        const float *hC = reinterpret_cast<const float *>(dsm + (p % S) * G::STAGE + G::H_OFF);
        const float *cC = reinterpret_cast<const float *>(dsm + (p % S) * G::STAGE + G::C_OFF);
        const float *eN = reinterpret_cast<const float *>(dsm + ((p + 1) % S) * G::STAGE);
        if (!bad) {
            if (wait_plane(p + 1)) waited = p + 2;
            else bad = 1;
        }
        const long long c = ((long long)k * ny + j) * pitch + i;
        float2 cA = make_float2(ch0, ch0), cB = make_float2(ch1, ch1), cZ = make_float2(ch2, ch2);
        if (J.muarr) {
            cA = ownA ? F2(J.ch + c) : make_float2(0.f, 0.f);
            cB = ownA ? F2(J.ch + ncell + c) : make_float2(0.f, 0.f);
            cZ = ownA ? F2(J.ch + 2 * ncell + c) : make_float2(0.f, 0.f);
        }
        const float2 ex = F2(&EV(eC, 0, sy, sx)), ey = F2(&EV(eC, 1, sy, sx)), ez = F2(&EV(eC, 2, sy, sx));
        const float eyx = EV(eC, 1, sy, sx + 2), ezx = EV(eC, 2, sy, sx + 2);
        const float2 exy = F2(&EV(eC, 0, sy + 1, sx)), ezy = F2(&EV(eC, 2, sy + 1, sx));
        const float2 exz = F2(&EV(eN, 0, sy, sx)), eyz = F2(&EV(eN, 1, sy, sx));
        const float2 ho0 = F2(&EV(hC, 0, sy, sx)), ho1 = F2(&EV(hC, 1, sy, sx)), ho2 = F2(&EV(hC, 2, sy, sx));
        // (C e)_x = e_y(q) + e_z(q+y) - e_y(q+z) - e_z(q)
        // (C e)_y = e_z(q) + e_x(q+z) - e_z(q+x) - e_x(q)
        // (C e)_z = e_x(q) + e_y(q+x) - e_x(q+y) - e_y(q)
        const float cxA = ey.x + ezy.x - eyz.x - ez.x, cxB = ey.y + ezy.y - eyz.y - ez.y;
        const float cyA = ez.x + exz.x - ez.y - ex.x, cyB = ez.y + exz.y - ezx - ex.y;
        const float czA = ex.x + ey.y - exy.x - ey.x, czB = ex.y + eyx - exy.y - ey.y;
        const float2 hxn = make_float2(ho0.x - cA.x * cxA, ho0.y - cA.y * cxB);
        const float2 hyn = make_float2(ho1.x - cB.x * cyA, ho1.y - cB.y * cyB);
        const float2 hzn = make_float2(ho2.x - cZ.x * czA, ho2.y - cZ.y * czB);
        if (!pro) {
            *reinterpret_cast<float2 *>(&sm.sH[0][sy][hx]) = hxn;
            *reinterpret_cast<float2 *>(&sm.sH[1][sy][hx]) = hyn;
            *reinterpret_cast<float2 *>(&sm.sH[2][sy][hx]) = hzn;
            if (hy_row) {   // cells (i0+2t, j0-1), (i0+2t+1, j0-1): window y = 0; h_x and h_z
                const int t = tid, x = 4 + 2 * t;
                float2 c0 = make_float2(ch0, ch0), c2 = make_float2(ch2, ch2);
                if (J.muarr) {
                    const bool in = j0 >= 1 && i0 + 2 * t < nx;
                    const long long hc = ((long long)k * ny + (j0 - 1)) * pitch + (i0 + 2 * t);
                    c0 = in ? F2(J.ch + hc) : make_float2(0.f, 0.f);
                    c2 = in ? F2(J.ch + 2 * ncell + hc) : make_float2(0.f, 0.f);
                }
                const float2 ez0 = F2(&EV(eC, 2, 0, x)), ez1 = F2(&EV(eC, 2, 1, x));
                const float2 ey0 = F2(&EV(eC, 1, 0, x)), eyN = F2(&EV(eN, 1, 0, x));
                const float ey0x = EV(eC, 1, 0, x + 2);
                const float2 ex0 = F2(&EV(eC, 0, 0, x)), ex1 = F2(&EV(eC, 0, 1, x));
                const float2 h0 = F2(&EV(hC, 0, 0, x)), h2 = F2(&EV(hC, 2, 0, x));
                const float cxa = ey0.x + ez1.x - eyN.x - ez0.x, cxb = ey0.y + ez1.y - eyN.y - ez0.y;
                const float cza = ex0.x + ey0.y - ex1.x - ey0.x, czb = ex0.y + ey0x - ex1.y - ey0.y;
                *reinterpret_cast<float2 *>(&sm.sH[0][0][2 * t + 2]) =
                    make_float2(h0.x - c0.x * cxa, h0.y - c0.y * cxb);
                *reinterpret_cast<float2 *>(&sm.sH[2][0][2 * t + 2]) =
                    make_float2(h2.x - c2.x * cza, h2.y - c2.y * czb);
            } else if (hx_col) {   // cell (i0-1, j0+y-1): window x = 3; h_y and h_z
                const int y = tid - (NT - TY) + 1;
                float c1 = ch1, c2 = ch2;
                if (J.muarr) {
                    const int hi = i0 - 1, hj = j0 + y - 1;
                    const bool in = hi >= 0 && hj < ny;
                    const long long hc = ((long long)k * ny + hj) * pitch + hi;
                    c1 = in ? J.ch[ncell + hc] : 0.f;
                    c2 = in ? J.ch[2 * ncell + hc] : 0.f;
                }
                const float cyh = EV(eC, 2, y, 3) + EV(eN, 0, y, 3) - EV(eC, 2, y, 4) - EV(eC, 0, y, 3);
                const float czh = EV(eC, 0, y, 3) + EV(eC, 1, y, 4) - EV(eC, 0, y + 1, 3) - EV(eC, 1, y, 3);
                sm.sH[1][y][1] = EV(hC, 1, y, 3) - c1 * cyh;
                sm.sH[2][y][1] = EV(hC, 2, y, 3) - c2 * czh;
            }
            if (ownA && !bad) {
                *reinterpret_cast<float2 *>(out + 3 * ncell + c) = hxn;
                *reinterpret_cast<float2 *>(out + 4 * ncell + c) = hyn;
                *reinterpret_cast<float2 *>(out + 5 * ncell + c) = hzn;
            }
        }
        if (__syncthreads_or(bad)) {   // (B) h plane complete
            aborted = true;
            break;
        }
        if (!pro && ownA) {
            const float2 hzmy = F2(&sm.sH[2][sy - 1][hx]), hxmy = F2(&sm.sH[0][sy - 1][hx]);
            const float hzmx = sm.sH[2][sy][hx - 1], hymx = sm.sH[1][sy][hx - 1];
            // (C~h)_x = h_z(q) - h_z(q-y) - h_y(q) + h_y(q-z)
            // (C~h)_y = h_x(q) - h_x(q-z) - h_z(q) + h_z(q-x)
            // (C~h)_z = h_y(q) - h_y(q-x) - h_x(q) + h_x(q-y)
            float txA = hzn.x - hzmy.x - hyn.x + hyp.x, txB = hzn.y - hzmy.y - hyn.y + hyp.y;
            float tyA = hxn.x - hxp.x - hzn.x + hzmx, tyB = hxn.y - hxp.y - hzn.y + hzn.x;
            float tzA = hyn.x - hymx - hxn.x + hxmy.x, tzB = hyn.y - hyn.x - hxn.y + hxmy.y;
            for (int q = 0; q < nsrc_cta; ++q) {
                const EdgeRef r = sm.src_ref[q];
                if (r.j == j && r.k == k && (r.i == i || r.i == i + 1)) {
                    const float jv = (float)J.amp[(J.step - J.amp_base) * J.nsrc + sm.src_idx[q]];
                    const bool b = r.i != i;
                    if (r.axis == 0) {
                        if (b) txB -= jv; else txA -= jv;
                    } else if (r.axis == 1) {
                        if (b) tyB -= jv; else tyA -= jv;
                    } else {
                        if (b) tzB -= jv; else tzA -= jv;
                    }
                }
            }
            const int cc = ty * TX + 2 * tx;
            const float2 bx = F2(cC + cc), by = F2(cC + TY * TX + cc), bz = F2(cC + 2 * TY * TX + cc);
            float2 exn, eyn, ezn;
            if (LOSSY) {
                const float2 ax = F2(cC + 3 * TY * TX + cc), ay = F2(cC + 4 * TY * TX + cc),
                             az = F2(cC + 5 * TY * TX + cc);
                exn = make_float2(ax.x * ex.x + bx.x * txA, ax.y * ex.y + bx.y * txB);
                eyn = make_float2(ay.x * ey.x + by.x * tyA, ay.y * ey.y + by.y * tyB);
                ezn = make_float2(az.x * ez.x + bz.x * tzA, az.y * ez.y + bz.y * tzB);
            } else {
                exn = make_float2(ex.x + bx.x * txA, ex.y + bx.y * txB);
                eyn = make_float2(ey.x + by.x * tyA, ey.y + by.y * tyB);
                ezn = make_float2(ez.x + bz.x * tzA, ez.y + bz.y * tzB);
            }
            if (!bad) {
                *reinterpret_cast<float2 *>(out + c) = exn;
                *reinterpret_cast<float2 *>(out + ncell + c) = eyn;
                *reinterpret_cast<float2 *>(out + 2 * ncell + c) = ezn;
            }
            if (EXTRA == kExtraDiff && !bad) {   // keep e^{n+1} - e^n for the adjoint's gradient
                float *d = J.gd;
                *reinterpret_cast<float2 *>(d + c) = make_float2(exn.x - ex.x, exn.y - ex.y);
                *reinterpret_cast<float2 *>(d + ncell + c) = make_float2(eyn.x - ey.x, eyn.y - ey.y);
                *reinterpret_cast<float2 *>(d + 2 * ncell + c) = make_float2(ezn.x - ez.x, ezn.y - ez.y);
            }
            if (EXTRA == kExtraGrad) {   // the input e is the adjoint state mu^{n+1}
                // e^{n+1} - e^n from two states, or (ge0 null) kept by the forward sweep in ge1
                const float2 zero = make_float2(0.f, 0.f);
                const float2 a1 = F2(J.ge1 + c), a0 = J.ge0 ? F2(J.ge0 + c) : zero;
                const float2 b1 = F2(J.ge1 + ncell + c), b0 = J.ge0 ? F2(J.ge0 + ncell + c) : zero;
                const float2 z1 = F2(J.ge1 + 2 * ncell + c), z0 = J.ge0 ? F2(J.ge0 + 2 * ncell + c) : zero;
                float2 *gx = reinterpret_cast<float2 *>(J.gb + c);
                float2 *gy = reinterpret_cast<float2 *>(J.gb + ncell + c);
                float2 *gz = reinterpret_cast<float2 *>(J.gb + 2 * ncell + c);
                float2 vx = *gx, vy = *gy, vz = *gz;
                vx.x += J.gk[0] * (ex.x * (a1.x - a0.x));
                vx.y += J.gk[0] * (ex.y * (a1.y - a0.y));
                vy.x += J.gk[1] * (ey.x * (b1.x - b0.x));
                vy.y += J.gk[1] * (ey.y * (b1.y - b0.y));
                vz.x += J.gk[2] * (ez.x * (z1.x - z0.x));
                vz.y += J.gk[2] * (ez.y * (z1.y - z0.y));
                *gx = vx;
                *gy = vy;
                *gz = vz;
            }
            for (int q = 0; q < nprb_cta; ++q) {
                const EdgeRef r = sm.prb_ref[q];
                if (r.j == j && r.k == k && (r.i == i || r.i == i + 1)) {
                    const bool b = r.i != i;
                    const float2 v = r.axis == 0 ? exn : (r.axis == 1 ? eyn : ezn);
                    J.probe[(J.step - J.probe_base) * J.nprb + sm.prb_idx[q]] = (double)(b ? v.y : v.x);
                }
            }
            if (J.energy) {
                for (int hh = 0; hh < 2; ++hh) {
                    if (hh == 1 && !ownB) break;
                    const long long cq = c + hh;
                    const float me0 = J.meps[cq], me1 = J.meps[ncell + cq], me2 = J.meps[2 * ncell + cq];
                    float m0 = mu0, m1 = mu1, m2 = mu2;
                    if (J.muarr) {
                        m0 = J.mmu[cq];
                        m1 = J.mmu[ncell + cq];
                        m2 = J.mmu[2 * ncell + cq];
                    }
                    const float e0 = hh ? ex.y : ex.x, e1 = hh ? ey.y : ey.x, e2 = hh ? ez.y : ez.x;
                    wacc.add(me0 * e0 * e0);
                    wacc.add(me1 * e1 * e1);
                    wacc.add(me2 * e2 * e2);
                    wacc.add(m0 * (hh ? ho0.y : ho0.x) * (hh ? hxn.y : hxn.x));
                    wacc.add(m1 * (hh ? ho1.y : ho1.x) * (hh ? hyn.y : hyn.x));
                    wacc.add(m2 * (hh ? ho2.y : ho2.x) * (hh ? hzn.y : hzn.x));
                }
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
#undef EV
#undef F2

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

// Single grid, two cells per thread: one CTA = one (member, tile, chunk), member fastest.
template <int TX, int TY, int S, bool LOSSY, int EXTRA = 0>
__global__ void __launch_bounds__(TX / 2 * TY, 4) step_tma2_kernel(const __grid_constant__ StepArgs<float> a,
                                                               const __grid_constant__ CUtensorMap tm_state,
                                                               const __grid_constant__ CUtensorMap tm_coef,
                                                               int muarr, int energy) {
    __shared__ TileSmem2<TX, TY, S> sm;
    unsigned char *dsm = aligned_dsm<float, TX, TY, S>();
    int rest = blockIdx.x;
    const int m = rest % a.nmem;
    rest /= a.nmem;
    const int tile_x = rest % a.tiles_x;
    rest /= a.tiles_x;
    const int tile_y = rest % a.tiles_y;
    const int chunk = rest / a.tiles_y;
    const Member mb = a.mem[m];
    TileJob<float> J;
    J.nx = a.nx; J.ny = a.ny; J.nz = a.nz; J.pitch = a.pitch; J.ncell = a.ncell;
    J.i0 = tile_x * TX;
    J.j0 = tile_y * TY;
    J.k0 = chunk * a.kz;
    J.k1 = min(a.nz, J.k0 + a.kz);
    J.ch = a.ch; J.meps = a.meps; J.mmu = a.mmu; J.muarr = muarr; J.energy = energy;
    J.step = mb.start + a.it;
    J.blk_in = a.parity ? mb.blk[1] : mb.blk[0];
    J.out = static_cast<float *>(a.parity ? mb.st[0] : mb.st[1]);
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
    J.gd = a.gd;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&sm.bar[s], 1);
        mbar_init_fence();
    }
    __syncthreads();
    uint32_t phase = 0;
    tma_tile2<TX, TY, S, LOSSY, EXTRA>(J, &tm_state, &tm_coef, dsm, sm, phase);
}

// Many grids, two cells per thread: the persistent work loop of batched_tma_kernel.
template <int TX, int TY, int S, bool LOSSY>
__global__ void __launch_bounds__(TX / 2 * TY, (TX / 2 * TY == 128 && S == 3) ? 5 : 4) batched_tma2_kernel(const __grid_constant__ BatchArgs<float> b) {
    __shared__ TileSmem2<TX, TY, S> sm;
    unsigned char *dsm = aligned_dsm<float, TX, TY, S>();
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
        const GridDesc<float> &gd = b.grids[w.grid];
        const Member mb = gd.mem[w.member];
        if (mb.start + b.it >= mb.end) continue;   // member finished: nothing to do
        const int tile_x = w.tile % gd.tiles_x;
        const int tile_y = w.tile / gd.tiles_x;
        TileJob<float> J;
        J.nx = gd.nx; J.ny = gd.ny; J.nz = gd.nz; J.pitch = gd.pitch; J.ncell = gd.ncell;
        J.i0 = tile_x * TX;
        J.j0 = tile_y * TY;
        J.k0 = w.chunk * gd.kz;
        J.k1 = min(gd.nz, J.k0 + gd.kz);
        J.ch = gd.ch; J.meps = nullptr; J.mmu = nullptr; J.muarr = gd.muarr; J.energy = 0;
        J.step = mb.start + b.it;
        J.blk_in = b.parity ? mb.blk[1] : mb.blk[0];
        J.out = static_cast<float *>(b.parity ? mb.st[0] : mb.st[1]);
        J.src_on = J.step >= mb.src_lo && J.step < mb.src_hi;
        J.amp = gd.amp; J.amp_base = gd.amp_base; J.nsrc = gd.nsrc; J.src = gd.src;
        J.nprb = gd.nprb; J.prb = gd.prb; J.probe = mb.probe; J.probe_base = mb.probe_base;
        J.energy_out = nullptr;
        J.err = b.err;
        J.wait_limit = 0;
        J.extra_tx = 0;
        J.ge1 = J.ge0 = nullptr;
        J.gb = nullptr;
        J.gk[0] = J.gk[1] = J.gk[2] = 0.f;
        J.gd = nullptr;
        if (!tma_tile2<TX, TY, S, LOSSY>(J, &b.maps[2 * w.grid], &b.maps[2 * w.grid + 1], dsm, sm, phase)) return;
    }
}

template <int TX, int TY, int S, bool LOSSY, int EXTRA = 0>
cudaError_t launch_two(const StepArgs<float> &a, const TmaMaps &maps, bool muarr, bool energy, cudaStream_t s) {
    using G = Geometry<float, TX, TY, S, LOSSY>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(step_tma2_kernel<TX, TY, S, LOSSY, EXTRA>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, G::DYN_SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (a.occ_out)
        return report_occupancy(step_tma2_kernel<TX, TY, S, LOSSY, EXTRA>, TX / 2 * TY, G::DYN_SMEM, a.occ_out);
    const long long blocks = (long long)a.nmem * a.tiles_x * a.tiles_y * a.nchunk;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    step_tma2_kernel<TX, TY, S, LOSSY, EXTRA><<<(unsigned)blocks, TX / 2 * TY, G::DYN_SMEM, s>>>(
        a, maps.state, maps.coef, muarr ? 1 : 0, energy ? 1 : 0);
    return cudaGetLastError();
}

template <int TX, int TY, int S, bool LOSSY>
cudaError_t launch_batched_two(const BatchArgs<float> &b, int ctas, cudaStream_t s) {
    using G = Geometry<float, TX, TY, S, LOSSY>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(batched_tma2_kernel<TX, TY, S, LOSSY>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, G::DYN_SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (b.nitems <= 0) return cudaSuccess;
    const int grid = ctas < b.nitems ? ctas : b.nitems;
    batched_tma2_kernel<TX, TY, S, LOSSY><<<grid, TX / 2 * TY, G::DYN_SMEM, s>>>(b);
    return cudaGetLastError();
}

template <int TX, int TY, int S, bool LOSSY>
int batched_two_occupancy() {
    using G = Geometry<float, TX, TY, S, LOSSY>;
    int n = 0;
    cudaFuncSetAttribute(batched_tma2_kernel<TX, TY, S, LOSSY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         G::DYN_SMEM);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batched_tma2_kernel<TX, TY, S, LOSSY>, TX / 2 * TY,
                                                      G::DYN_SMEM) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

}  // namespace tma
}  // namespace fitgb
