// step_comp.cu -- the fused FIT leapfrog step (Sec. II-A of the paper) with
// compensated FP32 fields: every e and h value is an unevaluated sum hi + lo
// of two floats (about 48 significant bits), and every update is carried out
// in FP32 arithmetic with error-free transformations:
//   two_sum(a, b)  -> s + r = a + b exactly        (Knuth)
//   two_prod(a, b) -> p + r = a * b exactly        (one FMA)
// The curls are summed term by term with two_sum, so the small difference
// C~h - j near a driven edge (where C~h nearly cancels the impressed current)
// keeps its relative accuracy; products with the float coefficients are
// exact up to the lo part; the result is renormalized with two_sum.  Plain
// FP32 fields lose that accuracy in the storage of h itself.  The rounding
// that remains is of the order of 2^-48 per value and step.
//
// Data: a state block has 12 components, e_hi, h_hi, e_lo, h_lo (3 each);
// TMA brings the four e/h windows and the coefficient tile of each plane into
// the stage ring exactly as in the FP32 kernel (step_tma.cuh), and the h plane
// in shared memory holds hi and lo.  Bytes per cell-update: 96 (fields in and
// out) + 12 (cb) or 24 (cb, ca).
#include "step_tma.cuh"

namespace fitgb {
namespace comp {

using tma::mbar_expect_tx;
using tma::mbar_init;
using tma::mbar_init_fence;
using tma::mbar_wait;
using tma::proxy_fence;
using tma::tma_load_4d;
using tma::tma_load_5d;

struct FF {   // hi + lo
    float h, l;
};

__device__ __forceinline__ FF two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ FF two_prod(float a, float b) {
    const float p = a * b;
    return {p, __fmaf_rn(a, b, -p)};
}

// a + b - c - d for float-float operands, summed exactly then renormalized
__device__ __forceinline__ FF sum4(FF a, FF b, FF c, FF d) {
    const FF s1 = two_sum(a.h, b.h);
    const FF s2 = two_sum(s1.h, -c.h);
    const FF s3 = two_sum(s2.h, -d.h);
    const float lo = ((s1.l + s2.l) + s3.l) + (((a.l + b.l) - c.l) - d.l);
    return two_sum(s3.h, lo);
}

// x - c * y (c a float coefficient)
__device__ __forceinline__ FF sub_scaled(FF x, float c, FF y) {
    const FF p = two_prod(c, y.h);
    const float pl = __fmaf_rn(c, y.l, p.l);
    const FF t = two_sum(x.h, -p.h);
    const float tl = (x.l - pl) + t.l;
    return two_sum(t.h, tl);
}

// a * x + b * y (a, b float coefficients)
__device__ __forceinline__ FF lin2(float a, FF x, float b, FF y) {
    const FF p = two_prod(a, x.h);
    const float pl = __fmaf_rn(a, x.l, p.l);
    const FF q = two_prod(b, y.h);
    const float ql = __fmaf_rn(b, y.l, q.l);
    const FF t = two_sum(p.h, q.h);
    const float tl = (pl + ql) + t.l;
    return two_sum(t.h, tl);
}

// x + b * y
__device__ __forceinline__ FF add_scaled(FF x, float b, FF y) {
    const FF q = two_prod(b, y.h);
    const float ql = __fmaf_rn(b, y.l, q.l);
    const FF t = two_sum(x.h, q.h);
    const float tl = (x.l + ql) + t.l;
    return two_sum(t.h, tl);
}

template <int TX, int TY, int S, bool LOSSY>
struct CGeom {
    static constexpr int NT = TX * TY;
    static constexpr int BX = TX + 8, EY = TY + 2;
    static constexpr int NC = LOSSY ? 6 : 3;
    static constexpr int W_BYTES = 3 * EY * BX * 4;     // one 3-component window
    static constexpr int C_BYTES = NC * TY * TX * 4;
    static constexpr int W_STRIDE = tma::align128(W_BYTES);
    static constexpr int C_OFF = 4 * W_STRIDE;           // e_hi, h_hi, e_lo, h_lo, then coefficients
    static constexpr int STAGE = C_OFF + tma::align128(C_BYTES);
    static constexpr uint32_t TX_BYTES = 4 * W_BYTES + C_BYTES;
    static constexpr int DYN_SMEM = S * STAGE + 128;
};

template <int TX, int TY, int S, bool LOSSY>
__global__ void __launch_bounds__(TX *TY) step_comp_kernel(const __grid_constant__ StepArgs<float> a,
                                                           const __grid_constant__ CUtensorMap tm_state,
                                                           const __grid_constant__ CUtensorMap tm_coef, int muarr,
                                                           int energy) {
    using G = CGeom<TX, TY, S, LOSSY>;
    constexpr int NT = G::NT, BX = G::BX, EY = G::EY;
    static_assert(S >= 3, "the e plane k+1 is read while plane k+S is in flight");
    extern __shared__ __align__(128) unsigned char dsm_raw[];
    unsigned char *dsm = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(dsm_raw) + 127) &
                                                           ~static_cast<uintptr_t>(127));
    __shared__ __align__(8) uint64_t bar[S];
    __shared__ float sHh[3][TY + 1][TX + 1], sHl[3][TY + 1][TX + 1];
    __shared__ EdgeRef sSrcRef[kMaxSrc], sPrbRef[kMaxPrb];
    __shared__ int sSrc[kMaxSrc], sPrb[kMaxPrb];
    __shared__ int sNsrc, sNprb;
    __shared__ double sRed[NT / 32];

    const int tid = threadIdx.x;
    const int lx = tid % TX, ly = tid / TX;
    int rest = blockIdx.x;
    const int m = rest % a.nmem;
    rest /= a.nmem;
    const int tile_x = rest % a.tiles_x;
    rest /= a.tiles_x;
    const int tile_y = rest % a.tiles_y;
    const int chunk = rest / a.tiles_y;
    const int nx = a.nx, ny = a.ny, nz = a.nz, pitch = a.pitch;
    const long long ncell = a.ncell;
    const int i0 = tile_x * TX, j0 = tile_y * TY;
    const int i = i0 + lx, j = j0 + ly;
    const bool own = (i < nx) && (j < ny);
    const int k0 = chunk * a.kz;
    const int k1 = min(nz, k0 + a.kz);
    const int kstart = (k0 > 0) ? k0 - 1 : k0;
    const int total = k1 - kstart + 1;
    const Member mb = a.mem[m];
    const long long step = mb.start + a.it;
    const int blk_in = a.parity ? mb.blk[1] : mb.blk[0];
    float *__restrict__ out = static_cast<float *>(a.parity ? mb.st[0] : mb.st[1]);

    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
        mbar_init_fence();
        int ns = 0, np = 0;
        const bool on = step >= mb.src_lo && step < mb.src_hi;
        for (int s = 0; s < a.nsrc && on; ++s) {
            const EdgeRef r = a.src[s];
            if (r.i >= i0 && r.i < i0 + TX && r.j >= j0 && r.j < j0 + TY && r.k >= k0 && r.k < k1) {
                sSrc[ns] = s;
                sSrcRef[ns] = r;
                ++ns;
            }
        }
        for (int p = 0; p < a.nprb && mb.probe; ++p) {
            const EdgeRef r = a.prb[p];
            if (r.i >= i0 && r.i < i0 + TX && r.j >= j0 && r.j < j0 + TY && r.k >= k0 && r.k < k1) {
                sPrb[np] = p;
                sPrbRef[np] = r;
                ++np;
            }
        }
        sNsrc = ns;
        sNprb = np;
    }
    __syncthreads();

    auto issue = [&](int p) {
        const int kk = kstart + p;
        unsigned char *st = dsm + (p % S) * G::STAGE;
        uint64_t *b = &bar[p % S];
        mbar_expect_tx(b, G::TX_BYTES);
        tma_load_5d(st, &tm_state, b, i0 - 4, j0 - 1, kk, 0, blk_in);                    // e_hi
        tma_load_5d(st + G::W_STRIDE, &tm_state, b, i0 - 4, j0 - 1, kk, 3, blk_in);      // h_hi
        tma_load_5d(st + 2 * G::W_STRIDE, &tm_state, b, i0 - 4, j0 - 1, kk, 6, blk_in);  // e_lo
        tma_load_5d(st + 3 * G::W_STRIDE, &tm_state, b, i0 - 4, j0 - 1, kk, 9, blk_in);  // h_lo
        tma_load_4d(st + G::C_OFF, &tm_coef, b, i0, j0, kk, 0);
    };
    int issued = 0;
    if (tid == 0) {
        proxy_fence();
        for (; issued < min(S, total); ++issued) issue(issued);
    }
    float ch[3] = {0.f, 0.f, 0.f};
    if (!muarr) {
        ch[0] = a.ch[0];
        ch[1] = a.ch[1];
        ch[2] = a.ch[2];
    }
    const bool hx_col = tid < TY;
    const bool hy_row = tid >= TY && tid < TY + TX;
    FF hxp = {0.f, 0.f}, hyp = {0.f, 0.f};
    double wsum = 0.0;
    uint32_t phase = 0;
    auto wait_plane = [&](int p) -> bool {
        const int st = p % S;
        const bool ok = mbar_wait(&bar[st], (phase >> st) & 1u);
        if (ok) phase ^= (1u << st);
        return ok;
    };
    int bad = wait_plane(0) ? 0 : 1;
    int waited = bad ? 0 : 1;
    bool aborted = false;

    for (int k = kstart; k < k1; ++k) {
        const int p = k - kstart;
        const bool pro = k < k0;
        const unsigned char *stc = dsm + (p % S) * G::STAGE;
        const unsigned char *stn = dsm + ((p + 1) % S) * G::STAGE;
        const float *eCh = reinterpret_cast<const float *>(stc);
        const float *hCh = reinterpret_cast<const float *>(stc + G::W_STRIDE);
        const float *eCl = reinterpret_cast<const float *>(stc + 2 * G::W_STRIDE);
        const float *hCl = reinterpret_cast<const float *>(stc + 3 * G::W_STRIDE);
        const float *cC = reinterpret_cast<const float *>(stc + G::C_OFF);
        const float *eNh = reinterpret_cast<const float *>(stn);
        const float *eNl = reinterpret_cast<const float *>(stn + 2 * G::W_STRIDE);
        if (!bad) {
            if (wait_plane(p + 1)) waited = p + 2;
            else bad = 1;
        }
#define W(buf, comp, y, x) (buf)[((comp) * EY + (y)) * BX + (x)]
#define EC(comp, y, x) FF{W(eCh, comp, y, x), W(eCl, comp, y, x)}
#define EN(comp, y, x) FF{W(eNh, comp, y, x), W(eNl, comp, y, x)}
#define HC(comp, y, x) FF{W(hCh, comp, y, x), W(hCl, comp, y, x)}
        const int sx = lx + 4, sy = ly + 1;
        const long long c = ((long long)k * ny + j) * pitch + i;
        float chl0 = ch[0], chl1 = ch[1], chl2 = ch[2];
        if (muarr) {
            chl0 = own ? a.ch[c] : 0.f;
            chl1 = own ? a.ch[ncell + c] : 0.f;
            chl2 = own ? a.ch[2 * ncell + c] : 0.f;
        }
        const FF ex0 = EC(0, sy, sx), ey0 = EC(1, sy, sx), ez0 = EC(2, sy, sx);
        const FF ho0 = HC(0, sy, sx), ho1 = HC(1, sy, sx), ho2 = HC(2, sy, sx);
        // (C e)_x = e_y(q) + e_z(q+y) - e_y(q+z) - e_z(q), and cyclic
        const FF cx = sum4(ey0, EC(2, sy + 1, sx), EN(1, sy, sx), ez0);
        const FF cy = sum4(ez0, EN(0, sy, sx), EC(2, sy, sx + 1), ex0);
        const FF cz = sum4(ex0, EC(1, sy, sx + 1), EC(0, sy + 1, sx), ey0);
        const FF hxn = sub_scaled(ho0, chl0, cx);
        const FF hyn = sub_scaled(ho1, chl1, cy);
        const FF hzn = sub_scaled(ho2, chl2, cz);
        if (!pro) {
            sHh[0][sy][lx + 1] = hxn.h; sHl[0][sy][lx + 1] = hxn.l;
            sHh[1][sy][lx + 1] = hyn.h; sHl[1][sy][lx + 1] = hyn.l;
            sHh[2][sy][lx + 1] = hzn.h; sHl[2][sy][lx + 1] = hzn.l;
            if (hx_col) {   // cell (i0-1, j0+tid): window x = 3
                const int y = tid + 1;
                float c1 = ch[1], c2 = ch[2];
                if (muarr) {
                    const int hi = i0 - 1, hj = j0 + tid;
                    const bool in = hi >= 0 && hj < ny;
                    const long long hc = ((long long)k * ny + hj) * pitch + hi;
                    c1 = in ? a.ch[ncell + hc] : 0.f;
                    c2 = in ? a.ch[2 * ncell + hc] : 0.f;
                }
                const FF cyh = sum4(EC(2, y, 3), EN(0, y, 3), EC(2, y, 4), EC(0, y, 3));
                const FF czh = sum4(EC(0, y, 3), EC(1, y, 4), EC(0, y + 1, 3), EC(1, y, 3));
                const FF v1 = sub_scaled(HC(1, y, 3), c1, cyh);
                const FF v2 = sub_scaled(HC(2, y, 3), c2, czh);
                sHh[1][y][0] = v1.h; sHl[1][y][0] = v1.l;
                sHh[2][y][0] = v2.h; sHl[2][y][0] = v2.l;
            } else if (hy_row) {   // cell (i0+t, j0-1): window y = 0
                const int t = tid - TY, x = t + 4;
                float c0 = ch[0], c2 = ch[2];
                if (muarr) {
                    const int hi = i0 + t, hj = j0 - 1;
                    const bool in = hj >= 0 && hi < nx;
                    const long long hc = ((long long)k * ny + hj) * pitch + hi;
                    c0 = in ? a.ch[hc] : 0.f;
                    c2 = in ? a.ch[2 * ncell + hc] : 0.f;
                }
                const FF cxh = sum4(EC(1, 0, x), EC(2, 1, x), EN(1, 0, x), EC(2, 0, x));
                const FF czh = sum4(EC(0, 0, x), EC(1, 0, x + 1), EC(0, 1, x), EC(1, 0, x));
                const FF v0 = sub_scaled(HC(0, 0, x), c0, cxh);
                const FF v2 = sub_scaled(HC(2, 0, x), c2, czh);
                sHh[0][0][t + 1] = v0.h; sHl[0][0][t + 1] = v0.l;
                sHh[2][0][t + 1] = v2.h; sHl[2][0][t + 1] = v2.l;
            }
            if (own) {
                out[3 * ncell + c] = hxn.h; out[9 * ncell + c] = hxn.l;
                out[4 * ncell + c] = hyn.h; out[10 * ncell + c] = hyn.l;
                out[5 * ncell + c] = hzn.h; out[11 * ncell + c] = hzn.l;
            }
        }
#undef W
#undef EC
#undef EN
#undef HC
        if (__syncthreads_or(bad)) {
            aborted = true;
            break;
        }
        if (!pro && own) {
            const int sxh = lx + 1;
#define SH(comp, y, x) FF{sHh[comp][y][x], sHl[comp][y][x]}
            // (C~h)_x = h_z(q) - h_z(q-y) - h_y(q) + h_y(q-z), written as a + b - c - d
            FF tx = sum4(hzn, hyp, SH(2, sy - 1, sxh), hyn);
            // (C~h)_y = h_x(q) - h_x(q-z) - h_z(q) + h_z(q-x)
            FF ty = sum4(hxn, SH(2, sy, sxh - 1), hxp, hzn);
            // (C~h)_z = h_y(q) - h_y(q-x) - h_x(q) + h_x(q-y)
            FF tz = sum4(hyn, SH(0, sy - 1, sxh), SH(1, sy, sxh - 1), hxn);
#undef SH
            for (int q = 0; q < sNsrc; ++q) {
                const EdgeRef r = sSrcRef[q];
                if (r.i == i && r.j == j && r.k == k) {
                    const double jd = a.amp[(step - a.amp_base) * a.nsrc + sSrc[q]];
                    const float jh = (float)jd;
                    const float jl = (float)(jd - (double)jh);
                    FF &t = r.axis == 0 ? tx : (r.axis == 1 ? ty : tz);
                    const FF s = two_sum(t.h, -jh);
                    t = two_sum(s.h, (t.l - jl) + s.l);
                }
            }
            const int cc = ly * TX + lx;
            const float bx = cC[cc], by = cC[TY * TX + cc], bz = cC[2 * TY * TX + cc];
            FF exn, eyn, ezn;
            if (LOSSY) {
                exn = lin2(cC[3 * TY * TX + cc], ex0, bx, tx);
                eyn = lin2(cC[4 * TY * TX + cc], ey0, by, ty);
                ezn = lin2(cC[5 * TY * TX + cc], ez0, bz, tz);
            } else {
                exn = add_scaled(ex0, bx, tx);
                eyn = add_scaled(ey0, by, ty);
                ezn = add_scaled(ez0, bz, tz);
            }
            out[c] = exn.h; out[6 * ncell + c] = exn.l;
            out[ncell + c] = eyn.h; out[7 * ncell + c] = eyn.l;
            out[2 * ncell + c] = ezn.h; out[8 * ncell + c] = ezn.l;
            for (int q = 0; q < sNprb; ++q) {
                const EdgeRef r = sPrbRef[q];
                if (r.i == i && r.j == j && r.k == k) {
                    const FF v = r.axis == 0 ? exn : (r.axis == 1 ? eyn : ezn);
                    mb.probe[(step - mb.probe_base) * a.nprb + sPrb[q]] = (double)v.h + (double)v.l;
                }
            }
            if (energy) {
                auto d = [](FF v) { return (double)v.h + (double)v.l; };
                double mu0, mu1, mu2;
                if (muarr) {
                    mu0 = a.mmu[c]; mu1 = a.mmu[ncell + c]; mu2 = a.mmu[2 * ncell + c];
                } else {
                    mu0 = a.mmu[0]; mu1 = a.mmu[1]; mu2 = a.mmu[2];
                }
                wsum += (double)a.meps[c] * d(ex0) * d(ex0) + (double)a.meps[ncell + c] * d(ey0) * d(ey0) +
                        (double)a.meps[2 * ncell + c] * d(ez0) * d(ez0) + mu0 * d(ho0) * d(hxn) +
                        mu1 * d(ho1) * d(hyn) + mu2 * d(ho2) * d(hzn);
            }
        }
        hxp = hxn;
        hyp = hyn;
        __syncthreads();
        if (tid == 0 && issued < total) {
            proxy_fence();
            issue(issued);
            ++issued;
        }
    }
    if (aborted) {
        if (tid == 0) {
            atomicOr(a.err, kErrTimeout);
            for (int p = waited; p < issued; ++p) wait_plane(p);
        }
        return;
    }
    if (energy) {
        double v = wsum;
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

template <int TX, int TY, int S, bool LOSSY>
cudaError_t launch(const StepArgs<float> &a, const TmaMaps &maps, bool muarr, bool energy, cudaStream_t s) {
    using G = CGeom<TX, TY, S, LOSSY>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(step_comp_kernel<TX, TY, S, LOSSY>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, G::DYN_SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (a.occ_out) return report_occupancy(step_comp_kernel<TX, TY, S, LOSSY>, TX * TY, G::DYN_SMEM, a.occ_out);
    const long long blocks = (long long)a.nmem * a.tiles_x * a.tiles_y * a.nchunk;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    step_comp_kernel<TX, TY, S, LOSSY><<<(unsigned)blocks, TX * TY, G::DYN_SMEM, s>>>(a, maps.state, maps.coef,
                                                                                    muarr ? 1 : 0, energy ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace comp

bool comp_tile_supported(int tx, int ty) { return tx == 32 && (ty == 4 || ty == 8); }

cudaError_t launch_step_comp(const StepArgs<float> &a, const TmaMaps &maps, Tile t, bool lossy, bool muarr,
                             bool energy, cudaStream_t s) {
    if (t.tx == 32 && t.ty == 8)
        return lossy ? comp::launch<32, 8, 3, true>(a, maps, muarr, energy, s)
                     : comp::launch<32, 8, 3, false>(a, maps, muarr, energy, s);
    if (t.tx == 32 && t.ty == 4)
        return lossy ? comp::launch<32, 4, 4, true>(a, maps, muarr, energy, s)
                     : comp::launch<32, 4, 4, false>(a, maps, muarr, energy, s);
    return cudaErrorInvalidValue;
}

}  // namespace fitgb
