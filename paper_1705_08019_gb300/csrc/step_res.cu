// step_res.cu -- the fused FIT leapfrog step (Sec. II-A of the paper) on FP32
// fields that carry a bfloat16 residual: every stored e and h value is
// hi + lo, hi a float and lo the rounding residual of hi kept to 8
// significant bits.  All arithmetic is FP32.
//
// Where plain FP32 fields lose their accuracy, and what this kernel does
// about each part:
//   * storage: rounding e and h to float after every update is a random
//     walk of half an ulp per value and step.  Here the update is summed
//     into hi with a fast two-sum and the residual is kept, so the stored
//     value is exact to about 2^-33 relative.
//   * the curl C e of the magnetic update: e carries a large curl-free part
//     (the charge a source leaves at its end nodes, and the static field of
//     that charge), whose curl must cancel to zero.  Summing its four terms in
//     float leaves an error of an ulp of the terms, not of the result, every
//     step.  Here each (C e) component is formed as the difference of two
//     same-component differences, both made error-free by two-sums, so the
//     result is accurate to an ulp of the curl itself.
//   * the products with the float coefficients: error-free by one FMA each
//     (two-product), their low parts go into the residual.
// What is left is the rounding of the dual curl C~h, of order an ulp of the
// increment per step (the increment is a small fraction of the field), and
// of the residual's rounding to bfloat16.
//
// Data: a state block has 9 components of 4 bytes: e_x, e_y, e_z, h_x, h_y,
// h_z (hi) and three words of two bfloat16 residuals each, (lo e_x, lo e_y),
// (lo e_z, lo h_x), (lo h_y, lo h_z), the first of each pair in the low 16
// bits.  TMA brings the e, h and residual windows of each plane (aligned
// 4-cell x halo, one row of y halo) and the coefficient tile into an S-deep
// shared-memory ring, completing on one mbarrier per stage, exactly like the
// FP32 kernel.  Algorithmic bytes per cell-update: 72 (6 floats and 3
// residual words, in and out) plus 12 (cb) or 24 (cb, ca); a launch over M
// members of one grid moves 72 M + 24 bytes per cell.  Every mbarrier wait is
// bounded.
#include <cuda_bf16.h>

#include "step_tma.cuh"

namespace fitgb {
namespace res {

using tma::mbar_expect_tx;
using tma::mbar_init;
using tma::mbar_init_fence;
using tma::mbar_wait;
using tma::proxy_fence;
using tma::tma_load_4d;
using tma::tma_load_5d;

// residual words: two bfloat16 in one 32-bit word, the first in the low half
__device__ __forceinline__ float lo_first(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float lo_second(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
__device__ __forceinline__ uint32_t pack_lo(float first, float second) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(first, second);   // .x = first (low half)
    return *reinterpret_cast<const uint32_t *>(&v);
}

// (a - b) - (c - d) for float terms: the two differences are made exact by
// two-sums (Knuth), their difference is rounded once; returns the rounded
// value and the sum of the two residuals
struct Curl {
    float v, r;
};
__device__ __forceinline__ Curl exact_pair_diff(float a, float b, float c, float d) {
    const float d1 = __fsub_rn(a, b);
    const float z1 = __fsub_rn(d1, a);
    const float r1 = __fadd_rn(__fsub_rn(a, __fsub_rn(d1, z1)), __fsub_rn(-b, z1));
    const float d2 = __fsub_rn(c, d);
    const float z2 = __fsub_rn(d2, c);
    const float r2 = __fadd_rn(__fsub_rn(c, __fsub_rn(d2, z2)), __fsub_rn(-d, z2));
    return {__fsub_rn(d1, d2), __fsub_rn(r1, r2)};
}

// hi + lo - c * x, x = the curl in float: the product is split exactly by one
// FMA, the subtraction from hi by a fast two-sum, and the result renormalized
// so that |lo| <= ulp(hi)/2
__device__ __forceinline__ void sub_scaled(float &hi, float &lo, float c, float x) {
    const float p = __fmul_rn(c, x);
    const float pe = __fmaf_rn(c, x, -p);
    const float s = __fsub_rn(hi, p);
    const float t = __fsub_rn(__fsub_rn(hi, s), p);
    const float l = __fsub_rn(__fadd_rn(lo, t), pe);
    hi = __fadd_rn(s, l);
    lo = __fsub_rn(l, __fsub_rn(hi, s));
}

// ca (hi + lo) + cb x (LOSSY) or hi + lo + cb x, renormalized
template <bool LOSSY>
__device__ __forceinline__ void lin_update(float &hi, float &lo, float ca, float cb, float x) {
    float p1 = hi, p1e = lo;
    if (LOSSY) {
        p1 = __fmul_rn(ca, hi);
        p1e = __fmaf_rn(ca, lo, __fmaf_rn(ca, hi, -p1));
    }
    const float p2 = __fmul_rn(cb, x);
    const float p2e = __fmaf_rn(cb, x, -p2);
    const float s = __fadd_rn(p1, p2);
    const float t = __fsub_rn(p2, __fsub_rn(s, p1));
    const float l = __fadd_rn(__fadd_rn(p1e, p2e), t);
    hi = __fadd_rn(s, l);
    lo = __fsub_rn(l, __fsub_rn(hi, s));
}

template <int TX, int TY, int S, bool LOSSY>
struct RGeom {
    static constexpr int NT = TX * TY;
    static constexpr int BX = TX + 8, EY = TY + 2;
    static constexpr int NC = LOSSY ? 6 : 3;
    static constexpr int W_BYTES = 3 * EY * BX * 4;   // one 3-component window
    static constexpr int C_BYTES = NC * TY * TX * 4;
    static constexpr int W_STRIDE = tma::align128(W_BYTES);
    static constexpr int C_OFF = 3 * W_STRIDE;         // e, h, residual words, then coefficients
    static constexpr int STAGE = C_OFF + tma::align128(C_BYTES);
    static constexpr uint32_t TX_BYTES = 3 * W_BYTES + C_BYTES;
    static constexpr int DYN_SMEM = S * STAGE + 128;
};

template <int TX, int TY, int S, bool LOSSY>
__global__ void __launch_bounds__(TX *TY, 3) step_res_kernel(const __grid_constant__ StepArgs<float> a,
                                                          const __grid_constant__ CUtensorMap tm_state,
                                                          const __grid_constant__ CUtensorMap tm_coef, int muarr,
                                                          int energy) {
    using G = RGeom<TX, TY, S, LOSSY>;
    constexpr int NT = G::NT, BX = G::BX, EY = G::EY;
    static_assert(S >= 3, "the e plane k+1 is read while plane k+S is in flight");
    static_assert(TX + TY <= NT, "halo threads");
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
    uint32_t *__restrict__ outw = reinterpret_cast<uint32_t *>(out + 6 * ncell);

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
        mbar_expect_tx(b, G::TX_BYTES + (p == 0 ? (uint32_t)a.extra_tx : 0u));
        tma_load_5d(st, &tm_state, b, i0 - 4, j0 - 1, kk, 0, blk_in);                  // e (hi)
        tma_load_5d(st + G::W_STRIDE, &tm_state, b, i0 - 4, j0 - 1, kk, 3, blk_in);    // h (hi)
        tma_load_5d(st + 2 * G::W_STRIDE, &tm_state, b, i0 - 4, j0 - 1, kk, 6, blk_in);// residual words
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
    float hxp = 0.f, hyp = 0.f, hxpl = 0.f, hypl = 0.f;   // h_x, h_y (hi, lo) at (i, j, k-1), step n+1/2
    double wsum = 0.0;
    uint32_t phase = 0;
    const int limit = a.wait_limit > 0 ? a.wait_limit : tma::kWaitLimit;
    auto wait_plane = [&](int p) -> bool {
        const int st = p % S;
        const bool ok = mbar_wait(&bar[st], (phase >> st) & 1u, limit);
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
        const float *eC = reinterpret_cast<const float *>(stc);
        const float *hC = reinterpret_cast<const float *>(stc + G::W_STRIDE);
        const uint32_t *wC = reinterpret_cast<const uint32_t *>(stc + 2 * G::W_STRIDE);
        const float *cC = reinterpret_cast<const float *>(stc + G::C_OFF);
        const float *eN = reinterpret_cast<const float *>(stn);
        const uint32_t *wN = reinterpret_cast<const uint32_t *>(stn + 2 * G::W_STRIDE);
        if (!bad) {
            if (wait_plane(p + 1)) waited = p + 2;
            else bad = 1;
        }
#define W(buf, comp, y, x) (buf)[((comp) * EY + (y)) * BX + (x)]
        const int sx = lx + 4, sy = ly + 1;
        const long long c = ((long long)k * ny + j) * pitch + i;
        float chl0 = ch[0], chl1 = ch[1], chl2 = ch[2];
        if (muarr) {
            chl0 = own ? a.ch[c] : 0.f;
            chl1 = own ? a.ch[ncell + c] : 0.f;
            chl2 = own ? a.ch[2 * ncell + c] : 0.f;
        }
        // own cell: e, h (hi) and the three residual words
        const float ex0 = W(eC, 0, sy, sx), ey0 = W(eC, 1, sy, sx), ez0 = W(eC, 2, sy, sx);
        const uint32_t w0 = W(wC, 0, sy, sx), w1 = W(wC, 1, sy, sx), w2 = W(wC, 2, sy, sx);
        const float exl = lo_first(w0), eyl = lo_second(w0), ezl = lo_first(w1);
        // neighbours: e at q+x (e_y, e_z), q+y (e_x, e_z), q+z (e_x, e_y)
        const uint32_t wx0 = W(wC, 0, sy, sx + 1), wx1 = W(wC, 1, sy, sx + 1);
        const uint32_t wy0 = W(wC, 0, sy + 1, sx), wy1 = W(wC, 1, sy + 1, sx);
        const uint32_t wz0 = W(wN, 0, sy, sx);
        // (C e)_x = [e_z(q+y) - e_z(q)] - [e_y(q+z) - e_y(q)], and cyclic
        Curl cx = exact_pair_diff(W(eC, 2, sy + 1, sx), ez0, W(eN, 1, sy, sx), ey0);
        Curl cy = exact_pair_diff(W(eN, 0, sy, sx), ex0, W(eC, 2, sy, sx + 1), ez0);
        Curl cz = exact_pair_diff(W(eC, 1, sy, sx + 1), ey0, W(eC, 0, sy + 1, sx), ex0);
        const float lcx = (lo_first(wy1) - ezl) - (lo_second(wz0) - eyl);
        const float lcy = (lo_first(wz0) - exl) - (lo_first(wx1) - ezl);
        const float lcz = (lo_second(wx0) - eyl) - (lo_first(wy0) - exl);
        float hxn = W(hC, 0, sy, sx), hxnl = lo_second(w1);
        float hyn = W(hC, 1, sy, sx), hynl = lo_first(w2);
        float hzn = W(hC, 2, sy, sx), hznl = lo_second(w2);
        sub_scaled(hxn, hxnl, chl0, cx.v + (cx.r + lcx));
        sub_scaled(hyn, hynl, chl1, cy.v + (cy.r + lcy));
        sub_scaled(hzn, hznl, chl2, cz.v + (cz.r + lcz));
        if (!pro) {
            sHh[0][sy][lx + 1] = hxn; sHl[0][sy][lx + 1] = hxnl;
            sHh[1][sy][lx + 1] = hyn; sHl[1][sy][lx + 1] = hynl;
            sHh[2][sy][lx + 1] = hzn; sHl[2][sy][lx + 1] = hznl;
            if (hx_col) {   // cell (i0-1, j0+tid): window x = 3; h_y and h_z
                const int y = tid + 1;
                float c1 = ch[1], c2 = ch[2];
                if (muarr) {
                    const int hi = i0 - 1, hj = j0 + tid;
                    const bool in = hi >= 0 && hj < ny;
                    const long long hc = ((long long)k * ny + hj) * pitch + hi;
                    c1 = in ? a.ch[ncell + hc] : 0.f;
                    c2 = in ? a.ch[2 * ncell + hc] : 0.f;
                }
                const uint32_t v0 = W(wC, 0, y, 3), v1 = W(wC, 1, y, 3), v2 = W(wC, 2, y, 3);
                const uint32_t vx0 = W(wC, 0, y, 4), vx1 = W(wC, 1, y, 4);
                const uint32_t vy0 = W(wC, 0, y + 1, 3), vz0 = W(wN, 0, y, 3);
                const Curl qy = exact_pair_diff(W(eN, 0, y, 3), W(eC, 0, y, 3), W(eC, 2, y, 4), W(eC, 2, y, 3));
                const Curl qz = exact_pair_diff(W(eC, 1, y, 4), W(eC, 1, y, 3), W(eC, 0, y + 1, 3), W(eC, 0, y, 3));
                const float ly_ = (lo_first(vz0) - lo_first(v0)) - (lo_first(vx1) - lo_first(v1));
                const float lz_ = (lo_second(vx0) - lo_second(v0)) - (lo_first(vy0) - lo_first(v0));
                float h1 = W(hC, 1, y, 3), h1l = lo_first(v2);
                float h2 = W(hC, 2, y, 3), h2l = lo_second(v2);
                sub_scaled(h1, h1l, c1, qy.v + (qy.r + ly_));
                sub_scaled(h2, h2l, c2, qz.v + (qz.r + lz_));
                sHh[1][y][0] = h1; sHl[1][y][0] = h1l;
                sHh[2][y][0] = h2; sHl[2][y][0] = h2l;
            } else if (hy_row) {   // cell (i0+t, j0-1): window y = 0; h_x and h_z
                const int t = tid - TY, x = t + 4;
                float c0 = ch[0], c2 = ch[2];
                if (muarr) {
                    const int hi = i0 + t, hj = j0 - 1;
                    const bool in = hj >= 0 && hi < nx;
                    const long long hc = ((long long)k * ny + hj) * pitch + hi;
                    c0 = in ? a.ch[hc] : 0.f;
                    c2 = in ? a.ch[2 * ncell + hc] : 0.f;
                }
                const uint32_t v0 = W(wC, 0, 0, x), v1 = W(wC, 1, 0, x), v2 = W(wC, 2, 0, x);
                const uint32_t vx0 = W(wC, 0, 0, x + 1);
                const uint32_t vy0 = W(wC, 0, 1, x), vy1 = W(wC, 1, 1, x), vz0 = W(wN, 0, 0, x);
                const Curl qx = exact_pair_diff(W(eC, 2, 1, x), W(eC, 2, 0, x), W(eN, 1, 0, x), W(eC, 1, 0, x));
                const Curl qz = exact_pair_diff(W(eC, 1, 0, x + 1), W(eC, 1, 0, x), W(eC, 0, 1, x), W(eC, 0, 0, x));
                const float lx_ = (lo_first(vy1) - lo_first(v1)) - (lo_second(vz0) - lo_second(v0));
                const float lz_ = (lo_second(vx0) - lo_second(v0)) - (lo_first(vy0) - lo_first(v0));
                float h0 = W(hC, 0, 0, x), h0l = lo_second(v1);
                float h2 = W(hC, 2, 0, x), h2l = lo_second(v2);
                sub_scaled(h0, h0l, c0, qx.v + (qx.r + lx_));
                sub_scaled(h2, h2l, c2, qz.v + (qz.r + lz_));
                sHh[0][0][t + 1] = h0; sHl[0][0][t + 1] = h0l;
                sHh[2][0][t + 1] = h2; sHl[2][0][t + 1] = h2l;
            }
            if (own && !bad) {
                out[3 * ncell + c] = hxn;
                out[4 * ncell + c] = hyn;
                out[5 * ncell + c] = hzn;
            }
        }
        if (__syncthreads_or(bad)) {   // (B) h plane complete
            aborted = true;
            break;
        }
        if (!pro && own) {
            const int sxh = lx + 1;
            // (C~h)_x = [h_z(q) - h_z(q-y)] - [h_y(q) - h_y(q-z)], and cyclic; residuals likewise
            float tx = (hzn - sHh[2][sy - 1][sxh]) - (hyn - hyp);
            float ty = (hxn - hxp) - (hzn - sHh[2][sy][sxh - 1]);
            float tz = (hyn - sHh[1][sy][sxh - 1]) - (hxn - sHh[0][sy - 1][sxh]);
            tx += (hznl - sHl[2][sy - 1][sxh]) - (hynl - hypl);
            ty += (hxnl - hxpl) - (hznl - sHl[2][sy][sxh - 1]);
            tz += (hynl - sHl[1][sy][sxh - 1]) - (hxnl - sHl[0][sy - 1][sxh]);
            for (int q = 0; q < sNsrc; ++q) {
                const EdgeRef r = sSrcRef[q];
                if (r.i == i && r.j == j && r.k == k) {
                    const double jd = a.amp[(step - a.amp_base) * a.nsrc + sSrc[q]];
                    const float jh = (float)jd;
                    const float jl = (float)(jd - (double)jh);
                    if (r.axis == 0) tx = (tx - jh) - jl;
                    else if (r.axis == 1) ty = (ty - jh) - jl;
                    else tz = (tz - jh) - jl;
                }
            }
            const int cc = ly * TX + lx;
            const float bx = cC[cc], by = cC[TY * TX + cc], bz = cC[2 * TY * TX + cc];
            float ax_ = 1.f, ay_ = 1.f, az_ = 1.f;
            if (LOSSY) {
                ax_ = cC[3 * TY * TX + cc];
                ay_ = cC[4 * TY * TX + cc];
                az_ = cC[5 * TY * TX + cc];
            }
            float exn = ex0, exnl = exl, eyn = ey0, eynl = eyl, ezn = ez0, eznl = ezl;
            lin_update<LOSSY>(exn, exnl, ax_, bx, tx);
            lin_update<LOSSY>(eyn, eynl, ay_, by, ty);
            lin_update<LOSSY>(ezn, eznl, az_, bz, tz);
            if (!bad) {
                out[c] = exn;
                out[ncell + c] = eyn;
                out[2 * ncell + c] = ezn;
                outw[c] = pack_lo(exnl, eynl);
                outw[ncell + c] = pack_lo(eznl, hxnl);
                outw[2 * ncell + c] = pack_lo(hynl, hznl);
            }
            for (int q = 0; q < sNprb; ++q) {
                const EdgeRef r = sPrbRef[q];
                if (r.i == i && r.j == j && r.k == k) {
                    const float vh = r.axis == 0 ? exn : (r.axis == 1 ? eyn : ezn);
                    const float vl = r.axis == 0 ? exnl : (r.axis == 1 ? eynl : eznl);
                    // the stored value: hi plus the residual as kept (bfloat16)
                    const float vs = __bfloat162float(__float2bfloat16_rn(vl));
                    mb.probe[(step - mb.probe_base) * a.nprb + sPrb[q]] = (double)vh + (double)vs;
                }
            }
            if (energy) {
                const double dex = (double)ex0 + exl, dey = (double)ey0 + eyl, dez = (double)ez0 + ezl;
                const double h0x = (double)W(hC, 0, sy, sx) + lo_second(w1);
                const double h0y = (double)W(hC, 1, sy, sx) + lo_first(w2);
                const double h0z = (double)W(hC, 2, sy, sx) + lo_second(w2);
                double mu0, mu1, mu2;
                if (muarr) {
                    mu0 = a.mmu[c]; mu1 = a.mmu[ncell + c]; mu2 = a.mmu[2 * ncell + c];
                } else {
                    mu0 = a.mmu[0]; mu1 = a.mmu[1]; mu2 = a.mmu[2];
                }
                wsum += (double)a.meps[c] * dex * dex + (double)a.meps[ncell + c] * dey * dey +
                        (double)a.meps[2 * ncell + c] * dez * dez + mu0 * h0x * ((double)hxn + hxnl) +
                        mu1 * h0y * ((double)hyn + hynl) + mu2 * h0z * ((double)hzn + hznl);
            }
        }
#undef W
        hxp = hxn;
        hyp = hyn;
        hxpl = hxnl;
        hypl = hynl;
        __syncthreads();   // (C) stage p and the h plane are free again
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

// Two cells per thread: thread (t, y) owns the x-adjacent cells A = (i0+2t, j)
// and B = A + u_x, so shared-memory and global accesses are 8 bytes wide, B's
// low-x neighbour is A itself and A's high-x neighbour is B.  The low-y halo
// row is computed by the first TX/2 threads (pairs), the low-x halo column by
// the last TY threads (single cells).
template <int TX, int TY, int S, bool LOSSY>
__global__ void __launch_bounds__(TX / 2 * TY, 3) step_res2_kernel(const __grid_constant__ StepArgs<float> a,
                                                               const __grid_constant__ CUtensorMap tm_state,
                                                               const __grid_constant__ CUtensorMap tm_coef,
                                                               int muarr, int energy) {
    using G = RGeom<TX, TY, S, LOSSY>;
    constexpr int BX = G::BX, EY = G::EY, HX = TX + 2;
    constexpr int PX = TX / 2, NT = PX * TY;
    static_assert(S >= 3, "the e plane k+1 is read while plane k+S is in flight");
    static_assert(TX % 2 == 0 && PX + TY <= NT, "pairs and halo threads");
    extern __shared__ __align__(128) unsigned char dsm_raw[];
    unsigned char *dsm = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(dsm_raw) + 127) &
                                                           ~static_cast<uintptr_t>(127));
    __shared__ __align__(8) uint64_t bar[S];
    // h^{n+1/2} of plane k (hi, lo): row 0 = low-y halo row, column 1 = low-x
    // halo column, cell x at column x + 2 (pairs 8-byte aligned)
    __shared__ __align__(16) float sHh[3][TY + 1][HX];
    __shared__ __align__(16) float sHl[3][TY + 1][HX];
    __shared__ EdgeRef sSrcRef[kMaxSrc], sPrbRef[kMaxPrb];
    __shared__ int sSrc[kMaxSrc], sPrb[kMaxPrb];
    __shared__ int sNsrc, sNprb;
    __shared__ double sRed[NT / 32 + 1];

    const int tid = threadIdx.x;
    const int tx = tid % PX, ty = tid / PX;
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
    const int i = i0 + 2 * tx, j = j0 + ty;
    const bool ownA = (i < nx) && (j < ny), ownB = (i + 1 < nx) && (j < ny);
    const int k0 = chunk * a.kz;
    const int k1 = min(nz, k0 + a.kz);
    const int kstart = (k0 > 0) ? k0 - 1 : k0;
    const int total = k1 - kstart + 1;
    const Member mb = a.mem[m];
    const long long step = mb.start + a.it;
    const int blk_in = a.parity ? mb.blk[1] : mb.blk[0];
    float *__restrict__ out = static_cast<float *>(a.parity ? mb.st[0] : mb.st[1]);
    uint32_t *__restrict__ outw = reinterpret_cast<uint32_t *>(out + 6 * ncell);

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
    const int nsrc_cta = sNsrc, nprb_cta = sNprb;

    auto issue = [&](int p) {
        const int kk = kstart + p;
        unsigned char *st = dsm + (p % S) * G::STAGE;
        uint64_t *b = &bar[p % S];
        mbar_expect_tx(b, G::TX_BYTES + (p == 0 ? (uint32_t)a.extra_tx : 0u));
        tma_load_5d(st, &tm_state, b, i0 - 4, j0 - 1, kk, 0, blk_in);                   // e (hi)
        tma_load_5d(st + G::W_STRIDE, &tm_state, b, i0 - 4, j0 - 1, kk, 3, blk_in);     // h (hi)
        tma_load_5d(st + 2 * G::W_STRIDE, &tm_state, b, i0 - 4, j0 - 1, kk, 6, blk_in); // residual words
        tma_load_4d(st + G::C_OFF, &tm_coef, b, i0, j0, kk, 0);
    };
    int issued = 0;
    if (tid == 0) {
        proxy_fence();
        for (; issued < min(S, total); ++issued) issue(issued);
    }
    float ch0 = 0.f, ch1 = 0.f, ch2 = 0.f;
    if (!muarr) {
        ch0 = a.ch[0];
        ch1 = a.ch[1];
        ch2 = a.ch[2];
    }
    const bool hy_row = tid < PX;                   // low-y halo row, pair tid
    // low-x halo column: the last TY threads, cell tid - (NT - TY) (another warp than the
    // halo row's whenever the tile has more than one warp, so no warp runs both branches)
    const bool hx_col = tid >= NT - TY;
    float2 hxp = make_float2(0.f, 0.f), hyp = hxp, hxpl = hxp, hypl = hxp;   // h_x, h_y of plane k-1
    double wsum = 0.0;
    uint32_t phase = 0;
    const int limit = a.wait_limit > 0 ? a.wait_limit : tma::kWaitLimit;
    auto wait_plane = [&](int p) -> bool {
        const int st = p % S;
        const bool ok = mbar_wait(&bar[st], (phase >> st) & 1u, limit);
        if (ok) phase ^= (1u << st);
        return ok;
    };
    int bad = wait_plane(0) ? 0 : 1;
    int waited = bad ? 0 : 1;
    bool aborted = false;
    const int sx = 4 + 2 * tx, sy = ty + 1, hx = 2 * tx + 2;

#define W(buf, comp, y, x) (buf)[((comp) * EY + (y)) * BX + (x)]
#define F2(ptr) (*reinterpret_cast<const float2 *>(ptr))
#define U2(ptr) (*reinterpret_cast<const uint2 *>(ptr))
    for (int k = kstart; k < k1; ++k) {
        const int p = k - kstart;
        const bool pro = k < k0;
        const unsigned char *stc = dsm + (p % S) * G::STAGE;
        const unsigned char *stn = dsm + ((p + 1) % S) * G::STAGE;
        const float *eC = reinterpret_cast<const float *>(stc);
        const float *hC = reinterpret_cast<const float *>(stc + G::W_STRIDE);
        const uint32_t *wC = reinterpret_cast<const uint32_t *>(stc + 2 * G::W_STRIDE);
        const float *cC = reinterpret_cast<const float *>(stc + G::C_OFF);
        const float *eN = reinterpret_cast<const float *>(stn);
        const uint32_t *wN = reinterpret_cast<const uint32_t *>(stn + 2 * G::W_STRIDE);
        if (!bad) {
            if (wait_plane(p + 1)) waited = p + 2;
            else bad = 1;
        }
        const long long c = ((long long)k * ny + j) * pitch + i;
        float2 cA = make_float2(ch0, ch0), cB = make_float2(ch1, ch1), cZ = make_float2(ch2, ch2);
        if (muarr) {
            cA = ownA ? F2(a.ch + c) : make_float2(0.f, 0.f);
            cB = ownA ? F2(a.ch + ncell + c) : make_float2(0.f, 0.f);
            cZ = ownA ? F2(a.ch + 2 * ncell + c) : make_float2(0.f, 0.f);
        }
        // e^n (hi) of the pair and its neighbours
        const float2 ex = F2(&W(eC, 0, sy, sx)), ey = F2(&W(eC, 1, sy, sx)), ez = F2(&W(eC, 2, sy, sx));
        const float eyx = W(eC, 1, sy, sx + 2), ezx = W(eC, 2, sy, sx + 2);
        const float2 exy = F2(&W(eC, 0, sy + 1, sx)), ezy = F2(&W(eC, 2, sy + 1, sx));
        const float2 exz = F2(&W(eN, 0, sy, sx)), eyz = F2(&W(eN, 1, sy, sx));
        // residual words: own (e_x,e_y | e_z,h_x | h_y,h_z), q+x, q+y, q+z
        const uint2 w0 = U2(&W(wC, 0, sy, sx)), w1 = U2(&W(wC, 1, sy, sx)), w2 = U2(&W(wC, 2, sy, sx));
        const uint32_t w0x = W(wC, 0, sy, sx + 2), w1x = W(wC, 1, sy, sx + 2);
        const uint2 w0y = U2(&W(wC, 0, sy + 1, sx)), w1y = U2(&W(wC, 1, sy + 1, sx));
        const uint2 w0z = U2(&W(wN, 0, sy, sx));
        const float exlA = lo_first(w0.x), exlB = lo_first(w0.y);
        const float eylA = lo_second(w0.x), eylB = lo_second(w0.y);
        const float ezlA = lo_first(w1.x), ezlB = lo_first(w1.y);
        // (C e)_x = [e_z(q+y) - e_z(q)] - [e_y(q+z) - e_y(q)]
        // (C e)_y = [e_x(q+z) - e_x(q)] - [e_z(q+x) - e_z(q)]
        // (C e)_z = [e_y(q+x) - e_y(q)] - [e_x(q+y) - e_x(q)]
        const Curl cxA = exact_pair_diff(ezy.x, ez.x, eyz.x, ey.x);
        const Curl cyA = exact_pair_diff(exz.x, ex.x, ez.y, ez.x);
        const Curl czA = exact_pair_diff(ey.y, ey.x, exy.x, ex.x);
        const Curl cxB = exact_pair_diff(ezy.y, ez.y, eyz.y, ey.y);
        const Curl cyB = exact_pair_diff(exz.y, ex.y, ezx, ez.y);
        const Curl czB = exact_pair_diff(eyx, ey.y, exy.y, ex.y);
        const float lcxA = (lo_first(w1y.x) - ezlA) - (lo_second(w0z.x) - eylA);
        const float lcyA = (lo_first(w0z.x) - exlA) - (ezlB - ezlA);
        const float lczA = (eylB - eylA) - (lo_first(w0y.x) - exlA);
        const float lcxB = (lo_first(w1y.y) - ezlB) - (lo_second(w0z.y) - eylB);
        const float lcyB = (lo_first(w0z.y) - exlB) - (lo_first(w1x) - ezlB);
        const float lczB = (lo_second(w0x) - eylB) - (lo_first(w0y.y) - exlB);
        const float2 hxo = F2(&W(hC, 0, sy, sx)), hyo = F2(&W(hC, 1, sy, sx)), hzo = F2(&W(hC, 2, sy, sx));
        float2 hxn = hxo, hyn = hyo, hzn = hzo;
        float2 hxnl = make_float2(lo_second(w1.x), lo_second(w1.y));
        float2 hynl = make_float2(lo_first(w2.x), lo_first(w2.y));
        float2 hznl = make_float2(lo_second(w2.x), lo_second(w2.y));
        sub_scaled(hxn.x, hxnl.x, cA.x, cxA.v + (cxA.r + lcxA));
        sub_scaled(hyn.x, hynl.x, cB.x, cyA.v + (cyA.r + lcyA));
        sub_scaled(hzn.x, hznl.x, cZ.x, czA.v + (czA.r + lczA));
        sub_scaled(hxn.y, hxnl.y, cA.y, cxB.v + (cxB.r + lcxB));
        sub_scaled(hyn.y, hynl.y, cB.y, cyB.v + (cyB.r + lcyB));
        sub_scaled(hzn.y, hznl.y, cZ.y, czB.v + (czB.r + lczB));
        if (!pro) {
            *reinterpret_cast<float2 *>(&sHh[0][sy][hx]) = hxn;
            *reinterpret_cast<float2 *>(&sHh[1][sy][hx]) = hyn;
            *reinterpret_cast<float2 *>(&sHh[2][sy][hx]) = hzn;
            *reinterpret_cast<float2 *>(&sHl[0][sy][hx]) = hxnl;
            *reinterpret_cast<float2 *>(&sHl[1][sy][hx]) = hynl;
            *reinterpret_cast<float2 *>(&sHl[2][sy][hx]) = hznl;
            if (hy_row) {   // cells (i0+2t, j0-1), (i0+2t+1, j0-1): window y = 0; h_x and h_z
                const int t = tid, x = 4 + 2 * t;
                float2 c0 = make_float2(ch0, ch0), c2 = make_float2(ch2, ch2);
                if (muarr) {
                    const bool in = j0 >= 1 && i0 + 2 * t < nx;
                    const long long hc = ((long long)k * ny + (j0 - 1)) * pitch + (i0 + 2 * t);
                    c0 = in ? F2(a.ch + hc) : make_float2(0.f, 0.f);
                    c2 = in ? F2(a.ch + 2 * ncell + hc) : make_float2(0.f, 0.f);
                }
                const float2 ez0 = F2(&W(eC, 2, 0, x)), ez1 = F2(&W(eC, 2, 1, x));
                const float2 ey0 = F2(&W(eC, 1, 0, x)), eyN = F2(&W(eN, 1, 0, x));
                const float ey0x = W(eC, 1, 0, x + 2);
                const float2 ex0 = F2(&W(eC, 0, 0, x)), ex1 = F2(&W(eC, 0, 1, x));
                const uint2 v0 = U2(&W(wC, 0, 0, x)), v1 = U2(&W(wC, 1, 0, x)), v2 = U2(&W(wC, 2, 0, x));
                const uint2 v0y = U2(&W(wC, 0, 1, x)), v1y = U2(&W(wC, 1, 1, x)), v0z = U2(&W(wN, 0, 0, x));
                const uint32_t v0x = W(wC, 0, 0, x + 2);
                const Curl qxA = exact_pair_diff(ez1.x, ez0.x, eyN.x, ey0.x);
                const Curl qzA = exact_pair_diff(ey0.y, ey0.x, ex1.x, ex0.x);
                const Curl qxB = exact_pair_diff(ez1.y, ez0.y, eyN.y, ey0.y);
                const Curl qzB = exact_pair_diff(ey0x, ey0.y, ex1.y, ex0.y);
                const float lxA = (lo_first(v1y.x) - lo_first(v1.x)) - (lo_second(v0z.x) - lo_second(v0.x));
                const float lzA = (lo_second(v0.y) - lo_second(v0.x)) - (lo_first(v0y.x) - lo_first(v0.x));
                const float lxB = (lo_first(v1y.y) - lo_first(v1.y)) - (lo_second(v0z.y) - lo_second(v0.y));
                const float lzB = (lo_second(v0x) - lo_second(v0.y)) - (lo_first(v0y.y) - lo_first(v0.y));
                float2 h0 = F2(&W(hC, 0, 0, x)), h2 = F2(&W(hC, 2, 0, x));
                float2 h0l = make_float2(lo_second(v1.x), lo_second(v1.y));
                float2 h2l = make_float2(lo_second(v2.x), lo_second(v2.y));
                sub_scaled(h0.x, h0l.x, c0.x, qxA.v + (qxA.r + lxA));
                sub_scaled(h2.x, h2l.x, c2.x, qzA.v + (qzA.r + lzA));
                sub_scaled(h0.y, h0l.y, c0.y, qxB.v + (qxB.r + lxB));
                sub_scaled(h2.y, h2l.y, c2.y, qzB.v + (qzB.r + lzB));
                *reinterpret_cast<float2 *>(&sHh[0][0][2 * t + 2]) = h0;
                *reinterpret_cast<float2 *>(&sHl[0][0][2 * t + 2]) = h0l;
                *reinterpret_cast<float2 *>(&sHh[2][0][2 * t + 2]) = h2;
                *reinterpret_cast<float2 *>(&sHl[2][0][2 * t + 2]) = h2l;
            } else if (hx_col) {   // cell (i0-1, j0+y-1): window x = 3; h_y and h_z
                const int y = tid - (NT - TY) + 1;
                float c1 = ch1, c2 = ch2;
                if (muarr) {
                    const int hi = i0 - 1, hj = j0 + y - 1;
                    const bool in = hi >= 0 && hj < ny;
                    const long long hc = ((long long)k * ny + hj) * pitch + hi;
                    c1 = in ? a.ch[ncell + hc] : 0.f;
                    c2 = in ? a.ch[2 * ncell + hc] : 0.f;
                }
                const uint32_t v0 = W(wC, 0, y, 3), v1 = W(wC, 1, y, 3), v2 = W(wC, 2, y, 3);
                const uint32_t vx0 = W(wC, 0, y, 4), vx1 = W(wC, 1, y, 4);
                const uint32_t vy0 = W(wC, 0, y + 1, 3), vz0 = W(wN, 0, y, 3);
                const Curl qy = exact_pair_diff(W(eN, 0, y, 3), W(eC, 0, y, 3), W(eC, 2, y, 4), W(eC, 2, y, 3));
                const Curl qz = exact_pair_diff(W(eC, 1, y, 4), W(eC, 1, y, 3), W(eC, 0, y + 1, 3), W(eC, 0, y, 3));
                const float ly_ = (lo_first(vz0) - lo_first(v0)) - (lo_first(vx1) - lo_first(v1));
                const float lz_ = (lo_second(vx0) - lo_second(v0)) - (lo_first(vy0) - lo_first(v0));
                float h1 = W(hC, 1, y, 3), h1l = lo_first(v2);
                float h2 = W(hC, 2, y, 3), h2l = lo_second(v2);
                sub_scaled(h1, h1l, c1, qy.v + (qy.r + ly_));
                sub_scaled(h2, h2l, c2, qz.v + (qz.r + lz_));
                sHh[1][y][1] = h1; sHl[1][y][1] = h1l;
                sHh[2][y][1] = h2; sHl[2][y][1] = h2l;
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
            // (C~h)_x = [h_z(q) - h_z(q-y)] - [h_y(q) - h_y(q-z)]
            // (C~h)_y = [h_x(q) - h_x(q-z)] - [h_z(q) - h_z(q-x)]
            // (C~h)_z = [h_y(q) - h_y(q-x)] - [h_x(q) - h_x(q-y)]
            const float2 hzmy = F2(&sHh[2][sy - 1][hx]), hzmyl = F2(&sHl[2][sy - 1][hx]);
            const float2 hxmy = F2(&sHh[0][sy - 1][hx]), hxmyl = F2(&sHl[0][sy - 1][hx]);
            const float hzmx = sHh[2][sy][hx - 1], hzmxl = sHl[2][sy][hx - 1];
            const float hymx = sHh[1][sy][hx - 1], hymxl = sHl[1][sy][hx - 1];
            float txA = ((hzn.x - hzmy.x) - (hyn.x - hyp.x)) + ((hznl.x - hzmyl.x) - (hynl.x - hypl.x));
            float tyA = ((hxn.x - hxp.x) - (hzn.x - hzmx)) + ((hxnl.x - hxpl.x) - (hznl.x - hzmxl));
            float tzA = ((hyn.x - hymx) - (hxn.x - hxmy.x)) + ((hynl.x - hymxl) - (hxnl.x - hxmyl.x));
            float txB = ((hzn.y - hzmy.y) - (hyn.y - hyp.y)) + ((hznl.y - hzmyl.y) - (hynl.y - hypl.y));
            float tyB = ((hxn.y - hxp.y) - (hzn.y - hzn.x)) + ((hxnl.y - hxpl.y) - (hznl.y - hznl.x));
            float tzB = ((hyn.y - hyn.x) - (hxn.y - hxmy.y)) + ((hynl.y - hynl.x) - (hxnl.y - hxmyl.y));
            for (int q = 0; q < nsrc_cta; ++q) {
                const EdgeRef r = sSrcRef[q];
                if (r.j == j && r.k == k && (r.i == i || r.i == i + 1)) {
                    const double jd = a.amp[(step - a.amp_base) * a.nsrc + sSrc[q]];
                    const float jh = (float)jd;
                    const float jl = (float)(jd - (double)jh);
                    const bool b = r.i != i;
                    if (r.axis == 0) {
                        if (b) txB = (txB - jh) - jl; else txA = (txA - jh) - jl;
                    } else if (r.axis == 1) {
                        if (b) tyB = (tyB - jh) - jl; else tyA = (tyA - jh) - jl;
                    } else {
                        if (b) tzB = (tzB - jh) - jl; else tzA = (tzA - jh) - jl;
                    }
                }
            }
            const int cc = ty * TX + 2 * tx;
            const float2 bx = F2(cC + cc), by = F2(cC + TY * TX + cc), bz = F2(cC + 2 * TY * TX + cc);
            float2 ax_ = make_float2(1.f, 1.f), ay_ = ax_, az_ = ax_;
            if (LOSSY) {
                ax_ = F2(cC + 3 * TY * TX + cc);
                ay_ = F2(cC + 4 * TY * TX + cc);
                az_ = F2(cC + 5 * TY * TX + cc);
            }
            float2 exn = ex, eyn = ey, ezn = ez;
            float2 exnl = make_float2(exlA, exlB), eynl = make_float2(eylA, eylB), eznl = make_float2(ezlA, ezlB);
            lin_update<LOSSY>(exn.x, exnl.x, ax_.x, bx.x, txA);
            lin_update<LOSSY>(eyn.x, eynl.x, ay_.x, by.x, tyA);
            lin_update<LOSSY>(ezn.x, eznl.x, az_.x, bz.x, tzA);
            lin_update<LOSSY>(exn.y, exnl.y, ax_.y, bx.y, txB);
            lin_update<LOSSY>(eyn.y, eynl.y, ay_.y, by.y, tyB);
            lin_update<LOSSY>(ezn.y, eznl.y, az_.y, bz.y, tzB);
            if (!bad) {
                *reinterpret_cast<float2 *>(out + c) = exn;
                *reinterpret_cast<float2 *>(out + ncell + c) = eyn;
                *reinterpret_cast<float2 *>(out + 2 * ncell + c) = ezn;
                *reinterpret_cast<uint2 *>(outw + c) = make_uint2(pack_lo(exnl.x, eynl.x), pack_lo(exnl.y, eynl.y));
                *reinterpret_cast<uint2 *>(outw + ncell + c) =
                    make_uint2(pack_lo(eznl.x, hxnl.x), pack_lo(eznl.y, hxnl.y));
                *reinterpret_cast<uint2 *>(outw + 2 * ncell + c) =
                    make_uint2(pack_lo(hynl.x, hznl.x), pack_lo(hynl.y, hznl.y));
            }
            for (int q = 0; q < nprb_cta; ++q) {
                const EdgeRef r = sPrbRef[q];
                if (r.j == j && r.k == k && (r.i == i || r.i == i + 1)) {
                    const bool b = r.i != i;
                    const float2 vh = r.axis == 0 ? exn : (r.axis == 1 ? eyn : ezn);
                    const float2 vl = r.axis == 0 ? exnl : (r.axis == 1 ? eynl : eznl);
                    // the stored value: hi plus the residual as kept (bfloat16)
                    const float vs = __bfloat162float(__float2bfloat16_rn(b ? vl.y : vl.x));
                    mb.probe[(step - mb.probe_base) * a.nprb + sPrb[q]] = (double)(b ? vh.y : vh.x) + (double)vs;
                }
            }
            if (energy) {
                double mu0, mu1, mu2;
                for (int h = 0; h < 2; ++h) {
                    if (h == 1 && !ownB) break;
                    const long long cq = c + h;
                    if (muarr) {
                        mu0 = a.mmu[cq]; mu1 = a.mmu[ncell + cq]; mu2 = a.mmu[2 * ncell + cq];
                    } else {
                        mu0 = a.mmu[0]; mu1 = a.mmu[1]; mu2 = a.mmu[2];
                    }
                    const uint32_t u0 = h ? w0.y : w0.x, u1 = h ? w1.y : w1.x, u2 = h ? w2.y : w2.x;
                    const double dex = (double)(h ? ex.y : ex.x) + lo_first(u0);
                    const double dey = (double)(h ? ey.y : ey.x) + lo_second(u0);
                    const double dez = (double)(h ? ez.y : ez.x) + lo_first(u1);
                    const double h0x = (double)(h ? hxo.y : hxo.x) + lo_second(u1);
                    const double h0y = (double)(h ? hyo.y : hyo.x) + lo_first(u2);
                    const double h0z = (double)(h ? hzo.y : hzo.x) + lo_second(u2);
                    const double h1x = (double)(h ? hxn.y : hxn.x) + (h ? hxnl.y : hxnl.x);
                    const double h1y = (double)(h ? hyn.y : hyn.x) + (h ? hynl.y : hynl.x);
                    const double h1z = (double)(h ? hzn.y : hzn.x) + (h ? hznl.y : hznl.x);
                    wsum += (double)a.meps[cq] * dex * dex + (double)a.meps[ncell + cq] * dey * dey +
                            (double)a.meps[2 * ncell + cq] * dez * dez + mu0 * h0x * h1x + mu1 * h0y * h1y +
                            mu2 * h0z * h1z;
                }
            }
        }
        hxp = hxn;
        hyp = hyn;
        hxpl = hxnl;
        hypl = hynl;
        __syncthreads();   // (C) stage p and the h plane are free again
        if (tid == 0 && issued < total) {
            proxy_fence();
            issue(issued);
            ++issued;
        }
    }
#undef W
#undef F2
#undef U2
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
cudaError_t launch2(const StepArgs<float> &a, const TmaMaps &maps, bool muarr, bool energy, cudaStream_t s) {
    using G = RGeom<TX, TY, S, LOSSY>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(step_res2_kernel<TX, TY, S, LOSSY>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, G::DYN_SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (a.occ_out) return report_occupancy(step_res2_kernel<TX, TY, S, LOSSY>, TX / 2 * TY, G::DYN_SMEM, a.occ_out);
    const long long blocks = (long long)a.nmem * a.tiles_x * a.tiles_y * a.nchunk;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    step_res2_kernel<TX, TY, S, LOSSY><<<(unsigned)blocks, TX / 2 * TY, G::DYN_SMEM, s>>>(
        a, maps.state, maps.coef, muarr ? 1 : 0, energy ? 1 : 0);
    return cudaGetLastError();
}

template <int TX, int TY, int S, bool LOSSY>
cudaError_t launch(const StepArgs<float> &a, const TmaMaps &maps, bool muarr, bool energy, cudaStream_t s) {
    using G = RGeom<TX, TY, S, LOSSY>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(step_res_kernel<TX, TY, S, LOSSY>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, G::DYN_SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (a.occ_out) return report_occupancy(step_res_kernel<TX, TY, S, LOSSY>, TX * TY, G::DYN_SMEM, a.occ_out);
    const long long blocks = (long long)a.nmem * a.tiles_x * a.tiles_y * a.nchunk;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    step_res_kernel<TX, TY, S, LOSSY><<<(unsigned)blocks, TX * TY, G::DYN_SMEM, s>>>(a, maps.state, maps.coef,
                                                                                   muarr ? 1 : 0, energy ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace res

bool res_tile_supported(int tx, int ty) { return (tx == 32 && (ty == 4 || ty == 8)) || (tx == 64 && ty == 4); }

cudaError_t launch_step_res(const StepArgs<float> &a, const TmaMaps &maps, Tile t, bool lossy, bool muarr,
                            bool energy, cudaStream_t s) {
    // two cells per thread unless one cell per thread (opts kernel 3) is asked for
    if (!t.single) {
#define FIT_R2(TX, TY, S)                                                               \
        if (t.tx == TX && t.ty == TY)                                                   \
            return lossy ? res::launch2<TX, TY, S, true>(a, maps, muarr, energy, s)     \
                         : res::launch2<TX, TY, S, false>(a, maps, muarr, energy, s);
        FIT_R2(64, 4, 3)
        FIT_R2(32, 8, 3)
#undef FIT_R2
    }
#define FIT_R(TX, TY, S)                                                                \
    if (t.tx == TX && t.ty == TY)                                                       \
        return lossy ? res::launch<TX, TY, S, true>(a, maps, muarr, energy, s)          \
                     : res::launch<TX, TY, S, false>(a, maps, muarr, energy, s);
    FIT_R(64, 4, 3)
    FIT_R(32, 8, 3)
    FIT_R(32, 4, 4)
#undef FIT_R
    return cudaErrorInvalidValue;
}

}  // namespace fitgb

// ---- conversions between the ABI's FP64 compact fields and the residual format ----
namespace fitgb {
namespace {

constexpr int kCvtThreads = 256;

inline unsigned cvt_grid(long long n) {
    long long b = (n + kCvtThreads - 1) / kCvtThreads;
    if (b > 152LL * 64) b = 152LL * 64;
    return (unsigned)(b > 0 ? b : 1);
}

// e (compact, 3 components) and h -> hi floats and residual words of the
// padded layout; entries that are not degrees of freedom become zero
__global__ void split_res_kernel(int nx, int ny, int nz, int pitch, const double *e, const double *h, float *hi,
                                 uint32_t *w) {
    const long long ncell = (long long)nx * ny * nz, ncp = (long long)pitch * ny * nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
         c += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(c % nx);
        const int j = (int)((c / nx) % ny);
        const int k = (int)(c / ((long long)nx * ny));
        const int q[3] = {i, j, k};
        const long long o = ((long long)k * ny + j) * pitch + i;
        float lo[6];
        for (int a = 0; a < 6; ++a) {
            const bool is_h = a >= 3;
            const int b = a % 3;
            const bool dof = is_h ? q[b] > 0 : (q[(b + 1) % 3] > 0 && q[(b + 2) % 3] > 0);
            const double *src = is_h ? h : e;
            const double v = (dof && src) ? src[(long long)b * ncell + c] : 0.0;
            const float vh = (float)v;
            hi[(long long)a * ncp + o] = vh;
            lo[a] = (float)(v - (double)vh);
        }
        w[o] = res::pack_lo(lo[0], lo[1]);
        w[ncp + o] = res::pack_lo(lo[2], lo[3]);
        w[2 * ncp + o] = res::pack_lo(lo[4], lo[5]);
    }
}

// value of component a (0..5: e_x..h_z) at padded index o
__device__ __forceinline__ double res_value(const float *hi, const uint32_t *w, long long ncp, int a, long long o) {
    const uint32_t word = w[(long long)(a / 2) * ncp + o];
    const float lo = (a & 1) ? res::lo_second(word) : res::lo_first(word);
    return (double)hi[(long long)a * ncp + o] + (double)lo;
}

__global__ void join_res_kernel(int nx, int ny, int nz, int pitch, const float *hi, const uint32_t *w, int part,
                                double *out) {
    const long long ncell = (long long)nx * ny * nz, ncp = (long long)pitch * ny * nz;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < 3 * ncell;
         t += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(t / ncell);
        const long long c = t % ncell;
        const int i = (int)(c % nx);
        const int j = (int)((c / nx) % ny);
        const int k = (int)(c / ((long long)nx * ny));
        out[t] = res_value(hi, w, ncp, 3 * part + b, ((long long)k * ny + j) * pitch + i);
    }
}

__global__ void accumulate_res_kernel(long long ncp, const float *hi, const uint32_t *w, int part, double *acc) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < 3 * ncp;
         t += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(t / ncp);
        acc[t] += res_value(hi, w, ncp, 3 * part + b, t % ncp);
    }
}

}  // namespace

cudaError_t split_res(int nx, int ny, int nz, int pitch, const double *e, const double *h, float *state,
                      cudaStream_t s) {
    const long long ncp = (long long)pitch * ny * nz;
    split_res_kernel<<<cvt_grid((long long)nx * ny * nz), kCvtThreads, 0, s>>>(
        nx, ny, nz, pitch, e, h, state, reinterpret_cast<uint32_t *>(state + 6 * ncp));
    return cudaGetLastError();
}

cudaError_t join_res(int nx, int ny, int nz, int pitch, const float *state, int part, double *out, cudaStream_t s) {
    const long long ncp = (long long)pitch * ny * nz;
    join_res_kernel<<<cvt_grid(3LL * nx * ny * nz), kCvtThreads, 0, s>>>(
        nx, ny, nz, pitch, state, reinterpret_cast<const uint32_t *>(state + 6 * ncp), part, out);
    return cudaGetLastError();
}

cudaError_t accumulate_res(long long ncp, const float *state, int part, double *acc, cudaStream_t s) {
    accumulate_res_kernel<<<cvt_grid(3 * ncp), kCvtThreads, 0, s>>>(
        ncp, state, reinterpret_cast<const uint32_t *>(state + 6 * ncp), part, acc);
    return cudaGetLastError();
}

}  // namespace fitgb
