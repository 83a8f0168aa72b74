// expo_tma.cu -- one fused pair of the Leja / Taylor Newton recurrence with a
// TMA pipeline (the GB300 path of the exponential propagators; the two-launch
// version in expo.cu stays for the init step and the synchronisation):
//     y  = X r,   r' = X y + eta_j^2 r,   p += alpha_j r + gamma_j y,
// X (e, h) = kappa (cb (.) C~h, -ch (.) C e).  y never reaches HBM: per cell
// and pair r is read once, p read and written once, r' written once.
//
// The two curls chain in opposite directions: y_h = -kappa ch C r_e looks at
// higher neighbours and feeds r'_e = kappa cb C~ y_h, which looks at lower
// ones; y_e = kappa cb C~ r_h looks at lower neighbours and feeds
// r'_h = -kappa ch C y_e, which looks at higher ones.  One CTA owns a TX x TY
// column of one member and streams it along z; at iteration k it has the r
// planes k and k+1 (window x in [i0-4, i0+TX+4), y in [j0-1, j0+TY+1), by
// TMA, out-of-grid cells zero) and the cb windows of the same planes, and
//   (a) computes y_h of plane k on the tile and its low-x column / low-y row,
//   (b) computes y_e of plane k+1 on the tile and its high-x column / high-y
//       row (cb of the halo cells comes with the window),
//   (c) finishes plane k: r'_e from y_h of planes k and k-1, r'_h from y_e of
//       planes k and k+1, and the p update.
// The plane-k values of y_h and y_e sit in shared memory; y_h of plane k-1
// and y_e of plane k+1 are needed only at the thread's own cell and stay in
// registers (y_e of plane k+1 is stored at the start of the next iteration).
// The first iteration (plane k0-1, zeros below the grid) only primes them.  Waits are bounded as in the
// leapfrog kernel: on timeout the CTA records kErrTimeout, waits (bounded)
// for its own copies and returns.
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

template <typename T, int TX, int TY, int S>
struct PairGeom {
    static constexpr int BX = TX + 8, EY = TY + 2;
    static constexpr int W_BYTES = 3 * EY * BX * (int)sizeof(T);   // one 3-component window
    static constexpr int H_OFF = tma::align128(W_BYTES);
    static constexpr int C_OFF = H_OFF + tma::align128(W_BYTES);
    static constexpr int STAGE = C_OFF + tma::align128(W_BYTES);
    static constexpr uint32_t TX_BYTES = 3 * W_BYTES;
    static constexpr int DYN_SMEM = S * STAGE + 128;
};

template <typename T, int TX, int TY, int S>
struct PairSmem {
    uint64_t bar[S];
    T yh[3][TY + 1][TX + 1];   // y_h of plane k; index 0 = low halo
    T ye[3][TY + 1][TX + 1];   // y_e of plane k; index TY / TX = high halo
};

template <typename T, int TX, int TY, int S, bool LAST, bool MUARR>
__global__ void __launch_bounds__(TX *TY, 4) expo_pair_tma_kernel(const __grid_constant__ ExpoArgs<T> a,
                                                               const __grid_constant__ CUtensorMap tm_r,
                                                               const __grid_constant__ CUtensorMap tm_cb,
                                                               int tiles_x, int tiles_y, int wait_limit) {
    using G = PairGeom<T, TX, TY, S>;
    constexpr int BX = G::BX, EY = G::EY;
    __shared__ PairSmem<T, TX, TY, S> sm;
    unsigned char *dsm = tma::aligned_dsm<T, TX, TY, S>();
    int rest = blockIdx.x;
    const int mem = rest % a.nmem;
    rest /= a.nmem;
    const int tx_ = rest % tiles_x;
    rest /= tiles_x;
    const int ty_ = rest % tiles_y;
    const int chunk = rest / tiles_y;
    const ExpoMember<T> M = a.mem[mem];
    const int tid = threadIdx.x, lx = tid % TX, ly = tid / TX;
    const int nx = a.nx, ny = a.ny, pitch = a.pitch;
    const long long n = a.ncp;
    const int i0 = tx_ * TX, j0 = ty_ * TY, i = i0 + lx, j = j0 + ly;
    const int k0 = chunk * a.kz, k1 = min(a.nz, k0 + a.kz);
    const bool own = i < nx && j < ny;
    // ping-pong: odd pairs read R and write Y, even pairs the reverse
    const bool odd = (a.pair & 1) != 0;
    const int blk_in = M.blk + (odd ? 1 : 2);
    T *__restrict__ rout = odd ? M.Y : M.R;
    T *__restrict__ P = M.P;
    const T *__restrict__ chp = a.ch;
    const T kap = (T)a.kappa, eta2 = (T)a.eta2;
    T al_e, ga_e, al_h, ga_h;
    if (a.substep == M.nsub - 1) {
        const double *f = M.fin + 4 * (a.pair - 1);
        al_e = (T)f[0]; ga_e = (T)f[1]; al_h = (T)f[2]; ga_h = (T)f[3];
    } else {
        al_e = al_h = (T)a.reg[2 * (a.pair - 1)];
        ga_e = ga_h = (T)a.reg[2 * (a.pair - 1) + 1];
    }
    T chs[3] = {T(0), T(0), T(0)};
    if (!MUARR) {
        chs[0] = __ldg(chp);
        chs[1] = __ldg(chp + 1);
        chs[2] = __ldg(chp + 2);
    }

    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&sm.bar[s], 1);
        mbar_init_fence();
    }
    __syncthreads();
    const int kstart = k0 - 1;             // plane k0-1 primes the y rings (zeros below the grid)
    const int total = k1 - kstart + 1;     // planes kstart .. k1
    auto issue = [&](int p) {
        const int kk = kstart + p;
        unsigned char *st = dsm + (p % S) * G::STAGE;
        uint64_t *b = &sm.bar[p % S];
        mbar_expect_tx(b, G::TX_BYTES + (p == 0 ? (uint32_t)a.extra_tx : 0u));
        tma_load_5d(st, &tm_r, b, i0 - 4, j0 - 1, kk, 0, blk_in);
        tma_load_5d(st + G::H_OFF, &tm_r, b, i0 - 4, j0 - 1, kk, 3, blk_in);
        tma_load_4d(st + G::C_OFF, &tm_cb, b, i0 - 4, j0 - 1, kk, 0);
    };
    const int limit = wait_limit > 0 ? wait_limit : tma::kWaitLimit;
    uint32_t phase = 0;
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
    int bad = wait_plane(0) ? 0 : 1;
    int waited = bad ? 0 : 1;
    bool aborted = false;
    // halo roles: y_h low column / row, y_e high column / row
    const bool lo_col = tid < TY, lo_row = tid >= TY && tid < TY + TX;
    const bool hi_col = tid >= TY + TX && tid < 2 * TY + TX, hi_row = tid >= 2 * TY + TX && tid < 2 * TY + 2 * TX;
    // carried along z: y_h of plane k-1 (x, y) and y_e of plane k+1 at this cell, and the
    // two y_e components of this thread's high-halo cell
    T yhp_x = T(0), yhp_y = T(0), ye_n0 = T(0), ye_n1 = T(0), ye_n2 = T(0), pend_a = T(0), pend_b = T(0);

#define RV(buf, comp, y, x) (buf)[((comp) * EY + (y)) * BX + (x)]
    for (int k = kstart; k < k1; ++k) {
        const int p = k - kstart;
        const T *eC = reinterpret_cast<const T *>(dsm + (p % S) * G::STAGE);
        const T *hC = reinterpret_cast<const T *>(dsm + (p % S) * G::STAGE + G::H_OFF);
        const T *bC = reinterpret_cast<const T *>(dsm + (p % S) * G::STAGE + G::C_OFF);
        const T *eN = reinterpret_cast<const T *>(dsm + ((p + 1) % S) * G::STAGE);
        const T *hN = reinterpret_cast<const T *>(dsm + ((p + 1) % S) * G::STAGE + G::H_OFF);
        const T *bN = reinterpret_cast<const T *>(dsm + ((p + 1) % S) * G::STAGE + G::C_OFF);
        if (!bad) {
            if (wait_plane(p + 1)) waited = p + 2;
            else bad = 1;
        }
        const int sx = lx + 4, sy = ly + 1;
        const long long c = ((long long)k * ny + j) * pitch + i;
        // y_e of plane k, computed in the previous iteration, into the shared plane
        sm.ye[0][ly][lx] = ye_n0;
        sm.ye[1][ly][lx] = ye_n1;
        sm.ye[2][ly][lx] = ye_n2;
        if (hi_col) {
            const int t = tid - TY - TX;
            sm.ye[1][t][TX] = pend_a;
            sm.ye[2][t][TX] = pend_b;
        } else if (hi_row) {
            const int t = tid - 2 * TY - TX;
            sm.ye[0][TY][t] = pend_a;
            sm.ye[2][TY][t] = pend_b;
        }
        // p of plane k: issue the loads early, used after the barrier
        T p0 = T(0), p1 = T(0), p2 = T(0), p3 = T(0), p4 = T(0), p5 = T(0);
        if (k >= k0 && own) {
            p0 = P[c]; p1 = P[n + c]; p2 = P[2 * n + c];
            p3 = P[3 * n + c]; p4 = P[4 * n + c]; p5 = P[5 * n + c];
        }
        // (a) y_h of plane k at (x, y) of the window: -kap ch (C r_e)
        auto yh_at = [&](int x, int y, T c0, T c1, T c2, T &o0, T &o1, T &o2) {
            const T ex = RV(eC, 0, y, x), ey = RV(eC, 1, y, x), ez = RV(eC, 2, y, x);
            const T cx = (ey + RV(eC, 2, y + 1, x)) - (RV(eN, 1, y, x) + ez);
            const T cy = (ez + RV(eN, 0, y, x)) - (RV(eC, 2, y, x + 1) + ex);
            const T cz = (ex + RV(eC, 1, y, x + 1)) - (RV(eC, 0, y + 1, x) + ey);
            o0 = -kap * (c0 * cx);
            o1 = -kap * (c1 * cy);
            o2 = -kap * (c2 * cz);
        };
        auto ch_at = [&](int ci, int cj, int comp) -> T {
            if (!MUARR) return chs[comp];
            if (ci < 0 || cj < 0 || ci >= nx || cj >= ny || k < 0) return T(0);
            return __ldg(chp + comp * n + ((long long)k * ny + cj) * pitch + ci);
        };
        T yhx, yhy, yhz;   // y_h of plane k at this cell
        yh_at(sx, sy, ch_at(i, j, 0), ch_at(i, j, 1), ch_at(i, j, 2), yhx, yhy, yhz);
        sm.yh[0][ly + 1][lx + 1] = yhx;
        sm.yh[1][ly + 1][lx + 1] = yhy;
        sm.yh[2][ly + 1][lx + 1] = yhz;
        {
            T o0, o1, o2;
            if (lo_col) {   // cell (i0-1, j0+tid): y_h y and z
                const int y = tid + 1;
                yh_at(3, y, T(0), ch_at(i0 - 1, j0 + tid, 1), ch_at(i0 - 1, j0 + tid, 2), o0, o1, o2);
                sm.yh[1][y][0] = o1;
                sm.yh[2][y][0] = o2;
            } else if (lo_row) {   // cell (i0+t, j0-1): y_h x and z
                const int t = tid - TY;
                yh_at(t + 4, 0, ch_at(i0 + t, j0 - 1, 0), T(0), ch_at(i0 + t, j0 - 1, 2), o0, o1, o2);
                sm.yh[0][0][t + 1] = o0;
                sm.yh[2][0][t + 1] = o2;
            }
        }
        // (b) y_e of plane k+1 at (x, y): kap cb (C~ r_h), r_h of planes k+1 and k; kept in
        // registers until the next iteration stores it
        auto ye_at = [&](int x, int y, T &o0, T &o1, T &o2) {
            const T hx = RV(hN, 0, y, x), hy = RV(hN, 1, y, x), hz = RV(hN, 2, y, x);
            const T tx = (hz - RV(hN, 2, y - 1, x)) - (hy - RV(hC, 1, y, x));
            const T ty = (hx - RV(hC, 0, y, x)) - (hz - RV(hN, 2, y, x - 1));
            const T tz = (hy - RV(hN, 1, y, x - 1)) - (hx - RV(hN, 0, y - 1, x));
            o0 = kap * (RV(bN, 0, y, x) * tx);
            o1 = kap * (RV(bN, 1, y, x) * ty);
            o2 = kap * (RV(bN, 2, y, x) * tz);
        };
        const T yex = ye_n0, yey = ye_n1, yez = ye_n2;   // y_e of plane k at this cell
        ye_at(sx, sy, ye_n0, ye_n1, ye_n2);
        {
            T o0, o1, o2;
            if (hi_col) {   // cell (i0+TX, j0+t): y_e y and z
                const int t = tid - TY - TX;
                ye_at(TX + 4, t + 1, o0, o1, o2);
                pend_a = o1;
                pend_b = o2;
            } else if (hi_row) {   // cell (i0+t, j0+TY): y_e x and z
                const int t = tid - 2 * TY - TX;
                ye_at(t + 4, TY + 1, o0, o1, o2);
                pend_a = o0;
                pend_b = o2;
            }
        }
        if (__syncthreads_or(bad)) {
            aborted = true;
            break;
        }
        // (c) finish plane k
        if (k >= k0 && own) {
            // r'_e = kap cb C~ y_h + eta^2 r_e (y_h of plane k-1 from registers)
            const T tx = (yhz - sm.yh[2][ly][lx + 1]) - (yhy - yhp_y);
            const T ty = (yhx - yhp_x) - (yhz - sm.yh[2][ly + 1][lx]);
            const T tz = (yhy - sm.yh[1][ly + 1][lx]) - (yhx - sm.yh[0][ly][lx + 1]);
            // r'_h = -kap ch C y_e + eta^2 r_h (y_e of plane k+1 from registers)
            const T cx = (yey + sm.ye[2][ly + 1][lx]) - (ye_n1 + yez);
            const T cy = (yez + ye_n0) - (sm.ye[2][ly][lx + 1] + yex);
            const T cz = (yex + sm.ye[1][ly][lx + 1]) - (sm.ye[0][ly + 1][lx] + yey);
            const T rex = RV(eC, 0, sy, sx), rey = RV(eC, 1, sy, sx), rez = RV(eC, 2, sy, sx);
            const T rhx = RV(hC, 0, sy, sx), rhy = RV(hC, 1, sy, sx), rhz = RV(hC, 2, sy, sx);
            if (!LAST) {
                rout[c] = kap * (RV(bC, 0, sy, sx) * tx) + eta2 * rex;
                rout[n + c] = kap * (RV(bC, 1, sy, sx) * ty) + eta2 * rey;
                rout[2 * n + c] = kap * (RV(bC, 2, sy, sx) * tz) + eta2 * rez;
                rout[3 * n + c] = -kap * (ch_at(i, j, 0) * cx) + eta2 * rhx;
                rout[4 * n + c] = -kap * (ch_at(i, j, 1) * cy) + eta2 * rhy;
                rout[5 * n + c] = -kap * (ch_at(i, j, 2) * cz) + eta2 * rhz;
            }
            P[c] = p0 + (al_e * rex + ga_e * yex);
            P[n + c] = p1 + (al_e * rey + ga_e * yey);
            P[2 * n + c] = p2 + (al_e * rez + ga_e * yez);
            P[3 * n + c] = p3 + (al_h * rhx + ga_h * yhx);
            P[4 * n + c] = p4 + (al_h * rhy + ga_h * yhy);
            P[5 * n + c] = p5 + (al_h * rhz + ga_h * yhz);
        }
        yhp_x = yhx;
        yhp_y = yhy;
        __syncthreads();   // stage p and the shared y planes are free again
        if (tid == 0 && issued < total) {
            proxy_fence();
            issue(issued);
            ++issued;
        }
    }
#undef RV
    if (aborted && tid == 0) {
        atomicOr(a.err, kErrTimeout);
        for (int q = waited; q < issued; ++q) wait_plane(q);
    }
}

template <typename T, int TX, int TY, int S, bool LAST, bool MUARR>
cudaError_t launch_pair(const ExpoArgs<T> &a, const CUtensorMap &tm_r, const CUtensorMap &tm_cb, int wait_limit,
                        cudaStream_t s) {
    using G = PairGeom<T, TX, TY, S>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(expo_pair_tma_kernel<T, TX, TY, S, LAST, MUARR>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, G::DYN_SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int tiles_x = (a.nx + TX - 1) / TX, tiles_y = (a.ny + TY - 1) / TY;
    const long long blocks = (long long)a.nmem * tiles_x * tiles_y * a.nchunk;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    expo_pair_tma_kernel<T, TX, TY, S, LAST, MUARR>
        <<<(unsigned)blocks, TX * TY, G::DYN_SMEM, s>>>(a, tm_r, tm_cb, tiles_x, tiles_y, wait_limit);
    return cudaGetLastError();
}

// y = X r at the probe edges (e components), from the pair's input block
template <typename T>
__global__ void expo_gather_fused_kernel(const ExpoArgs<T> a) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.nmem * a.nprb) return;
    const int mem = t / a.nprb, p = t - mem * a.nprb;
    const ExpoMember<T> M = a.mem[mem];
    const T *x = (a.pair & 1) ? M.R : M.Y;
    const EdgeRef q = a.prb[p];
    const long long n = a.ncp, pitch = a.pitch, plane = (long long)a.pitch * a.ny;
    const long long c = q.i + pitch * ((long long)q.j + (long long)a.ny * q.k);
    auto h = [&](int comp, int di, int dj, int dk) -> T {
        const int ii = q.i + di, jj = q.j + dj, kk = q.k + dk;
        if (ii < 0 || jj < 0 || kk < 0) return T(0);
        return x[(3 + comp) * n + c + di + dj * pitch + dk * plane];
    };
    T curl;
    if (q.axis == 0) curl = (h(2, 0, 0, 0) - h(2, 0, -1, 0)) - (h(1, 0, 0, 0) - h(1, 0, 0, -1));
    else if (q.axis == 1) curl = (h(0, 0, 0, 0) - h(0, 0, 0, -1)) - (h(2, 0, 0, 0) - h(2, -1, 0, 0));
    else curl = (h(1, 0, 0, 0) - h(1, -1, 0, 0)) - (h(0, 0, 0, 0) - h(0, 0, -1, 0));
    const T y = (T)a.kappa * (a.cb[q.axis * n + c] * curl);
    double *row = M.basis + (long long)a.substep * a.m1 * a.nprb;
    row[(long long)(2 * a.pair - 1) * a.nprb + p] = (double)x[q.axis * n + c];
    row[(long long)(2 * a.pair) * a.nprb + p] = (double)y;
}

}  // namespace

bool expo_pair_tma_supported(int elem_bytes, int nx) {
    (void)nx;
    return elem_bytes == 4 || elem_bytes == 8;
}

template <typename T>
cudaError_t launch_expo_pair_tma(const ExpoArgs<T> &a, const CUtensorMap &tm_r, const CUtensorMap &tm_cb,
                                 bool last, bool mu_array, int wait_limit, cudaStream_t s) {
    if (a.nmem <= 0) return cudaSuccess;
    constexpr int TX = 32, TY = sizeof(T) == 4 ? 8 : 4, S = 3;
#define FIT_PAIR(L, MU) return launch_pair<T, TX, TY, S, L, MU>(a, tm_r, tm_cb, wait_limit, s)
    if (last) {
        if (mu_array) FIT_PAIR(true, true);
        FIT_PAIR(true, false);
    }
    if (mu_array) FIT_PAIR(false, true);
    FIT_PAIR(false, false);
#undef FIT_PAIR
}

template <typename T>
cudaError_t launch_expo_gather_fused(const ExpoArgs<T> &a, cudaStream_t s) {
    const int n = a.nmem * a.nprb;
    if (n <= 0) return cudaSuccess;
    expo_gather_fused_kernel<T><<<(n + 127) / 128, 128, 0, s>>>(a);
    return cudaGetLastError();
}

int expo_pair_tile_x(int elem_bytes) { return 32 + 0 * elem_bytes; }
int expo_pair_tile_y(int elem_bytes) { return elem_bytes == 4 ? 8 : 4; }

template cudaError_t launch_expo_pair_tma<float>(const ExpoArgs<float> &, const CUtensorMap &, const CUtensorMap &,
                                                 bool, bool, int, cudaStream_t);
template cudaError_t launch_expo_pair_tma<double>(const ExpoArgs<double> &, const CUtensorMap &,
                                                  const CUtensorMap &, bool, bool, int, cudaStream_t);
template cudaError_t launch_expo_gather_fused<float>(const ExpoArgs<float> &, cudaStream_t);
template cudaError_t launch_expo_gather_fused<double>(const ExpoArgs<double> &, cudaStream_t);

}  // namespace fitgb
