// expo.cu -- device side of the exponential propagators of the homogeneous
// ParaExp problems (Sec. III-B): the real Newton form of the Leja (or Taylor)
// interpolant of exp(c X), X = dt_CFL A, applied in untransformed voltages,
//     X (e, h) = kappa (cb (.) C~h, -ch (.) C e),   kappa = dt_CFL / dt,
// which is similar to the paper's transformed skew A (the polynomial of
// M^{-1}K and of T M^{-1}K T^{-1} are the same up to the similarity T).
//
// One substep of the interpolant p_m, m = 2J:
//     init:           R = X P                         (P holds b)
//     pair j, part 1: Y = X R,  P += alpha_j R + gamma_j Y
//     pair j, part 2: R = X Y + eta_j^2 R             (not after the last pair)
// so P ends as p_m(X) b with d_0 = exp(0) = 1.  Each launch is one operator
// application over every active member: a thread owns one (i, j) column of
// kz cells and streams along z, keeping the h_x, h_y of plane k-1 and the
// e_x, e_y of plane k+1 in registers; the x and y neighbours come through
// L1/L2.  The last substep of a member uses its own coefficients for the e
// and for the h components (the final e and h fall at different fractions
// of that substep).  A fourth mode performs the half magnetic step that
// brings a leapfrog state (e^n, h^{n-1/2}) to (e^n, h^n):
//     h += (dt / (2 dt_CFL)) (X (e, h))_h = h - (1/2) ch (.) C e.
#include <algorithm>

#include "internal.h"

namespace fitgb {
namespace {

constexpr int kEx = 32, kEy = 8;   // threads per block along x and y

template <typename T, int MODE, bool MUARR>
__global__ void __launch_bounds__(kEx * kEy) expo_kernel(const ExpoArgs<T> a) {
    constexpr bool kNeedCh = MODE != kExpoSync;   // the synchronisation only needs (C e)
    const int mem = blockIdx.z / a.nchunk;
    if (mem >= a.nmem) return;
    const int chunk = blockIdx.z - mem * a.nchunk;
    const int i = blockIdx.x * kEx + threadIdx.x;
    const int j = blockIdx.y * kEy + threadIdx.y;
    if (i >= a.nx || j >= a.ny) return;   // no block-wide synchronisation below
    const ExpoMember<T> M = a.mem[mem];
    const long long n = a.ncp;
    const int pitch = a.pitch;
    const long long plane = (long long)pitch * a.ny;
    const int k0 = chunk * a.kz;
    const int k1 = min(a.nz, k0 + a.kz);

    // the stencil input is not written by this launch (the synchronisation
    // writes only the h of its own cell, after reading it): read-only loads
    const T *__restrict__ x = MODE == kExpoPair1 ? M.R : MODE == kExpoPair2 ? M.Y : M.P;
    const T *__restrict__ cb = a.cb;
    const T *__restrict__ chp = a.ch;
    const T kap = (T)a.kappa;

    T al_e = T(0), ga_e = T(0), al_h = T(0), ga_h = T(0);
    if (MODE == kExpoPair1) {
        if (a.substep == M.nsub - 1) {
            const double *f = M.fin + 4 * (a.pair - 1);
            al_e = (T)f[0]; ga_e = (T)f[1]; al_h = (T)f[2]; ga_h = (T)f[3];
        } else {
            al_e = al_h = (T)a.reg[2 * (a.pair - 1)];
            ga_e = ga_h = (T)a.reg[2 * (a.pair - 1) + 1];
        }
    }
    const T eta2 = (T)a.eta2;
    const T sync = (T)a.sync;
    const T chs0 = MUARR ? T(0) : __ldg(chp), chs1 = MUARR ? T(0) : __ldg(chp + 1), chs2 = MUARR ? T(0) : __ldg(chp + 2);

    const bool xup = i + 1 < a.nx, yup = j + 1 < a.ny, xdn = i > 0, ydn = j > 0;
    long long c = (long long)i + (long long)pitch * j + plane * k0;
    // carried along z: h_x, h_y of plane k-1 and e_x, e_y of plane k
    T hx_m = (kNeedCh && k0 > 0) ? __ldg(x + 3 * n + c - plane) : T(0);
    T hy_m = (kNeedCh && k0 > 0) ? __ldg(x + 4 * n + c - plane) : T(0);
    T ex_0 = __ldg(x + c), ey_0 = __ldg(x + n + c);
    for (int k = k0; k < k1; ++k, c += plane) {
        const bool zup = k + 1 < a.nz;
        const T ex_p = zup ? __ldg(x + c + plane) : T(0);
        const T ey_p = zup ? __ldg(x + n + c + plane) : T(0);
        const T ez = __ldg(x + 2 * n + c);
        const T hx = __ldg(x + 3 * n + c), hy = __ldg(x + 4 * n + c), hz = __ldg(x + 5 * n + c);
        const T ey_ip = xup ? __ldg(x + n + c + 1) : T(0);
        const T ez_ip = xup ? __ldg(x + 2 * n + c + 1) : T(0);
        const T ex_jp = yup ? __ldg(x + c + pitch) : T(0);
        const T ez_jp = yup ? __ldg(x + 2 * n + c + pitch) : T(0);
        const T hy_im = (kNeedCh && xdn) ? __ldg(x + 4 * n + c - 1) : T(0);
        const T hz_im = (kNeedCh && xdn) ? __ldg(x + 5 * n + c - 1) : T(0);
        const T hx_jm = (kNeedCh && ydn) ? __ldg(x + 3 * n + c - pitch) : T(0);
        const T hz_jm = (kNeedCh && ydn) ? __ldg(x + 5 * n + c - pitch) : T(0);
        // (C e) on the faces with lowest corner (i, j, k): circulation, (a, b, c) cyclic
        const T cex = (ey_0 + ez_jp) - (ey_p + ez);
        const T cey = (ez + ex_p) - (ez_ip + ex_0);
        const T cez = (ex_0 + ey_ip) - (ex_jp + ey_0);
        // (C~ h) on the edges starting at (i, j, k)
        const T chx = (hz - hz_jm) - (hy - hy_m);
        const T chy = (hx - hx_m) - (hz - hz_im);
        const T chz = (hy - hy_im) - (hx - hx_jm);
        const T ch0 = MUARR ? __ldg(chp + c) : chs0;
        const T ch1 = MUARR ? __ldg(chp + n + c) : chs1;
        const T ch2 = MUARR ? __ldg(chp + 2 * n + c) : chs2;
        const T y0 = kNeedCh ? kap * (__ldg(cb + c) * chx) : T(0);
        const T y1 = kNeedCh ? kap * (__ldg(cb + n + c) * chy) : T(0);
        const T y2 = kNeedCh ? kap * (__ldg(cb + 2 * n + c) * chz) : T(0);
        const T y3 = -kap * (ch0 * cex);
        const T y4 = -kap * (ch1 * cey);
        const T y5 = -kap * (ch2 * cez);
        if (MODE == kExpoInit) {
            T *R = M.R;
            R[c] = y0; R[n + c] = y1; R[2 * n + c] = y2;
            R[3 * n + c] = y3; R[4 * n + c] = y4; R[5 * n + c] = y5;
        } else if (MODE == kExpoPair1) {
            T *Y = M.Y, *P = M.P;
            Y[c] = y0; Y[n + c] = y1; Y[2 * n + c] = y2;
            Y[3 * n + c] = y3; Y[4 * n + c] = y4; Y[5 * n + c] = y5;
            P[c] += al_e * ex_0 + ga_e * y0;
            P[n + c] += al_e * ey_0 + ga_e * y1;
            P[2 * n + c] += al_e * ez + ga_e * y2;
            P[3 * n + c] += al_h * hx + ga_h * y3;
            P[4 * n + c] += al_h * hy + ga_h * y4;
            P[5 * n + c] += al_h * hz + ga_h * y5;
        } else if (MODE == kExpoPair2) {
            T *R = M.R;
            R[c] = y0 + eta2 * R[c];
            R[n + c] = y1 + eta2 * R[n + c];
            R[2 * n + c] = y2 + eta2 * R[2 * n + c];
            R[3 * n + c] = y3 + eta2 * R[3 * n + c];
            R[4 * n + c] = y4 + eta2 * R[4 * n + c];
            R[5 * n + c] = y5 + eta2 * R[5 * n + c];
        } else {   // kExpoSync: only h changes, and it depends on e alone
            T *P = M.P;
            P[3 * n + c] = hx + sync * y3;
            P[4 * n + c] = hy + sync * y4;
            P[5 * n + c] = hz + sync * y5;
        }
        hx_m = hx;
        hy_m = hy;
        ex_0 = ex_p;
        ey_0 = ey_p;
    }
}

// Probe rows of the Newton basis: after init, row 0 = b (in P); after the
// first part of pair j, rows 2j-1 = R_{j-1} b and 2j = Y_j = X R_{j-1} b.
template <typename T>
__global__ void expo_gather_kernel(const ExpoArgs<T> a) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.nmem * a.nprb) return;
    const int mem = t / a.nprb, p = t - mem * a.nprb;
    const ExpoMember<T> M = a.mem[mem];
    const EdgeRef q = a.prb[p];
    const long long c = (long long)q.axis * a.ncp + (long long)q.i +
                        (long long)a.pitch * ((long long)q.j + (long long)a.ny * q.k);
    double *row = M.basis + (long long)a.substep * a.m1 * a.nprb;
    if (a.mode == kExpoInit) {
        row[p] = (double)M.P[c];
    } else {
        row[(long long)(2 * a.pair - 1) * a.nprb + p] = (double)M.R[c];
        row[(long long)(2 * a.pair) * a.nprb + p] = (double)M.Y[c];
    }
}

__global__ void expo_dense_kernel(const double *const *basis, const long long *nrem, const long long *row0,
                                  long long max_rows, int q, int m1, int nprb, const double *D, double *out,
                                  long long ostride) {
    const int mem = blockIdx.y;
    const long long nr = nrem[mem];
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < nr && r < max_rows;
         r += (long long)gridDim.x * blockDim.x) {
        const long long s = r / q;
        const int i = (int)(r - s * q);
        const double *B = basis[mem] + s * m1 * nprb;
        const double *Drow = D + (long long)i * m1;
        double *o = out + mem * ostride + (row0[mem] + r) * nprb;
        for (int p = 0; p < nprb; ++p) {
            double v = 0.0;
            for (int k = 0; k < m1; ++k) v += Drow[k] * B[(long long)k * nprb + p];
            o[p] = v;
        }
    }
}

__global__ void add_members_kernel(int nmem, long long len, const double *pm, long long stride, double *out) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < len;
         t += (long long)gridDim.x * blockDim.x) {
        double s = out[t];
        for (int m = 0; m < nmem; ++m) s += pm[(long long)m * stride + t];
        out[t] = s;
    }
}

}  // namespace

template <typename T>
cudaError_t launch_expo(const ExpoArgs<T> &a, bool mu_array, cudaStream_t s) {
    if (a.nmem <= 0) return cudaSuccess;
    const long long gz = (long long)a.nchunk * a.nmem;
    if (gz > 65535) return cudaErrorInvalidConfiguration;
    dim3 grid((a.nx + kEx - 1) / kEx, (a.ny + kEy - 1) / kEy, (unsigned)gz), block(kEx, kEy);
#define FIT_EXPO_LAUNCH(MODE)                                        \
    do {                                                             \
        if (mu_array)                                                \
            expo_kernel<T, MODE, true><<<grid, block, 0, s>>>(a);    \
        else                                                         \
            expo_kernel<T, MODE, false><<<grid, block, 0, s>>>(a);   \
    } while (0)
    switch (a.mode) {
    case kExpoInit: FIT_EXPO_LAUNCH(kExpoInit); break;
    case kExpoPair1: FIT_EXPO_LAUNCH(kExpoPair1); break;
    case kExpoPair2: FIT_EXPO_LAUNCH(kExpoPair2); break;
    case kExpoSync: FIT_EXPO_LAUNCH(kExpoSync); break;
    default: return cudaErrorInvalidValue;
    }
#undef FIT_EXPO_LAUNCH
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_expo_gather(const ExpoArgs<T> &a, cudaStream_t s) {
    const int n = a.nmem * a.nprb;
    if (n <= 0) return cudaSuccess;
    expo_gather_kernel<T><<<(n + 127) / 128, 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_expo_dense(int nmem, const double *const *basis, const long long *nrem, const long long *row0,
                              long long max_rows, int q, int m1, int nprb, const double *D, double *out,
                              long long ostride, cudaStream_t s) {
    if (nmem <= 0 || max_rows <= 0 || nprb <= 0) return cudaSuccess;
    const long long bx = std::min<long long>((max_rows + 127) / 128, 4096);
    expo_dense_kernel<<<dim3((unsigned)bx, nmem), 128, 0, s>>>(basis, nrem, row0, max_rows, q, m1, nprb, D, out,
                                                               ostride);
    return cudaGetLastError();
}

cudaError_t add_members(int nmem, long long len, const double *pm, long long stride, double *out, cudaStream_t s) {
    if (len <= 0) return cudaSuccess;
    const long long b = std::min<long long>((len + 255) / 256, 4096);
    add_members_kernel<<<(unsigned)b, 256, 0, s>>>(nmem, len, pm, stride, out);
    return cudaGetLastError();
}

template cudaError_t launch_expo<float>(const ExpoArgs<float> &, bool, cudaStream_t);
template cudaError_t launch_expo<double>(const ExpoArgs<double> &, bool, cudaStream_t);
template cudaError_t launch_expo_gather<float>(const ExpoArgs<float> &, cudaStream_t);
template cudaError_t launch_expo_gather<double>(const ExpoArgs<double> &, cudaStream_t);

}  // namespace fitgb
