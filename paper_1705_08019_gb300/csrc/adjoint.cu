// adjoint.cu -- kernels of the adjoint gradient dJ/d eps_r.
//
// Functional: J = sum_{n=1..N} sum_p (e_p^n / L_p)^2 over the probe edges.
// The reverse sweep transposes the leapfrog step of Sec. II-A.  Written in
// the scaled adjoint variables mu = cb (.) lambda_e and nu = -ch (.) lambda_h
// it reads
//     nu^{n+1/2} = nu^{n+3/2} - ch (.) C mu^{n+1}
//     mu^n       = ca (.) mu^{n+1} + cb (.) (C~ nu^{n+1/2} + dJ/de^n)
// which is the forward step itself with the impressed current -j replaced by
// the probe derivative dJ/de^n = 2 e_p^n / L_p^2, so the fused step kernels
// run it unchanged (the probe edges become its sources).
//
// Gradient.  With M_eps = eps0 eps_bar A/L on an edge, the discrete Ampere
// law of the leapfrog, M_eps (e^{n+1}-e^n)/dt = C~h - M_sigma e_s - j (e_s the
// sigma scheme's e), depends on eps_bar only through M_eps.  Its Lagrange
// multiplier in the update e^{n+1} = ca e^n + cb (...) is cb (.) lambda_e =
// mu, so per edge
//     dJ/d eps_bar = -(eps0 A / (L dt)) sum_n mu^{n+1} (e^{n+1} - e^n),
// and d eps_bar / d eps_r(cell) = 1/4 for each of the four cells around the
// edge.  Edges in a PEC wall have cb = 0, so mu and their gradient vanish by
// themselves.
//
// Graded grids: M_eps = (eps0 / d_a) sum over the four cells of
// eps_r d_b d_c / 4, so each cell's weight is its own d_b d_c / 4 and the
// edge length d_a is that cell's size along a as well.  The accumulation then
// runs with K = -eps0 / dt on every axis, and the scatter multiplies the four
// a-edges of a cell by d_b d_c / d_a of that cell (the 1/4 stays).
#include "internal.h"

namespace fitgb {
namespace {

constexpr int kThreads = 256;

inline unsigned grid_for(long long n) {
    long long b = (n + kThreads - 1) / kThreads;
    if (b > 152LL * 64) b = 152LL * 64;
    return (unsigned)(b > 0 ? b : 1);
}

struct ProbeList {
    int n;
    EdgeRef p[kMaxSrc];
    double inv_l2[kMaxSrc];   // 1 / L_p^2
};

// mu^N = cb (.) dJ/de^N on the probe edges (the adjoint state is zero before)
template <typename T>
__global__ void adjoint_init_kernel(ProbeList pl, const double *probe_last, const T *cb, T *mu, int pitch, int ny,
                                    long long ncp) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    for (int q = 0; q < pl.n; ++q) {   // serial: probes may share an edge
        const EdgeRef r = pl.p[q];
        const long long c = (long long)r.axis * ncp + ((long long)r.k * ny + r.j) * pitch + r.i;
        mu[c] += (T)((double)cb[c] * 2.0 * probe_last[q] * pl.inv_l2[q]);
    }
}

// sources of the adjoint sweep: at adjoint iteration t the step produces
// mu^n, n = N-1-t, whose impressed current is -dJ/de^n (zero for n = 0)
__global__ void adjoint_amp_kernel(ProbeList pl, const double *probe, long long N, double *amp) {
    const long long total = N * pl.n;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long it = t / pl.n;
        const int q = (int)(t % pl.n);
        const long long n = N - 1 - it;
        amp[t] = n >= 1 ? -2.0 * probe[(n - 1) * pl.n + q] * pl.inv_l2[q] : 0.0;
    }
}

// g_a += K_a mu^{n+1} (e^{n+1} - e^n) on every edge, K_a = -eps0 A_a / (L_a dt)
template <typename T>
__global__ void grad_accum_kernel(long long ncp, const T *mu, const T *e1, const T *e0, double k0, double k1,
                                  double k2, double *g) {
    const long long n3 = 3 * ncp;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n3;
         c += (long long)gridDim.x * blockDim.x) {
        const T prod = mu[c] * (e1[c] - e0[c]);
        const double k = c < ncp ? k0 : (c < 2 * ncp ? k1 : k2);
        g[c] += k * (double)prod;
    }
}

// the same into an FP32 block sum (FP32 fields): the FP64 total then takes one
// read-modify-write per block of steps instead of one per step
__global__ void grad_accum_block_kernel(long long ncp, const float *mu, const float *e1, const float *e0, float k0,
                                        float k1, float k2, float *gb) {
    const long long n3 = 3 * ncp;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n3;
         c += (long long)gridDim.x * blockDim.x) {
        const float prod = mu[c] * (e1[c] - e0[c]);
        const float k = c < ncp ? k0 : (c < 2 * ncp ? k1 : k2);
        gb[c] += k * prod;
    }
}

__global__ void grad_flush_kernel(long long n3, float *gb, double *g) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n3;
         c += (long long)gridDim.x * blockDim.x) {
        g[c] += (double)gb[c];
        gb[c] = 0.f;
    }
}

// dJ/d eps_r(cell) = 1/4 sum over the 12 edges around the cell of g_edge;
// spc (graded grids; null on uniform ones): dx[nx], dy[ny], dz[nz] in a row,
// the edges along a weighted by the cell's d_b d_c / d_a
__global__ void scatter_kernel(int nx, int ny, int nz, int pitch, long long ncp, const double *g, const double *spc,
                               double *grad) {
    const long long ncell = (long long)nx * ny * nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
         c += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(c % nx);
        const int j = (int)((c / nx) % ny);
        const int k = (int)(c / ((long long)nx * ny));
        auto at = [&](int a, int ii, int jj, int kk) -> double {
            if (ii >= nx || jj >= ny || kk >= nz) return 0.0;   // edge in a wall: no degree of freedom
            return g[(long long)a * ncp + ((long long)kk * ny + jj) * pitch + ii];
        };
        if (spc) {
            double sx = 0.0, sy = 0.0, sz = 0.0;
            for (int u = 0; u < 2; ++u)
                for (int v = 0; v < 2; ++v) {
                    sx += at(0, i, j + u, k + v);
                    sy += at(1, i + u, j, k + v);
                    sz += at(2, i + u, j + v, k);
                }
            const double dx = spc[i], dy = spc[nx + j], dz = spc[nx + ny + k];
            grad[c] = 0.25 * (sx * (dy * dz / dx) + sy * (dz * dx / dy) + sz * (dx * dy / dz));
            continue;
        }
        double s = 0.0;
        for (int u = 0; u < 2; ++u)
            for (int v = 0; v < 2; ++v) {
                s += at(0, i, j + u, k + v);   // x-edges of the cell
                s += at(1, i + u, j, k + v);   // y-edges
                s += at(2, i + u, j + v, k);   // z-edges
            }
        grad[c] = 0.25 * s;
    }
}

// J = sum over the N x nprb probe record of (e / L)^2, in FP64
__global__ void functional_kernel(ProbeList pl, const double *probe, long long N, double *J) {
    __shared__ double red[kThreads / 32];
    double s = 0.0;
    const long long total = N * pl.n;
    for (long long t = threadIdx.x; t < total; t += blockDim.x) {
        const double v = probe[t];
        s += v * v * pl.inv_l2[t % pl.n];
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += red[w];
        *J = t;
    }
}

// plen: the length of each probe's edge (host, nprb values)
ProbeList make_list(const fit_probe *prb, int nprb, const double *plen) {
    ProbeList pl;
    pl.n = nprb;
    for (int q = 0; q < nprb && q < kMaxSrc; ++q) {
        pl.p[q] = {prb[q].axis, prb[q].i, prb[q].j, prb[q].k};
        const double L = plen[q];
        pl.inv_l2[q] = 1.0 / (L * L);
    }
    return pl;
}

}  // namespace

template <typename T>
cudaError_t adjoint_init(const fit_probe *prb, int nprb, const double *plen, const double *probe_last, const T *cb,
                         T *mu, int pitch, int ny, long long ncp, cudaStream_t s) {
    adjoint_init_kernel<T><<<1, 32, 0, s>>>(make_list(prb, nprb, plen), probe_last, cb, mu, pitch, ny, ncp);
    return cudaGetLastError();
}

cudaError_t adjoint_sources(const fit_probe *prb, int nprb, const double *plen, const double *probe, long long N,
                            double *amp, cudaStream_t s) {
    adjoint_amp_kernel<<<grid_for(N * nprb), kThreads, 0, s>>>(make_list(prb, nprb, plen), probe, N, amp);
    return cudaGetLastError();
}

template <typename T>
cudaError_t grad_accumulate(long long ncp, const T *mu, const T *e1, const T *e0, const double k[3], double *g,
                            cudaStream_t s) {
    grad_accum_kernel<T><<<grid_for(3 * ncp), kThreads, 0, s>>>(ncp, mu, e1, e0, k[0], k[1], k[2], g);
    return cudaGetLastError();
}

cudaError_t grad_accumulate_block(long long ncp, const float *mu, const float *e1, const float *e0, const double k[3],
                                  float *gb, cudaStream_t s) {
    grad_accum_block_kernel<<<grid_for(3 * ncp), kThreads, 0, s>>>(ncp, mu, e1, e0, (float)k[0], (float)k[1],
                                                                   (float)k[2], gb);
    return cudaGetLastError();
}

cudaError_t grad_flush(long long ncp, float *gb, double *g, cudaStream_t s) {
    grad_flush_kernel<<<grid_for(3 * ncp), kThreads, 0, s>>>(3 * ncp, gb, g);
    return cudaGetLastError();
}

cudaError_t grad_scatter(int nx, int ny, int nz, int pitch, long long ncp, const double *g, const double *spc,
                         double *grad, cudaStream_t s) {
    scatter_kernel<<<grid_for((long long)nx * ny * nz), kThreads, 0, s>>>(nx, ny, nz, pitch, ncp, g, spc, grad);
    return cudaGetLastError();
}

cudaError_t probe_functional(const fit_probe *prb, int nprb, const double *plen, const double *probe, long long N,
                             double *J, cudaStream_t s) {
    functional_kernel<<<1, kThreads, 0, s>>>(make_list(prb, nprb, plen), probe, N, J);
    return cudaGetLastError();
}

template cudaError_t adjoint_init<float>(const fit_probe *, int, const double *, const double *, const float *,
                                         float *, int, int, long long, cudaStream_t);
template cudaError_t adjoint_init<double>(const fit_probe *, int, const double *, const double *, const double *,
                                          double *, int, int, long long, cudaStream_t);
template cudaError_t grad_accumulate<float>(long long, const float *, const float *, const float *, const double *,
                                            double *, cudaStream_t);
template cudaError_t grad_accumulate<double>(long long, const double *, const double *, const double *,
                                             const double *, double *, cudaStream_t);

}  // namespace fitgb
