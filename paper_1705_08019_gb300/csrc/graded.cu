// graded.cu -- tensor-product graded grids: cell (i, j, k) has the size
// dx[i] x dy[j] x dz[k].  Material matrices, leapfrog coefficients, the CFL
// estimate of eq. (cfl) with each cell's own sizes, and the absolute row sums
// of the skew matrix A of eq. (FIT_ode_2), whose maximum ||A||_1 = ||A||_inf
// bounds the spectrum the exponential propagators interpolate on.
//
// Material matrices (Sec. II, eq. maxwell_grid3) with local sizes:
//   M_eps(edge a at q) = eps0 / d_a[q_a] * sum over the four cells around the
//     edge of eps_r * d_b * d_c / 4   (each cell's part of the dual facet),
//   M_sigma likewise,
//   M_mu(face a at q)  = mu0 * d_b[q_b] d_c[q_c] / s,
//     s = (d_a[q_a-1]/2) / mu_r(q - u_a) + (d_a[q_a]/2) / mu_r(q)
//     (the two halves of the dual edge in series).
// On a grid with constant sizes these are the uniform expressions of aux.cu.
// All arithmetic is FP64 with explicit _rn intrinsics (no fused multiply-add),
// in the order stated, so the values are reproducible bit for bit.
#include <cmath>
#include <cstring>

#include "internal.h"

namespace fitgb {
namespace {

constexpr int kThreads = 256;

inline unsigned blocks_for(long long n) {
    long long b = (n + kThreads - 1) / kThreads;
    if (b > 152LL * 64) b = 152LL * 64;
    return (unsigned)(b > 0 ? b : 1);
}

struct GradedGeom {
    int n[3];
    const double *d[3];   // device: sizes along x, y, z
    const float *eps, *mu, *sig;
};

__device__ __forceinline__ long long cell_of(const GradedGeom &G, int i, int j, int k) {
    return (long long)i + (long long)G.n[0] * ((long long)j + (long long)G.n[1] * k);
}

__device__ __forceinline__ bool edge_free(const GradedGeom &G, int a, const int q[3]) {
    const int b = (a + 1) % 3, c = (a + 2) % 3;
    return q[a] >= 0 && q[a] < G.n[a] && q[b] > 0 && q[b] < G.n[b] && q[c] > 0 && q[c] < G.n[c];
}

__device__ __forceinline__ bool face_interior(const GradedGeom &G, int a, const int q[3]) {
    const int b = (a + 1) % 3, c = (a + 2) % 3;
    return q[a] > 0 && q[a] < G.n[a] && q[b] >= 0 && q[b] < G.n[b] && q[c] >= 0 && q[c] < G.n[c];
}

// M_eps and M_sigma of a free edge along a at q
__device__ void edge_mats(const GradedGeom &G, int a, const int q[3], double *me, double *ms) {
    const int b = (a + 1) % 3, c = (a + 2) % 3;
    double esum = 0.0, ssum = 0.0;
    for (int sb = 0; sb < 2; ++sb)
        for (int sc = 0; sc < 2; ++sc) {
            int r[3] = {q[0], q[1], q[2]};
            r[b] -= sb;
            r[c] -= sc;
            const long long cc = cell_of(G, r[0], r[1], r[2]);
            const double w = __ddiv_rn(__dmul_rn(G.d[b][r[b]], G.d[c][r[c]]), 4.0);
            esum = __dadd_rn(esum, __dmul_rn((double)G.eps[cc], w));
            ssum = __dadd_rn(ssum, __dmul_rn(G.sig ? (double)G.sig[cc] : 0.0, w));
        }
    const double len = G.d[a][q[a]];
    *me = __ddiv_rn(__dmul_rn(kEps0, esum), len);
    *ms = __ddiv_rn(ssum, len);
}

// M_mu of an interior face normal to a at q
__device__ double face_mat(const GradedGeom &G, int a, const int q[3]) {
    const int b = (a + 1) % 3, c = (a + 2) % 3;
    int r[3] = {q[0], q[1], q[2]};
    r[a] -= 1;
    const double m1 = G.mu ? (double)G.mu[cell_of(G, r[0], r[1], r[2])] : 1.0;
    const double m2 = G.mu ? (double)G.mu[cell_of(G, q[0], q[1], q[2])] : 1.0;
    const double area = __dmul_rn(G.d[b][q[b]], G.d[c][q[c]]);
    const double s = __dadd_rn(__ddiv_rn(__ddiv_rn(G.d[a][q[a] - 1], 2.0), m1),
                               __ddiv_rn(__ddiv_rn(G.d[a][q[a]], 2.0), m2));
    return __ddiv_rn(__dmul_rn(kMu0, area), s);
}

template <typename T>
__global__ void coeff_graded_kernel(GradedGeom G, int pitch, double dt, int scheme, T *ca, T *cb, T *ch, T *meps,
                                    T *mmu, int round_float) {
    const int nx = G.n[0], ny = G.n[1], nz = G.n[2];
    const long long ncell = (long long)pitch * ny * nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
         c += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(c % pitch);
        const int j = (int)((c / pitch) % ny);
        const int k = (int)(c / ((long long)pitch * ny));
        const int q[3] = {i, j, k};
        const bool pad = i >= nx;
        for (int a = 0; a < 3; ++a) {
            const long long o = (long long)a * ncell + c;
            T vca = T(0), vcb = T(0), vme = T(0), vch = T(0), vmm = T(0);
            if (!pad && edge_free(G, a, q)) {
                double Me, Ms;
                edge_mats(G, a, q, &Me, &Ms);
                const double av = __ddiv_rn(__dmul_rn(dt, Ms), __dmul_rn(2.0, Me));
                double xa, xb;
                if (scheme == 0) {
                    xa = __ddiv_rn(__dsub_rn(1.0, av), __dadd_rn(1.0, av));
                    xb = __ddiv_rn(dt, __dmul_rn(Me, __dadd_rn(1.0, av)));
                } else {
                    xa = __dsub_rn(1.0, __dmul_rn(2.0, av));
                    xb = __ddiv_rn(dt, Me);
                }
                if (round_float) {
                    xa = (double)(float)xa;
                    xb = (double)(float)xb;
                }
                vca = (T)xa;
                vcb = (T)xb;
                vme = (T)Me;
            }
            if (!pad && face_interior(G, a, q)) {
                const double Mm = face_mat(G, a, q);
                const double x = __ddiv_rn(dt, Mm);
                vch = (T)(round_float ? (double)(float)x : x);
                vmm = (T)Mm;
            }
            if (ca) ca[o] = vca;
            cb[o] = vcb;
            ch[o] = vch;
            if (meps) meps[o] = vme;
            if (mmu) mmu[o] = vmm;
        }
    }
}

// min over cells of sqrt(eps mu / (1/dx^2 + 1/dy^2 + 1/dz^2)), eps, mu absolute (eq. cfl)
__global__ void cfl_graded_kernel(GradedGeom G, unsigned long long *mnbits) {
    const long long n = (long long)G.n[0] * G.n[1] * G.n[2];
    double mn = INFINITY;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(c % G.n[0]);
        const int j = (int)((c / G.n[0]) % G.n[1]);
        const int k = (int)(c / ((long long)G.n[0] * G.n[1]));
        const double dx = G.d[0][i], dy = G.d[1][j], dz = G.d[2][k];
        const double inv = __dadd_rn(__dadd_rn(__ddiv_rn(1.0, __dmul_rn(dx, dx)), __ddiv_rn(1.0, __dmul_rn(dy, dy))),
                                     __ddiv_rn(1.0, __dmul_rn(dz, dz)));
        const double em = __dmul_rn(__dmul_rn(__dmul_rn(kEps0, (double)G.eps[c]), kMu0),
                                    G.mu ? (double)G.mu[c] : 1.0);
        const double t = __dsqrt_rn(__ddiv_rn(em, inv));
        mn = fmin(mn, t);
    }
    for (int off = 16; off > 0; off >>= 1) mn = fmin(mn, __shfl_down_sync(0xffffffffu, mn, off));
    if ((threadIdx.x & 31) == 0 && isfinite(mn)) atomicMin(mnbits, (unsigned long long)__double_as_longlong(mn));
}

__device__ __forceinline__ double inv_sqrt_me(const GradedGeom &G, int a, const int q[3]) {
    if (!edge_free(G, a, q)) return 0.0;
    double me, ms;
    edge_mats(G, a, q, &me, &ms);
    return __ddiv_rn(1.0, __dsqrt_rn(me));
}

__device__ __forceinline__ double inv_sqrt_mm(const GradedGeom &G, int a, const int q[3]) {
    if (!face_interior(G, a, q)) return 0.0;
    return __ddiv_rn(1.0, __dsqrt_rn(face_mat(G, a, q)));
}

// max over rows of A of the absolute row sum (edges and faces of the degrees of freedom)
__global__ void rowsum_graded_kernel(GradedGeom G, unsigned long long *mxbits) {
    const long long n = (long long)G.n[0] * G.n[1] * G.n[2];
    double mx = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        const int q[3] = {(int)(c % G.n[0]), (int)((c / G.n[0]) % G.n[1]), (int)(c / ((long long)G.n[0] * G.n[1]))};
        for (int a = 0; a < 3; ++a) {
            const int b = (a + 1) % 3, cc = (a + 2) % 3;
            if (edge_free(G, a, q)) {   // faces h_c(q), h_b(q), h_c(q - u_b), h_b(q - u_c)
                int qb[3] = {q[0], q[1], q[2]}, qc[3] = {q[0], q[1], q[2]};
                qb[b] -= 1;
                qc[cc] -= 1;
                double s = __dadd_rn(inv_sqrt_mm(G, cc, q), inv_sqrt_mm(G, b, q));
                if (qb[b] >= 0) s = __dadd_rn(s, inv_sqrt_mm(G, cc, qb));
                if (qc[cc] >= 0) s = __dadd_rn(s, inv_sqrt_mm(G, b, qc));
                mx = fmax(mx, __dmul_rn(inv_sqrt_me(G, a, q), s));
            }
            if (face_interior(G, a, q)) {   // edges e_b(q), e_c(q), e_c(q + u_b), e_b(q + u_c)
                int qb[3] = {q[0], q[1], q[2]}, qc[3] = {q[0], q[1], q[2]};
                qb[b] += 1;
                qc[cc] += 1;
                double s = __dadd_rn(inv_sqrt_me(G, b, q), inv_sqrt_me(G, cc, q));
                if (qb[b] <= G.n[b]) s = __dadd_rn(s, inv_sqrt_me(G, cc, qb));
                if (qc[cc] <= G.n[cc]) s = __dadd_rn(s, inv_sqrt_me(G, b, qc));
                mx = fmax(mx, __dmul_rn(inv_sqrt_mm(G, a, q), s));
            }
        }
    }
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, off));
    if ((threadIdx.x & 31) == 0) atomicMax(mxbits, (unsigned long long)__double_as_longlong(mx));
}

GradedGeom geom(int nx, int ny, int nz, const double *spc, const float *eps, const float *mu, const float *sig) {
    GradedGeom G;
    G.n[0] = nx; G.n[1] = ny; G.n[2] = nz;
    G.d[0] = spc; G.d[1] = spc + nx; G.d[2] = spc + nx + ny;
    G.eps = eps; G.mu = mu; G.sig = sig;
    return G;
}

}  // namespace

template <typename T>
cudaError_t build_coeffs_graded(int nx, int ny, int nz, int pitch, const double *spc_dev, const float *eps,
                                const float *mu, const float *sig, double dt, int scheme, T *ca, T *cb, T *ch,
                                T *meps, T *mmu, cudaStream_t s, bool round_float) {
    const GradedGeom G = geom(nx, ny, nz, spc_dev, eps, mu, sig);
    coeff_graded_kernel<T><<<blocks_for((long long)pitch * ny * nz), kThreads, 0, s>>>(
        G, pitch, dt, scheme, ca, cb, ch, meps, mmu, round_float ? 1 : 0);
    return cudaGetLastError();
}

template cudaError_t build_coeffs_graded<float>(int, int, int, int, const double *, const float *, const float *,
                                                const float *, double, int, float *, float *, float *, float *,
                                                float *, cudaStream_t, bool);
template cudaError_t build_coeffs_graded<double>(int, int, int, int, const double *, const float *, const float *,
                                                 const float *, double, int, double *, double *, double *, double *,
                                                 double *, cudaStream_t, bool);

cudaError_t graded_cfl_and_bound(int nx, int ny, int nz, const double *spc_dev, const float *eps, const float *mu,
                                 void *scratch, double *cfl, double *rowsum_max, cudaStream_t s) {
    const GradedGeom G = geom(nx, ny, nz, spc_dev, eps, mu, nullptr);
    unsigned long long *bits = static_cast<unsigned long long *>(scratch);
    unsigned long long init[2];
    const double inf = INFINITY, zero = 0.0;
    memcpy(&init[0], &inf, sizeof(double));
    memcpy(&init[1], &zero, sizeof(double));
    cudaError_t err = cudaMemcpyAsync(bits, init, sizeof(init), cudaMemcpyHostToDevice, s);
    if (err != cudaSuccess) return err;
    const long long n = (long long)nx * ny * nz;
    cfl_graded_kernel<<<blocks_for(n), kThreads, 0, s>>>(G, bits);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    rowsum_graded_kernel<<<blocks_for(n), kThreads, 0, s>>>(G, bits + 1);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    unsigned long long h[2];
    if ((err = cudaMemcpyAsync(h, bits, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return err;
    if ((err = cudaStreamSynchronize(s)) != cudaSuccess) return err;
    memcpy(cfl, &h[0], sizeof(double));
    memcpy(rowsum_max, &h[1], sizeof(double));
    return cudaSuccess;
}

}  // namespace fitgb
