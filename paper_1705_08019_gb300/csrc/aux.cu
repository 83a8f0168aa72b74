// aux.cu -- once-per-run kernels around the fused step: material checks,
// leapfrog coefficients, source tables, state masking and the ParaExp
// superposition sums.
#include <cmath>
#include <cstring>

#include "internal.h"

namespace fitgb {
namespace {

constexpr int kThreads = 256;

inline unsigned grid_for(long long n, int per = kThreads) {
    long long b = (n + per - 1) / per;
    if (b > 152LL * 64) b = 152LL * 64;   // grid-stride beyond 64 CTAs per SM
    return (unsigned)(b > 0 ? b : 1);
}

// flags[0..4]: bad_eps, bad_mu, bad_sigma, mu_nonuniform, lossy; *mnbits: min(eps*mu) as FP64 bits
__global__ void check_kernel(const float *eps, const float *mu, const float *sig, long long n, int *flags,
                             unsigned long long *mnbits) {
    int bad_e = 0, bad_m = 0, bad_s = 0, nonu = 0, lossy = 0;
    double mn = INFINITY;
    const float mu_ref = mu ? mu[0] : 1.0f;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const float e = eps[c];
        const float m = mu ? mu[c] : 1.0f;
        const float s = sig ? sig[c] : 0.0f;
        if (!(e > 0.0f) || !isfinite(e)) bad_e = 1;
        if (!(m > 0.0f) || !isfinite(m)) bad_m = 1;
        if (!(s >= 0.0f) || !isfinite(s)) bad_s = 1;
        if (m != mu_ref) nonu = 1;
        if (s != 0.0f) lossy = 1;
        const double em = (double)e * (double)m;
        if (em < mn) mn = em;
    }
    bad_e = __syncthreads_or(bad_e);
    bad_m = __syncthreads_or(bad_m);
    bad_s = __syncthreads_or(bad_s);
    nonu = __syncthreads_or(nonu);
    lossy = __syncthreads_or(lossy);
    for (int off = 16; off > 0; off >>= 1) mn = fmin(mn, __shfl_down_sync(0xffffffffu, mn, off));
    if (threadIdx.x == 0) {
        if (bad_e) atomicOr(flags + 0, 1);
        if (bad_m) atomicOr(flags + 1, 1);
        if (bad_s) atomicOr(flags + 2, 1);
        if (nonu) atomicOr(flags + 3, 1);
        if (lossy) atomicOr(flags + 4, 1);
    }
    // non-negative doubles order like their bit patterns
    if ((threadIdx.x & 31) == 0 && mn >= 0.0 && isfinite(mn))
        atomicMin(mnbits, (unsigned long long)__double_as_longlong(mn));
}

// Leapfrog coefficients of one point (i,j,k): its three edges and three faces.
// The arithmetic is FP64 and rounds once to T at the end.  Explicit _rn
// intrinsics keep the compiler from fusing multiply-adds, so the FP64 values
// are the correctly rounded results of the stated operations in the stated
// order.
template <typename T>
__global__ void coeff_kernel(int nx, int ny, int nz, int pitch, double d0, double d1, double d2, const float *eps,
                             const float *mu, const float *sig, double dt, int scheme, int mu_array,
                             T *ca, T *cb, T *ch, T *meps, T *mmu, int round_float) {
    const long long ncell = (long long)pitch * ny * nz;   // padded component stride
    const double d[3] = {d0, d1, d2};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
         c += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(c % pitch);
        const int j = (int)((c / pitch) % ny);
        const int k = (int)(c / ((long long)pitch * ny));
        const int q[3] = {i, j, k};
        const long long cell = (long long)i + (long long)nx * ((long long)j + (long long)ny * k);
        const bool pad = i >= nx;
        for (int a = 0; a < 3; ++a) {
            const int b = (a + 1) % 3, cc = (a + 2) % 3;
            const double len = d[a];
            const double area = __dmul_rn(d[b], d[cc]);
            const long long o = (long long)a * ncell + c;
            // edge along a: a degree of freedom iff both other indices are > 0
            if (!pad && q[b] > 0 && q[cc] > 0) {
                double esum = 0.0, ssum = 0.0;
                for (int sb = 0; sb < 2; ++sb)
                    for (int sc = 0; sc < 2; ++sc) {
                        int r[3] = {q[0], q[1], q[2]};
                        r[b] -= sb;
                        r[cc] -= sc;
                        const long long rc = (long long)r[0] + (long long)nx * ((long long)r[1] + (long long)ny * r[2]);
                        esum = __dadd_rn(esum, (double)eps[rc]);
                        ssum = __dadd_rn(ssum, sig ? (double)sig[rc] : 0.0);
                    }
                const double ebar = __ddiv_rn(esum, 4.0), sbar = __ddiv_rn(ssum, 4.0);
                const double Me = __ddiv_rn(__dmul_rn(__dmul_rn(kEps0, ebar), area), len);
                const double Ms = __ddiv_rn(__dmul_rn(sbar, area), len);
                const double av = __ddiv_rn(__dmul_rn(dt, Ms), __dmul_rn(2.0, Me));
                double vca, vcb;
                if (scheme == 0) {
                    vca = __ddiv_rn(__dsub_rn(1.0, av), __dadd_rn(1.0, av));
                    vcb = __ddiv_rn(dt, __dmul_rn(Me, __dadd_rn(1.0, av)));
                } else {
                    vca = __dsub_rn(1.0, __dmul_rn(2.0, av));
                    vcb = __ddiv_rn(dt, Me);
                }
                if (round_float) {
                    vca = (double)(float)vca;
                    vcb = (double)(float)vcb;
                }
                if (ca) ca[o] = (T)vca;
                cb[o] = (T)vcb;
                if (meps) meps[o] = (T)Me;
            } else {
                if (ca) ca[o] = T(0);
                cb[o] = T(0);
                if (meps) meps[o] = T(0);
            }
            // face normal to a: interior iff q[a] > 0
            if (mu_array) {
                T vch = T(0), vmm = T(0);
                if (!pad && q[a] > 0) {
                    int r[3] = {q[0], q[1], q[2]};
                    r[a] -= 1;
                    const long long rc = (long long)r[0] + (long long)nx * ((long long)r[1] + (long long)ny * r[2]);
                    const double m1 = mu ? (double)mu[cell] : 1.0;
                    const double m2 = mu ? (double)mu[rc] : 1.0;
                    const double mt = __ddiv_rn(2.0, __dadd_rn(__ddiv_rn(1.0, m1), __ddiv_rn(1.0, m2)));
                    const double Mm = __ddiv_rn(__dmul_rn(__dmul_rn(kMu0, mt), area), len);
                    const double q = __ddiv_rn(dt, Mm);
                    vch = (T)(round_float ? (double)(float)q : q);
                    vmm = (T)Mm;
                }
                ch[o] = vch;
                if (mmu) mmu[o] = vmm;
            }
        }
    }
    // uniform mu: one value per component (mu of cell 0 holds for every cell)
    if (!mu_array && blockIdx.x == 0 && threadIdx.x < 3) {
        const int a = threadIdx.x;
        const int b = (a + 1) % 3, cc = (a + 2) % 3;
        const double area = __dmul_rn(d[b], d[cc]);
        const double m1 = mu ? (double)mu[0] : 1.0;
        const double mt = __ddiv_rn(2.0, __dadd_rn(__ddiv_rn(1.0, m1), __ddiv_rn(1.0, m1)));
        const double Mm = __ddiv_rn(__dmul_rn(__dmul_rn(kMu0, mt), area), d[a]);
        const double q = __ddiv_rn(dt, Mm);
        ch[a] = (T)(round_float ? (double)(float)q : q);
        if (mmu) mmu[a] = (T)Mm;
    }
}

__global__ void source_kernel(const fit_source *src, int nsrc, long long base, long long len, double dt,
                              double *amp) {
    const long long total = len * nsrc;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long n = t / nsrc;
        const int s = (int)(t % nsrc);
        const fit_source q = src[s];
        const double tt = ((double)(base + n) + 0.5) * dt;
        double v = 0.0;
        if (q.waveform == FIT_WAVE_GAUSS_SINE) {
            const double x = (tt - q.delay) / q.width;
            v = q.amp * sin(2.0 * kPi * q.f0 * (tt - q.delay)) * exp(-4.0 * x * x);
        } else if (q.waveform == FIT_WAVE_GAUSS) {
            const double x = (tt - q.delay) / q.width;
            v = q.amp * exp(-4.0 * x * x);
        } else if (q.waveform == FIT_WAVE_SINE) {
            v = q.amp * sin(2.0 * kPi * q.f0 * tt);
        }
        amp[t] = v;
    }
}

// zero every entry that is not a degree of freedom, and the row padding
template <typename T>
__global__ void mask_kernel(int nx, int ny, int nz, int pitch, T *e, T *h) {
    const long long ncell = (long long)pitch * ny * nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
         c += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(c % pitch);
        const int j = (int)((c / pitch) % ny);
        const int k = (int)(c / ((long long)pitch * ny));
        const bool pad = i >= nx;
        if (e) {
            if (pad || j == 0 || k == 0) e[c] = T(0);
            if (pad || i == 0 || k == 0) e[ncell + c] = T(0);
            if (pad || i == 0 || j == 0) e[2 * ncell + c] = T(0);
        }
        if (h) {
            if (pad || i == 0) h[c] = T(0);
            if (pad || j == 0) h[ncell + c] = T(0);
            if (pad || k == 0) h[2 * ncell + c] = T(0);
        }
    }
}

template <typename T>
__global__ void accumulate_kernel(long long n, const T *st, double *acc) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x)
        acc[c] += (double)st[c];
}

template <typename T>
__global__ void accumulate_kahan_kernel(long long n, const T *st, float *sum, float *comp) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        const float y = (float)st[c] - comp[c];
        const float s = sum[c];
        const float t = s + y;
        comp[c] = (t - s) - y;
        sum[c] = t;
    }
}

__global__ void kahan_finish_kernel(long long n, const float *sum, const float *comp, double *out) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x)
        out[c] = (double)sum[c] - (double)comp[c];
}

// FP64 compact (3 components) -> pitched hi/lo floats, zeroing entries that
// are not degrees of freedom (e: tangential to a wall; h: normal to it)
__global__ void split_kernel(int nx, int ny, int nz, int pitch, const double *in, float *hi, float *lo, int is_h) {
    const long long ncell = (long long)nx * ny * nz, ncp = (long long)pitch * ny * nz;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < 3 * ncell;
         t += (long long)gridDim.x * blockDim.x) {
        const int a = (int)(t / ncell);
        const long long c = t % ncell;
        const int i = (int)(c % nx);
        const int j = (int)((c / nx) % ny);
        const int k = (int)(c / ((long long)nx * ny));
        const int q[3] = {i, j, k};
        const bool dof = is_h ? q[a] > 0 : (q[(a + 1) % 3] > 0 && q[(a + 2) % 3] > 0);
        const double v = dof ? in[t] : 0.0;
        const float h = (float)v;
        const long long o = (long long)a * ncp + ((long long)k * ny + j) * pitch + i;
        hi[o] = h;
        lo[o] = (float)(v - (double)h);
    }
}

__global__ void join_kernel(int nx, int ny, int nz, int pitch, const float *hi, const float *lo, double *out) {
    const long long ncell = (long long)nx * ny * nz, ncp = (long long)pitch * ny * nz;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < 3 * ncell;
         t += (long long)gridDim.x * blockDim.x) {
        const int a = (int)(t / ncell);
        const long long c = t % ncell;
        const int i = (int)(c % nx);
        const int j = (int)((c / nx) % ny);
        const int k = (int)(c / ((long long)nx * ny));
        const long long o = (long long)a * ncp + ((long long)k * ny + j) * pitch + i;
        out[t] = (double)hi[o] + (double)lo[o];
    }
}

__global__ void accumulate_pairs_kernel(long long n, const float *hi, const float *lo, double *acc) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x)
        acc[c] += (double)hi[c] + (double)lo[c];
}

__global__ void sum_members_kernel(int nmem, long long len, const double *pm, long long stride, double *out) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < len;
         t += (long long)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int m = 0; m < nmem; ++m) s += pm[(long long)m * stride + t];
        out[t] = s;
    }
}


}  // namespace

cudaError_t check_materials(const float *eps, const float *mu, const float *sig, long long ncell,
                            MaterialFlags *out, void *scratch, cudaStream_t s) {
    int *flags = static_cast<int *>(scratch);
    unsigned long long *mnbits = reinterpret_cast<unsigned long long *>(flags + 8);
    int init[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    const double inf = INFINITY;
    memcpy(&init[8], &inf, sizeof(double));
    cudaError_t err = cudaMemcpyAsync(flags, init, sizeof(init), cudaMemcpyHostToDevice, s);
    if (err != cudaSuccess) return err;
    check_kernel<<<grid_for(ncell), kThreads, 0, s>>>(eps, mu, sig, ncell, flags, mnbits);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    int h[10];
    if ((err = cudaMemcpyAsync(h, flags, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return err;
    if ((err = cudaStreamSynchronize(s)) != cudaSuccess) return err;
    out->bad_eps = h[0];
    out->bad_mu = h[1];
    out->bad_sigma = h[2];
    out->mu_nonuniform = h[3];
    out->lossy = h[4];
    double mn;
    memcpy(&mn, &h[8], sizeof(double));
    out->eps_mu_min = mn;
    return cudaSuccess;
}

template <typename T>
cudaError_t build_coeffs(int nx, int ny, int nz, int pitch, const double d[3], const float *eps, const float *mu,
                         const float *sig, double dt, int scheme, bool mu_array, T *ca, T *cb, T *ch, T *meps,
                         T *mmu, cudaStream_t s, bool round_float) {
    const long long n = (long long)pitch * ny * nz;
    coeff_kernel<T><<<grid_for(n), kThreads, 0, s>>>(nx, ny, nz, pitch, d[0], d[1], d[2], eps, mu, sig, dt,
                                                     scheme, mu_array ? 1 : 0, ca, cb, ch, meps, mmu,
                                                     round_float ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t source_table(const fit_source *src_dev, int nsrc, long long base, long long len, double dt,
                         double *amp, cudaStream_t s) {
    if (nsrc <= 0 || len <= 0) return cudaSuccess;
    source_kernel<<<grid_for(len * nsrc), kThreads, 0, s>>>(src_dev, nsrc, base, len, dt, amp);
    return cudaGetLastError();
}

template <typename T>
cudaError_t mask_state(int nx, int ny, int nz, int pitch, T *e, T *h, cudaStream_t s) {
    mask_kernel<T><<<grid_for((long long)pitch * ny * nz), kThreads, 0, s>>>(nx, ny, nz, pitch, e, h);
    return cudaGetLastError();
}

template <typename T>
cudaError_t accumulate_state(long long n6, const T *st, double *acc, cudaStream_t s) {
    accumulate_kernel<T><<<grid_for(n6), kThreads, 0, s>>>(n6, st, acc);
    return cudaGetLastError();
}

template <typename T>
cudaError_t accumulate_state_kahan(long long n6, const T *st, float *sum, float *comp, cudaStream_t s) {
    accumulate_kahan_kernel<T><<<grid_for(n6), kThreads, 0, s>>>(n6, st, sum, comp);
    return cudaGetLastError();
}

cudaError_t kahan_finish(long long n, const float *sum, const float *comp, double *out, cudaStream_t s) {
    kahan_finish_kernel<<<grid_for(n), kThreads, 0, s>>>(n, sum, comp, out);
    return cudaGetLastError();
}

cudaError_t sum_members(int nmem, long long len, const double *pm, long long stride, double *out, cudaStream_t s) {
    if (len <= 0) return cudaSuccess;
    sum_members_kernel<<<grid_for(len), kThreads, 0, s>>>(nmem, len, pm, stride, out);
    return cudaGetLastError();
}

cudaError_t split_pairs(int nx, int ny, int nz, int pitch, const double *in, float *hi, float *lo, int is_h,
                        cudaStream_t s) {
    split_kernel<<<grid_for(3LL * nx * ny * nz), kThreads, 0, s>>>(nx, ny, nz, pitch, in, hi, lo, is_h);
    return cudaGetLastError();
}

cudaError_t join_pairs(int nx, int ny, int nz, int pitch, const float *hi, const float *lo, double *out,
                       cudaStream_t s) {
    join_kernel<<<grid_for(3LL * nx * ny * nz), kThreads, 0, s>>>(nx, ny, nz, pitch, hi, lo, out);
    return cudaGetLastError();
}

cudaError_t accumulate_pairs(long long n, const float *hi, const float *lo, double *acc, cudaStream_t s) {
    accumulate_pairs_kernel<<<grid_for(n), kThreads, 0, s>>>(n, hi, lo, acc);
    return cudaGetLastError();
}

template cudaError_t build_coeffs<float>(int, int, int, int, const double *, const float *, const float *,
                                         const float *, double, int, bool, float *, float *, float *, float *,
                                         float *, cudaStream_t, bool);
template cudaError_t build_coeffs<double>(int, int, int, int, const double *, const float *, const float *,
                                          const float *, double, int, bool, double *, double *, double *,
                                          double *, double *, cudaStream_t, bool);
template cudaError_t mask_state<float>(int, int, int, int, float *, float *, cudaStream_t);
template cudaError_t mask_state<double>(int, int, int, int, double *, double *, cudaStream_t);
template cudaError_t accumulate_state<float>(long long, const float *, double *, cudaStream_t);
template cudaError_t accumulate_state<double>(long long, const double *, double *, cudaStream_t);
template cudaError_t accumulate_state_kahan<float>(long long, const float *, float *, float *, cudaStream_t);
template cudaError_t accumulate_state_kahan<double>(long long, const double *, float *, float *, cudaStream_t);

}  // namespace fitgb
