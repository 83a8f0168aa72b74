/*
 * fit_oracle.c -- plain serial FP64 reference of the FIT leapfrog + ParaExp
 * method (Merkel, Niyonzima, Schoeps, "ParaExp using Leapfrog as Integrator
 * for High-Frequency Electromagnetic Simulations").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or helper with
 * the CUDA library.
 *
 * Layout (canonical FIT indexing, Sec. II): a grid of nx*ny*nz cells has
 * Np = (nx+1)(ny+1)(nz+1) primal points.  Every field component is an array
 * of Np values indexed by the start point of its edge (e), or the lowest
 * corner of the primal face its dual edge pierces (h):
 *     P(i,j,k) = i + (nx+1)*(j + (ny+1)*k),     component a at offset a*Np.
 * e_a(p) is the primal edge p -> p + u_a; it is a degree of freedom ("free")
 * when it lies inside the box and not on the PEC wall (tangential e = 0).
 * h_a(p) sits on the face normal to a with lowest corner p; it is a degree of
 * freedom when the face is interior (the normal flux on a PEC wall stays 0).
 * Entries that are not degrees of freedom are kept at exactly zero.
 *
 * Per-cell material arrays (eps_r, mu_r, sigma) have nx*ny*nz entries,
 * x fastest: c(i,j,k) = i + nx*(j + ny*k).
 *
 * Each function cites the passage of the paper it follows.  Where the paper
 * is silent the reading used is stated at the function.
 *
 * Build: gcc -O2 -std=c99 -ffp-contract=off -fPIC -shared  (no FMA
 * contraction, so x86 and aarch64 hosts give the same bits).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846
#define OR_C0 299792458.0                      /* speed of light [m/s]      */
#define OR_MU0 (4.0e-7 * OR_PI)                /* [H/m], classical value    */
#define OR_EPS0 (1.0 / (OR_MU0 * OR_C0 * OR_C0)) /* [F/m]                    */

typedef struct {
    int nx, ny, nz;       /* cells                                            */
    double d[3];          /* dx, dy, dz [m]                                   */
    double dt;            /* time step [s]                                    */
    const double *ca;     /* 3*Np: e <- ca*e + cb*(C~h - j)                   */
    const double *cb;     /* 3*Np                                             */
    const double *ch;     /* 3*Np: h <- h - ch*(C e)                          */
    const double *meps;   /* 3*Np: diagonal of M_eps (for the energy)         */
    const double *mmu;    /* 3*Np: diagonal of M_mu                           */
    int store32;          /* 1: round every stored e, h to float after its    */
                          /* update (exact arithmetic, FP32 storage): the     */
                          /* error model of a method that keeps its fields in */
                          /* float, used to derive FP32 tolerances            */
} or_grid;

typedef struct { int axis, i, j, k, waveform; double amp, f0, width, delay; } or_source;
typedef struct { int axis, i, j, k; } or_probe;

/* ------------------------------------------------------------------ */
/* indexing                                                             */
/* ------------------------------------------------------------------ */

static long np_of(const or_grid *g) { return (long)(g->nx + 1) * (g->ny + 1) * (g->nz + 1); }

static long pidx(int nx, int ny, int i, int j, int k) {
    return (long)i + (long)(nx + 1) * ((long)j + (long)(ny + 1) * k);
}

static long cidx(int nx, int ny, int i, int j, int k) {
    return (long)i + (long)nx * ((long)j + (long)ny * k);
}

/* Is the primal edge along `a` starting at point q a degree of freedom?
 * It must lie in the box (q_a < n_a) and off the PEC wall (the two other
 * coordinates strictly inside). */
static int edge_free(const int n[3], int a, const int q[3]) {
    int b = (a + 1) % 3, c = (a + 2) % 3;
    if (q[a] < 0 || q[a] >= n[a]) return 0;
    if (q[b] <= 0 || q[b] >= n[b]) return 0;
    if (q[c] <= 0 || q[c] >= n[c]) return 0;
    return 1;
}

/* Is the primal face normal to `a` with lowest corner q interior? */
static int face_interior(const int n[3], int a, const int q[3]) {
    int b = (a + 1) % 3, c = (a + 2) % 3;
    if (q[a] <= 0 || q[a] >= n[a]) return 0;
    if (q[b] < 0 || q[b] >= n[b]) return 0;
    if (q[c] < 0 || q[c] >= n[c]) return 0;
    return 1;
}

/* ------------------------------------------------------------------ */
/* Eq. (cfl): dt_CFL = min_j sqrt(eps_j mu_j / (1/dx^2 + 1/dy^2 + 1/dz^2)) */
/* ------------------------------------------------------------------ */
double oracle_cfl_dt(int nx, int ny, int nz, double dx, double dy, double dz,
                     const float *eps_r, const float *mu_r) {
    double inv = 1.0 / (dx * dx) + 1.0 / (dy * dy) + 1.0 / (dz * dz);
    double best = -1.0;
    long ncell = (long)nx * ny * nz;
    for (long c = 0; c < ncell; ++c) {
        double em = OR_EPS0 * (double)eps_r[c] * OR_MU0 * (mu_r ? (double)mu_r[c] : 1.0);
        double t = sqrt(em / inv);
        if (best < 0.0 || t < best) best = t;
    }
    return best;
}

/* ------------------------------------------------------------------ */
/* Material matrices and update coefficients (Sec. II, eq. maxwell_grid3; */
/* leapfrog coefficients of Sec. II-A).                                  */
/*                                                                        */
/* Readings (the paper is silent on these):                               */
/*  - M_eps on a primal edge: eps0 * (area-weighted mean of eps_r over the */
/*    four cells around the edge) * (dual facet area) / (edge length).     */
/*    On a uniform grid every cell holds a quarter of the dual facet, so   */
/*    the weights are 1/4.  M_sigma: the same with sigma.                  */
/*  - M_mu on a primal face: mu0 * (harmonic mean of mu_r of the two cells */
/*    sharing the face, the cells being in series along the dual edge) *   */
/*    (face area) / (dual edge length).                                    */
/*  - sigma enters with e at the half step, (e^n + e^{n+1})/2:             */
/*      a  = dt M_sigma / (2 M_eps),                                       */
/*      ca = (1 - a)/(1 + a),  cb = dt / (M_eps (1 + a)).                  */
/*    sigma_scheme = 1 takes e^n instead: ca = 1 - 2a, cb = dt / M_eps.    */
/*  - ch = dt / M_mu.                                                      */
/*  - Entries that are not degrees of freedom get all coefficients 0.      */
/*  - round32 != 0 rounds ca, cb, ch to the nearest float (the FP32 field */
/*    path stores its coefficients in float).                            */
/* ------------------------------------------------------------------ */
int oracle_coeffs(int nx, int ny, int nz, double dx, double dy, double dz,
                  const float *eps_r, const float *mu_r, const float *sigma,
                  double dt, int sigma_scheme, int round32,
                  double *ca, double *cb, double *ch,
                  double *meps, double *msig, double *mmu) {
    int n[3] = {nx, ny, nz};
    double d[3] = {dx, dy, dz};
    long Np = (long)(nx + 1) * (ny + 1) * (nz + 1);
    if (nx < 1 || ny < 1 || nz < 1 || !(dt > 0.0)) return -1;
    memset(ca, 0, sizeof(double) * 3 * Np);
    memset(cb, 0, sizeof(double) * 3 * Np);
    memset(ch, 0, sizeof(double) * 3 * Np);
    memset(meps, 0, sizeof(double) * 3 * Np);
    memset(msig, 0, sizeof(double) * 3 * Np);
    memset(mmu, 0, sizeof(double) * 3 * Np);
    for (int a = 0; a < 3; ++a) {
        int b = (a + 1) % 3, c = (a + 2) % 3;
        double len = d[a], area = d[b] * d[c];
        for (int k = 0; k <= nz; ++k)
            for (int j = 0; j <= ny; ++j)
                for (int i = 0; i <= nx; ++i) {
                    int q[3] = {i, j, k};
                    long p = (long)a * Np + pidx(nx, ny, i, j, k);
                    if (edge_free(n, a, q)) {
                        /* the four cells around the edge: q - sb*u_b - sc*u_c */
                        double esum = 0.0, ssum = 0.0;
                        for (int sb = 0; sb < 2; ++sb)
                            for (int sc = 0; sc < 2; ++sc) {
                                int r[3] = {q[0], q[1], q[2]};
                                r[b] -= sb;
                                r[c] -= sc;
                                long cc = cidx(nx, ny, r[0], r[1], r[2]);
                                esum += (double)eps_r[cc];
                                ssum += sigma ? (double)sigma[cc] : 0.0;
                            }
                        double ebar = esum / 4.0, sbar = ssum / 4.0;
                        double Me = OR_EPS0 * ebar * area / len;
                        double Ms = sbar * area / len;
                        double av = dt * Ms / (2.0 * Me);
                        double vca, vcb;
                        if (sigma_scheme == 0) {
                            vca = (1.0 - av) / (1.0 + av);
                            vcb = dt / (Me * (1.0 + av));
                        } else {
                            vca = 1.0 - 2.0 * av;
                            vcb = dt / Me;
                        }
                        if (round32) { vca = (double)(float)vca; vcb = (double)(float)vcb; }
                        ca[p] = vca;
                        cb[p] = vcb;
                        meps[p] = Me;
                        msig[p] = Ms;
                    }
                    if (face_interior(n, a, q)) {
                        /* the two cells sharing the face: q and q - u_a */
                        int r[3] = {q[0], q[1], q[2]};
                        r[a] -= 1;
                        double m1 = mu_r ? (double)mu_r[cidx(nx, ny, q[0], q[1], q[2])] : 1.0;
                        double m2 = mu_r ? (double)mu_r[cidx(nx, ny, r[0], r[1], r[2])] : 1.0;
                        double mtil = 2.0 / (1.0 / m1 + 1.0 / m2);
                        double Mm = OR_MU0 * mtil * area / len;
                        double vch = dt / Mm;
                        if (round32) vch = (double)(float)vch;
                        ch[p] = vch;
                        mmu[p] = Mm;
                    }
                }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Source waveforms (edge current i(t) in A).                            */
/*  0: Gaussian-modulated sine  amp*sin(2 pi f0 (t-delay))*exp(-4((t-delay)/width)^2) */
/*  1: Gaussian pulse, eq. (line_current): amp*exp(-4((t-delay)/width)^2) */
/*  2: sine  amp*sin(2 pi f0 t)                                          */
/* ------------------------------------------------------------------ */
double oracle_waveform(int waveform, double amp, double f0, double width, double delay, double t) {
    double x;
    switch (waveform) {
    case 0:
        x = (t - delay) / width;
        return amp * sin(2.0 * OR_PI * f0 * (t - delay)) * exp(-4.0 * x * x);
    case 1:
        x = (t - delay) / width;
        return amp * exp(-4.0 * x * x);
    case 2:
        return amp * sin(2.0 * OR_PI * f0 * t);
    default:
        return 0.0;
    }
}

/* ------------------------------------------------------------------ */
/* (C e)_a on the face normal to a with corner q (Sec. II, eq. maxwell_grid1): */
/* the circulation of e around the face, counter-clockwise seen from +a:   */
/*   e_b(q) + e_c(q+u_b) - e_b(q+u_c) - e_c(q),  (a,b,c) cyclic.           */
/* ------------------------------------------------------------------ */
static double curl_e(const double *e, int nx, int ny, long Np, int a, const int q[3]) {
    int b = (a + 1) % 3, c = (a + 2) % 3;
    int qb[3] = {q[0], q[1], q[2]}, qc[3] = {q[0], q[1], q[2]};
    qb[b] += 1;
    qc[c] += 1;
    return e[(long)b * Np + pidx(nx, ny, q[0], q[1], q[2])]
         + e[(long)c * Np + pidx(nx, ny, qb[0], qb[1], qb[2])]
         - e[(long)b * Np + pidx(nx, ny, qc[0], qc[1], qc[2])]
         - e[(long)c * Np + pidx(nx, ny, q[0], q[1], q[2])];
}

/* (C~ h)_a on the primal edge along a starting at q, C~ = C^T (Sec. II):
 *   h_c(q) - h_c(q-u_b) - h_b(q) + h_b(q-u_c). */
static double curl_h(const double *h, int nx, int ny, long Np, int a, const int q[3]) {
    int b = (a + 1) % 3, c = (a + 2) % 3;
    int qb[3] = {q[0], q[1], q[2]}, qc[3] = {q[0], q[1], q[2]};
    qb[b] -= 1;
    qc[c] -= 1;
    return h[(long)c * Np + pidx(nx, ny, q[0], q[1], q[2])]
         - h[(long)c * Np + pidx(nx, ny, qb[0], qb[1], qb[2])]
         - h[(long)b * Np + pidx(nx, ny, q[0], q[1], q[2])]
         + h[(long)b * Np + pidx(nx, ny, qc[0], qc[1], qc[2])];
}

static int check_edge(const or_grid *g, int axis, int i, int j, int k, int need_free) {
    int n[3] = {g->nx, g->ny, g->nz};
    int q[3] = {i, j, k};
    if (axis < 0 || axis > 2) return 0;
    for (int t = 0; t < 3; ++t)
        if (q[t] < 0 || q[t] > n[t]) return 0;
    if (q[axis] >= n[axis]) return 0;
    if (need_free && !edge_free(n, axis, q)) return 0;
    return 1;
}

/* ------------------------------------------------------------------ */
/* Leapfrog (Sec. II-A).  State at step n: (e^n, h^{n-1/2}).  Step n:     */
/*   h^{n+1/2} = h^{n-1/2} - ch * (C e^n)                                  */
/*   e^{n+1}   = ca * e^n + cb * (C~ h^{n+1/2} - j^{n+1/2})                */
/* with j^{n+1/2} = i((step0 + n + 1/2) dt) on each source edge while the */
/* absolute step lies in [src_lo, src_hi).                                */
/* Readings: the H update applies the primal curl C to e (the printed     */
/* update shows the dual curl, which cannot act on e); the current enters */
/* with a minus sign (Ampere: C~h = d/dt d + j); h is updated first, so  */
/* the order is the one of the printed scheme shifted by half a step.     */
/* Outputs per step n (n = 0..nsteps-1):                                  */
/*   probe_out[n*nprb + p] = e^{n+1} on probe edge p (volts), if non-NULL  */
/*   energy_out[n] = W^n = e^n' Meps e^n + h^{n-1/2}' Mmu h^{n+1/2}        */
/*   (the interleaved discrete energy of eq. (energy)), if non-NULL.       */
/* e and h (3*Np each) hold the initial state on entry and the final one  */
/* on exit.  Returns 0, or -1 on a bad source/probe.                      */
/* ------------------------------------------------------------------ */
int oracle_leapfrog(const or_grid *g, long nsteps, long step0, long src_lo, long src_hi,
                    const or_source *src, int nsrc, const or_probe *prb, int nprb,
                    double *probe_out, double *energy_out, double *e, double *h) {
    int nx = g->nx, ny = g->ny, nz = g->nz;
    int n[3] = {nx, ny, nz};
    long Np = np_of(g);
    for (int s = 0; s < nsrc; ++s)
        if (!check_edge(g, src[s].axis, src[s].i, src[s].j, src[s].k, 1)) return -1;
    for (int p = 0; p < nprb; ++p)
        if (!check_edge(g, prb[p].axis, prb[p].i, prb[p].j, prb[p].k, 0)) return -1;

    for (long step = 0; step < nsteps; ++step) {
        long abs_step = step0 + step;
        double w_e = 0.0, w_h = 0.0;
        /* electric part of W^n, before e changes */
        if (energy_out)
            for (long t = 0; t < 3 * Np; ++t) w_e += g->meps[t] * e[t] * e[t];
        /* H half step: h depends on e only, so the update can be in place */
        for (int a = 0; a < 3; ++a)
            for (int k = 0; k <= nz; ++k)
                for (int j = 0; j <= ny; ++j)
                    for (int i = 0; i <= nx; ++i) {
                        int q[3] = {i, j, k};
                        if (!face_interior(n, a, q)) continue;
                        long p = (long)a * Np + pidx(nx, ny, i, j, k);
                        double hold = h[p];
                        double hnew = hold - g->ch[p] * curl_e(e, nx, ny, Np, a, q);
                        if (g->store32) hnew = (double)(float)hnew;
                        w_h += g->mmu[p] * hold * hnew;
                        h[p] = hnew;
                    }
        /* E half step: e depends on the new h only */
        for (int a = 0; a < 3; ++a)
            for (int k = 0; k <= nz; ++k)
                for (int j = 0; j <= ny; ++j)
                    for (int i = 0; i <= nx; ++i) {
                        int q[3] = {i, j, k};
                        if (!edge_free(n, a, q)) continue;
                        long p = (long)a * Np + pidx(nx, ny, i, j, k);
                        double jsrc = 0.0;
                        if (abs_step >= src_lo && abs_step < src_hi)
                            for (int s = 0; s < nsrc; ++s)
                                if (src[s].axis == a && src[s].i == i && src[s].j == j && src[s].k == k)
                                    jsrc += oracle_waveform(src[s].waveform, src[s].amp, src[s].f0,
                                                            src[s].width, src[s].delay,
                                                            ((double)abs_step + 0.5) * g->dt);
                        e[p] = g->ca[p] * e[p] + g->cb[p] * (curl_h(h, nx, ny, Np, a, q) - jsrc);
                        if (g->store32) e[p] = (double)(float)e[p];
                    }
        if (probe_out)
            for (int p = 0; p < nprb; ++p)
                probe_out[step * nprb + p] =
                    e[(long)prb[p].axis * Np + pidx(nx, ny, prb[p].i, prb[p].j, prb[p].k)];
        if (energy_out) energy_out[step] = w_e + w_h;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* ParaExp (Sec. III, Algorithm 1, eqs. solution-particular-paraexp,     */
/* solution-homogeneous-paraexp, solution-particular-para, averaging1/2). */
/* The interval of steps [win[0], win[K]) is cut into K windows           */
/* [win[j-1], win[j]).  Member j (j = 1..K) starts from the zero state at */
/* step win[j-1] and carries the source only inside its window: that is  */
/* v_j.  Continued source-free to win[K] it is w_{j+1}, the homogeneous   */
/* problem started from v_j(T_j), here integrated by leapfrog as well.    */
/* w_1 propagates the initial value (e0, h0) (zero when both are NULL).   */
/* The superposition sums all members at every step; e at integer steps   */
/* and h at half steps, so the staggering of the leapfrog is kept and no  */
/* similarity transform is needed (the members are in untransformed     */
/* voltages).  Members are run one after another, sums are in FP64.       */
/* probe_out: (win[K]-win[0])*nprb, index m <-> absolute step win[0]+m+1.  */
/* e_fin, h_fin (3*Np): e^{win[K]} and h^{win[K]-1/2} of the sum.         */
/* ------------------------------------------------------------------ */
int oracle_paraexp(const or_grid *g, int K, const long *win,
                   const or_source *src, int nsrc, const or_probe *prb, int nprb,
                   const double *e0, const double *h0,
                   double *probe_out, double *e_fin, double *h_fin) {
    long Np = np_of(g);
    long nt = win[K] - win[0];
    if (K < 1 || nt < 0) return -1;
    for (int j = 1; j <= K; ++j)
        if (win[j] < win[j - 1]) return -1;
    double *e = (double *)malloc(sizeof(double) * 3 * Np);
    double *h = (double *)malloc(sizeof(double) * 3 * Np);
    double *pr = (double *)malloc(sizeof(double) * (size_t)(nt > 0 ? nt : 1) * (nprb > 0 ? nprb : 1));
    int rc = 0;
    if (!e || !h || !pr) { rc = -2; goto done; }
    if (probe_out) memset(probe_out, 0, sizeof(double) * (size_t)nt * nprb);
    memset(e_fin, 0, sizeof(double) * 3 * Np);
    memset(h_fin, 0, sizeof(double) * 3 * Np);
    for (int j = (e0 || h0) ? 0 : 1; j <= K; ++j) {
        long start, lo, hi;
        if (j == 0) {               /* w_1: homogeneous propagation of u0 */
            if (e0) memcpy(e, e0, sizeof(double) * 3 * Np); else memset(e, 0, sizeof(double) * 3 * Np);
            if (h0) memcpy(h, h0, sizeof(double) * 3 * Np); else memset(h, 0, sizeof(double) * 3 * Np);
            start = win[0]; lo = 0; hi = 0;
        } else {                    /* v_j, then w_{j+1} */
            memset(e, 0, sizeof(double) * 3 * Np);
            memset(h, 0, sizeof(double) * 3 * Np);
            start = win[j - 1]; lo = win[j - 1]; hi = win[j];
        }
        long ns = win[K] - start;
        rc = oracle_leapfrog(g, ns, start, lo, hi, src, nsrc, prb, nprb, pr, NULL, e, h);
        if (rc) goto done;
        if (probe_out) {
            long off = start - win[0];
            for (long m = 0; m < ns; ++m)
                for (int p = 0; p < nprb; ++p)
                    probe_out[(off + m) * nprb + p] += pr[m * nprb + p];
        }
        for (long t = 0; t < 3 * Np; ++t) { e_fin[t] += e[t]; h_fin[t] += h[t]; }
    }
done:
    free(e); free(h); free(pr);
    return rc;
}

/* length of a probe's edge: the grid step along its axis, or on a graded */
/* grid the size of the cell the edge runs through                          */
static double probe_len(const or_grid *g, const double *const *ds, const or_probe *p) {
    if (!ds) return g->d[p->axis];
    const int q[3] = {p->i, p->j, p->k};
    return ds[p->axis][q[p->axis]];
}

/* graded chain rule of one free edge (a, q) at offset p: adds             */
/* w * (gca dca/dE + gcb dcb/dE) to each of its four cells (see            */
/* oracle_adjoint_graded)                                                   */
static void graded_chain(const or_grid *g, const double *const *ds, const float *eps_r, const float *sigma,
                         int sigma_scheme, int a, const int q[3], long p, double gca, double gcb,
                         double *grad) {
    int nx = g->nx, ny = g->ny;
    int b = (a + 1) % 3, c = (a + 2) % 3;
    double E = 0.0, S = 0.0, w[4];
    long cells[4];
    int nc = 0;
    for (int sb = 0; sb < 2; ++sb)
        for (int sc = 0; sc < 2; ++sc) {
            int r[3] = {q[0], q[1], q[2]};
            r[b] -= sb;
            r[c] -= sc;
            long cc = cidx(nx, ny, r[0], r[1], r[2]);
            w[nc] = ds[b][r[b]] * ds[c][r[c]] / 4.0;
            E += (double)eps_r[cc] * w[nc];
            S += (sigma ? (double)sigma[cc] : 0.0) * w[nc];
            cells[nc++] = cc;
        }
    double s = g->dt * S / (2.0 * OR_EPS0);
    double dca, dcb;
    if (sigma_scheme == 0) {
        dca = 2.0 * s / ((E + s) * (E + s));
        dcb = -g->cb[p] / (E + s);
    } else {
        dca = 2.0 * s / (E * E);
        dcb = -g->cb[p] / E;
    }
    double dJ = gca * dca + gcb * dcb;
    for (int t = 0; t < 4; ++t) grad[cells[t]] += w[t] * dJ;
}

/* ------------------------------------------------------------------ */
/* Adjoint gradient of the probe functional                              */
/*   J = sum_{n=1..N} sum_p (e_p^n / L_p)^2      (L_p: probe edge length)  */
/* with respect to the per-cell eps_r.  The reverse sweep is the exact    */
/* transpose of the leapfrog step above (derived from Sec. II-A):         */
/*   lam_e^N = dJ/de^N, lam_h = 0, and for n = N-1 .. 0:                  */
/*     g_ca += lam_e (.) e^n                                              */
/*     g_cb += lam_e (.) (C~ h^{n+1/2} - j^{n+1/2})                       */
/*     lam_h += C (cb (.) lam_e)                                          */
/*     lam_e  = ca (.) lam_e - C~ (ch (.) lam_h) + dJ/de^n   (n >= 1)     */
/* then the chain rule through ca(eps_bar), cb(eps_bar) of oracle_coeffs  */
/* (s = dt sigma_bar / (2 eps0)):                                         */
/*   scheme 0: dca/deps_bar = 2s/(eps_bar+s)^2, dcb/deps_bar = -cb/(eps_bar+s) */
/*   scheme 1: dca/deps_bar = 2s/eps_bar^2,     dcb/deps_bar = -cb/eps_bar   */
/* and d eps_bar / d eps_r(cell) = 1/4 for each of the four cells around a */
/* free edge.  Every state is kept in memory (no checkpointing).          */
/* grad: nx*ny*nz doubles.  The coefficients in g are used as given (they */
/* may be float-rounded); the derivative is that of the unrounded map.    */
/* ------------------------------------------------------------------ */
/* ds: NULL on a uniform grid, else the per-cell sizes {dx, dy, dz} of a    */
/* graded grid (the chain rule of oracle_adjoint_graded below).            */
static int adjoint_core(const or_grid *g, const double *const *ds, const float *eps_r, const float *sigma,
                        int sigma_scheme, long nsteps, long step0, const or_source *src, int nsrc,
                        const or_probe *prb, int nprb, double *J_out, double *grad) {
    int nx = g->nx, ny = g->ny, nz = g->nz;
    int n[3] = {nx, ny, nz};
    long Np = np_of(g);
    long S = 3 * Np;
    int rc = 0;
    if (nsteps < 1) return -1;
    for (int s = 0; s < nsrc; ++s)
        if (!check_edge(g, src[s].axis, src[s].i, src[s].j, src[s].k, 1)) return -1;
    for (int p = 0; p < nprb; ++p)
        if (!check_edge(g, prb[p].axis, prb[p].i, prb[p].j, prb[p].k, 0)) return -1;
    /* E[n] = e^n for n = 0..N ; H[n] = h^{n+1/2} for n = 0..N-1 */
    double *E = (double *)calloc((size_t)(nsteps + 1) * S, sizeof(double));
    double *H = (double *)calloc((size_t)nsteps * S, sizeof(double));
    double *le = (double *)calloc(S, sizeof(double));
    double *lh = (double *)calloc(S, sizeof(double));
    double *tmp = (double *)calloc(S, sizeof(double));
    double *gca = (double *)calloc(S, sizeof(double));
    double *gcb = (double *)calloc(S, sizeof(double));
    double *e = (double *)calloc(S, sizeof(double));
    double *h = (double *)calloc(S, sizeof(double));
    if (!E || !H || !le || !lh || !tmp || !gca || !gcb || !e || !h) { rc = -2; goto done; }

    /* forward sweep, keeping every state */
    {
        double J = 0.0;
        for (long st = 0; st < nsteps; ++st) {
            rc = oracle_leapfrog(g, 1, step0 + st, step0, step0 + nsteps, src, nsrc, NULL, 0,
                                 NULL, NULL, e, h);
            if (rc) goto done;
            memcpy(H + (size_t)st * S, h, sizeof(double) * S);
            memcpy(E + (size_t)(st + 1) * S, e, sizeof(double) * S);
            for (int p = 0; p < nprb; ++p) {
                double L = probe_len(g, ds, &prb[p]);
                double v = e[(long)prb[p].axis * Np + pidx(nx, ny, prb[p].i, prb[p].j, prb[p].k)] / L;
                J += v * v;
            }
        }
        *J_out = J;
    }

    /* lam_e^N = dJ/de^N */
    for (int p = 0; p < nprb; ++p) {
        double L = probe_len(g, ds, &prb[p]);
        long t = (long)prb[p].axis * Np + pidx(nx, ny, prb[p].i, prb[p].j, prb[p].k);
        le[t] += 2.0 * E[(size_t)nsteps * S + t] / (L * L);
    }
    for (long st = nsteps - 1; st >= 0; --st) {
        const double *en = E + (size_t)st * S;
        const double *hp = H + (size_t)st * S;
        long abs_step = step0 + st;
        /* parameter gradients */
        for (int a = 0; a < 3; ++a)
            for (int k = 0; k <= nz; ++k)
                for (int j = 0; j <= ny; ++j)
                    for (int i = 0; i <= nx; ++i) {
                        int q[3] = {i, j, k};
                        if (!edge_free(n, a, q)) continue;
                        long p = (long)a * Np + pidx(nx, ny, i, j, k);
                        double jsrc = 0.0;
                        for (int s = 0; s < nsrc; ++s)
                            if (src[s].axis == a && src[s].i == i && src[s].j == j && src[s].k == k)
                                jsrc += oracle_waveform(src[s].waveform, src[s].amp, src[s].f0,
                                                        src[s].width, src[s].delay,
                                                        ((double)abs_step + 0.5) * g->dt);
                        gca[p] += le[p] * en[p];
                        gcb[p] += le[p] * (curl_h(hp, nx, ny, Np, a, q) - jsrc);
                    }
        /* lam_h += C (cb lam_e) */
        for (long t = 0; t < S; ++t) tmp[t] = g->cb[t] * le[t];
        for (int a = 0; a < 3; ++a)
            for (int k = 0; k <= nz; ++k)
                for (int j = 0; j <= ny; ++j)
                    for (int i = 0; i <= nx; ++i) {
                        int q[3] = {i, j, k};
                        if (!face_interior(n, a, q)) continue;
                        long p = (long)a * Np + pidx(nx, ny, i, j, k);
                        lh[p] += curl_e(tmp, nx, ny, Np, a, q);
                    }
        /* lam_e = ca lam_e - C~ (ch lam_h) + dJ/de^n */
        for (long t = 0; t < S; ++t) tmp[t] = g->ch[t] * lh[t];
        for (int a = 0; a < 3; ++a)
            for (int k = 0; k <= nz; ++k)
                for (int j = 0; j <= ny; ++j)
                    for (int i = 0; i <= nx; ++i) {
                        int q[3] = {i, j, k};
                        if (!edge_free(n, a, q)) continue;
                        long p = (long)a * Np + pidx(nx, ny, i, j, k);
                        le[p] = g->ca[p] * le[p] - curl_h(tmp, nx, ny, Np, a, q);
                    }
        if (st >= 1)
            for (int p = 0; p < nprb; ++p) {
                double L = probe_len(g, ds, &prb[p]);
                long t = (long)prb[p].axis * Np + pidx(nx, ny, prb[p].i, prb[p].j, prb[p].k);
                le[t] += 2.0 * en[t] / (L * L);
            }
    }

    /* chain rule to eps_bar per edge, then scatter to the cells */
    memset(grad, 0, sizeof(double) * (size_t)nx * ny * nz);
    for (int a = 0; a < 3; ++a) {
        int b = (a + 1) % 3, c = (a + 2) % 3;
        for (int k = 0; k <= nz; ++k)
            for (int j = 0; j <= ny; ++j)
                for (int i = 0; i <= nx; ++i) {
                    int q[3] = {i, j, k};
                    if (!edge_free(n, a, q)) continue;
                    long p = (long)a * Np + pidx(nx, ny, i, j, k);
                    double esum = 0.0, ssum = 0.0;
                    long cells[4];
                    int nc = 0;
                    for (int sb = 0; sb < 2; ++sb)
                        for (int sc = 0; sc < 2; ++sc) {
                            int r[3] = {q[0], q[1], q[2]};
                            r[b] -= sb;
                            r[c] -= sc;
                            long cc = cidx(nx, ny, r[0], r[1], r[2]);
                            cells[nc++] = cc;
                            esum += (double)eps_r[cc];
                            ssum += sigma ? (double)sigma[cc] : 0.0;
                        }
                    if (ds) {
                        graded_chain(g, ds, eps_r, sigma, sigma_scheme, a, q, p, gca[p], gcb[p], grad);
                        continue;
                    }
                    double ebar = esum / 4.0, sbar = ssum / 4.0;
                    double s = g->dt * sbar / (2.0 * OR_EPS0);
                    double dca, dcb;
                    if (sigma_scheme == 0) {
                        dca = 2.0 * s / ((ebar + s) * (ebar + s));
                        dcb = -g->cb[p] / (ebar + s);
                    } else {
                        dca = 2.0 * s / (ebar * ebar);
                        dcb = -g->cb[p] / ebar;
                    }
                    double dJ = gca[p] * dca + gcb[p] * dcb;
                    for (int t = 0; t < 4; ++t) grad[cells[t]] += 0.25 * dJ;
                }
    }
done:
    free(E); free(H); free(le); free(lh); free(tmp); free(gca); free(gcb); free(e); free(h);
    return rc;
}

int oracle_adjoint(const or_grid *g, const float *eps_r, const float *sigma, int sigma_scheme,
                   long nsteps, long step0, const or_source *src, int nsrc,
                   const or_probe *prb, int nprb, double *J_out, double *grad) {
    return adjoint_core(g, NULL, eps_r, sigma, sigma_scheme, nsteps, step0, src, nsrc, prb, nprb, J_out, grad);
}

/* ------------------------------------------------------------------ */
/* The adjoint gradient on a graded grid (g built by oracle_coeffs_graded */
/* from the same sizes).  The reverse sweep is the one above.  J uses the */
/* probe edge's own length, d_a at its index along a.  The chain rule      */
/* follows the graded material matrices: with the weight                   */
/* w = d_b d_c / 4 of each of the four cells around an edge (the part of   */
/* the dual facet inside it), E = sum w eps_r, S = sum w sigma and         */
/* s = dt S / (2 eps0), the coefficients are                               */
/*   scheme 0: ca = (E - s)/(E + s), cb = dt L / (eps0 (E + s))            */
/*   scheme 1: ca = 1 - 2 s/E,       cb = dt L / (eps0 E)                  */
/* so dca/dE = 2s/(E+s)^2, dcb/dE = -cb/(E+s) (scheme 1: 2s/E^2, -cb/E)    */
/* and dE/deps_r(cell) = w of that cell.                                   */
/* ------------------------------------------------------------------ */
int oracle_adjoint_graded(const or_grid *g, const double *dx, const double *dy, const double *dz,
                          const float *eps_r, const float *sigma, int sigma_scheme,
                          long nsteps, long step0, const or_source *src, int nsrc,
                          const or_probe *prb, int nprb, double *J_out, double *grad) {
    const double *ds[3] = {dx, dy, dz};
    if (!dx || !dy || !dz) return -1;
    return adjoint_core(g, ds, eps_r, sigma, sigma_scheme, nsteps, step0, src, nsrc, prb, nprb, J_out, grad);
}

/* Physical constants as used above, exported so a caller can state them. */
void oracle_constants(double *c0, double *mu0, double *eps0) {
    *c0 = OR_C0;
    *mu0 = OR_MU0;
    *eps0 = OR_EPS0;
}

/* ------------------------------------------------------------------ */
/* The skew-symmetric system matrix of eq. (FIT_ode_2) acting on the      */
/* transformed unknowns u = [M_mu^{1/2} h, M_eps^{1/2} e] (Sec. II):       */
/*   (A u)_h = -M_mu^{-1/2}  C  M_eps^{-1/2} u_e                           */
/*   (A u)_e =  M_eps^{-1/2} C~ M_mu^{-1/2}  u_h                           */
/* The sign of the first block row follows the printed A, which agrees   */
/* with the curl equations (C e = -db/dt, C~h = dd/dt + j) read above;    */
/* the printed K carries the opposite signs in both block rows.           */
/* Only degrees of freedom take part (PEC): ue and uh must be zero off     */
/* them and the outputs are zero there.  Lossless grids only (M_sigma is  */
/* not part of A).  ue, uh, oe, oh: 3*Np each, canonical layout.          */
/* ------------------------------------------------------------------ */
int oracle_apply_A(const or_grid *g, const double *ue, const double *uh, double *oe, double *oh) {
    int nx = g->nx, ny = g->ny, nz = g->nz;
    int n[3] = {nx, ny, nz};
    long Np = np_of(g);
    double *te = (double *)calloc((size_t)(3 * Np), sizeof(double));
    double *th = (double *)calloc((size_t)(3 * Np), sizeof(double));
    if (!te || !th) { free(te); free(th); return -2; }
    /* te = M_eps^{-1/2} u_e,  th = M_mu^{-1/2} u_h */
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k <= nz; ++k)
            for (int j = 0; j <= ny; ++j)
                for (int i = 0; i <= nx; ++i) {
                    int q[3] = {i, j, k};
                    long p = (long)a * Np + pidx(nx, ny, i, j, k);
                    if (edge_free(n, a, q)) te[p] = ue[p] / sqrt(g->meps[p]);
                    if (face_interior(n, a, q)) th[p] = uh[p] / sqrt(g->mmu[p]);
                }
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k <= nz; ++k)
            for (int j = 0; j <= ny; ++j)
                for (int i = 0; i <= nx; ++i) {
                    int q[3] = {i, j, k};
                    long p = (long)a * Np + pidx(nx, ny, i, j, k);
                    oe[p] = edge_free(n, a, q) ? curl_h(th, nx, ny, Np, a, q) / sqrt(g->meps[p]) : 0.0;
                    oh[p] = face_interior(n, a, q) ? -curl_e(te, nx, ny, Np, a, q) / sqrt(g->mmu[p]) : 0.0;
                }
    free(te); free(th);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Graded (tensor-product) grids: cell (i,j,k) has the size             */
/* dx[i] x dy[j] x dz[k].  Eq. (cfl) takes each cell's own sizes:        */
/*   dt_CFL = min_j sqrt(eps_j mu_j / (1/dx_j^2 + 1/dy_j^2 + 1/dz_j^2)). */
/* ------------------------------------------------------------------ */
double oracle_cfl_dt_graded(int nx, int ny, int nz, const double *dx, const double *dy, const double *dz,
                            const float *eps_r, const float *mu_r) {
    double best = -1.0;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                long c = cidx(nx, ny, i, j, k);
                double inv = 1.0 / (dx[i] * dx[i]) + 1.0 / (dy[j] * dy[j]) + 1.0 / (dz[k] * dz[k]);
                double em = OR_EPS0 * (double)eps_r[c] * OR_MU0 * (mu_r ? (double)mu_r[c] : 1.0);
                double t = sqrt(em / inv);
                if (best < 0.0 || t < best) best = t;
            }
    return best;
}

/* ------------------------------------------------------------------ */
/* Material matrices on a graded grid (Sec. II, eq. maxwell_grid3), the   */
/* same readings as oracle_coeffs with the local sizes:                   */
/*  - M_eps of the edge along a at q: eps0 / L * sum over the four cells   */
/*    around it of eps_r * (d_b/2)(d_c/2) (the part of the dual facet     */
/*    inside each cell), L = d_a[q_a]: the area-weighted mean times the   */
/*    dual area over the length.  M_sigma likewise.                        */
/*  - M_mu of the face normal to a at q: mu0 * A / s with A = d_b[q_b]     */
/*    d_c[q_c] and s = (d_a[q_a-1]/2)/mu_r(q - u_a) + (d_a[q_a]/2)/mu_r(q):*/
/*    the two halves of the dual edge in series (the length-weighted      */
/*    harmonic mean of mu_r).                                              */
/*  - ca, cb, ch as in oracle_coeffs.                                      */
/* ------------------------------------------------------------------ */
int oracle_coeffs_graded(int nx, int ny, int nz, const double *dx, const double *dy, const double *dz,
                         const float *eps_r, const float *mu_r, const float *sigma,
                         double dt, int sigma_scheme, int round32,
                         double *ca, double *cb, double *ch,
                         double *meps, double *msig, double *mmu) {
    int n[3] = {nx, ny, nz};
    const double *ds[3] = {dx, dy, dz};
    long Np = (long)(nx + 1) * (ny + 1) * (nz + 1);
    if (nx < 1 || ny < 1 || nz < 1 || !(dt > 0.0)) return -1;
    memset(ca, 0, sizeof(double) * 3 * Np);
    memset(cb, 0, sizeof(double) * 3 * Np);
    memset(ch, 0, sizeof(double) * 3 * Np);
    memset(meps, 0, sizeof(double) * 3 * Np);
    memset(msig, 0, sizeof(double) * 3 * Np);
    memset(mmu, 0, sizeof(double) * 3 * Np);
    for (int a = 0; a < 3; ++a) {
        int b = (a + 1) % 3, c = (a + 2) % 3;
        for (int k = 0; k <= nz; ++k)
            for (int j = 0; j <= ny; ++j)
                for (int i = 0; i <= nx; ++i) {
                    int q[3] = {i, j, k};
                    long p = (long)a * Np + pidx(nx, ny, i, j, k);
                    if (edge_free(n, a, q)) {
                        double len = ds[a][q[a]];
                        double esum = 0.0, ssum = 0.0;
                        for (int sb = 0; sb < 2; ++sb)
                            for (int sc = 0; sc < 2; ++sc) {
                                int r[3] = {q[0], q[1], q[2]};
                                r[b] -= sb;
                                r[c] -= sc;
                                long cc = cidx(nx, ny, r[0], r[1], r[2]);
                                double w = ds[b][r[b]] * ds[c][r[c]] / 4.0;
                                esum += (double)eps_r[cc] * w;
                                ssum += (sigma ? (double)sigma[cc] : 0.0) * w;
                            }
                        double Me = OR_EPS0 * esum / len;
                        double Ms = ssum / len;
                        double av = dt * Ms / (2.0 * Me);
                        double vca, vcb;
                        if (sigma_scheme == 0) {
                            vca = (1.0 - av) / (1.0 + av);
                            vcb = dt / (Me * (1.0 + av));
                        } else {
                            vca = 1.0 - 2.0 * av;
                            vcb = dt / Me;
                        }
                        if (round32) { vca = (double)(float)vca; vcb = (double)(float)vcb; }
                        ca[p] = vca;
                        cb[p] = vcb;
                        meps[p] = Me;
                        msig[p] = Ms;
                    }
                    if (face_interior(n, a, q)) {
                        int r[3] = {q[0], q[1], q[2]};
                        r[a] -= 1;
                        double m1 = mu_r ? (double)mu_r[cidx(nx, ny, r[0], r[1], r[2])] : 1.0;
                        double m2 = mu_r ? (double)mu_r[cidx(nx, ny, q[0], q[1], q[2])] : 1.0;
                        double area = ds[b][q[b]] * ds[c][q[c]];
                        double s = (ds[a][q[a] - 1] / 2.0) / m1 + (ds[a][q[a]] / 2.0) / m2;
                        double Mm = OR_MU0 * area / s;
                        double vch = dt / Mm;
                        if (round32) vch = (double)(float)vch;
                        ch[p] = vch;
                        mmu[p] = Mm;
                    }
                }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Absolute row sums of the skew matrix A of eq. (FIT_ode_2), the norm   */
/* ||A||_1 = ||A||_inf of Higham's parameter selection being their max:  */
/*   edge e: M_eps(e)^{-1/2} sum_{faces f of e} M_mu(f)^{-1/2}            */
/*   face f: M_mu(f)^{-1/2} sum_{edges e of f} M_eps(e)^{-1/2}            */
/* over the degrees of freedom (the incidences of curl_h and curl_e).     */
/* Returns the maximum; oe, oh (3*Np each, or NULL) receive the sums.     */
/* ------------------------------------------------------------------ */
double oracle_A_rowsum(const or_grid *g, double *oe, double *oh) {
    int nx = g->nx, ny = g->ny, nz = g->nz;
    int n[3] = {nx, ny, nz};
    long Np = np_of(g);
    double *ie = (double *)calloc((size_t)(3 * Np), sizeof(double));
    double *ih = (double *)calloc((size_t)(3 * Np), sizeof(double));
    double best = 0.0;
    if (!ie || !ih) { free(ie); free(ih); return -1.0; }
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k <= nz; ++k)
            for (int j = 0; j <= ny; ++j)
                for (int i = 0; i <= nx; ++i) {
                    int q[3] = {i, j, k};
                    long p = (long)a * Np + pidx(nx, ny, i, j, k);
                    if (edge_free(n, a, q)) ie[p] = 1.0 / sqrt(g->meps[p]);
                    if (face_interior(n, a, q)) ih[p] = 1.0 / sqrt(g->mmu[p]);
                }
    for (int a = 0; a < 3; ++a) {
        int b = (a + 1) % 3, c = (a + 2) % 3;
        for (int k = 0; k <= nz; ++k)
            for (int j = 0; j <= ny; ++j)
                for (int i = 0; i <= nx; ++i) {
                    int q[3] = {i, j, k};
                    long p = (long)a * Np + pidx(nx, ny, i, j, k);
                    double se = 0.0, sh = 0.0;
                    if (edge_free(n, a, q)) {   /* faces h_c(q), h_c(q-u_b), h_b(q), h_b(q-u_c) */
                        int qb[3] = {q[0], q[1], q[2]}, qc[3] = {q[0], q[1], q[2]};
                        qb[b] -= 1;
                        qc[c] -= 1;
                        double s = ih[(long)c * Np + pidx(nx, ny, q[0], q[1], q[2])] + ih[(long)b * Np + pidx(nx, ny, q[0], q[1], q[2])];
                        if (qb[b] >= 0) s += ih[(long)c * Np + pidx(nx, ny, qb[0], qb[1], qb[2])];
                        if (qc[c] >= 0) s += ih[(long)b * Np + pidx(nx, ny, qc[0], qc[1], qc[2])];
                        se = ie[p] * s;
                    }
                    if (face_interior(n, a, q)) {   /* edges e_b(q), e_c(q+u_b), e_b(q+u_c), e_c(q) */
                        int qb[3] = {q[0], q[1], q[2]}, qc[3] = {q[0], q[1], q[2]};
                        qb[b] += 1;
                        qc[c] += 1;
                        double s = ie[(long)b * Np + pidx(nx, ny, q[0], q[1], q[2])] + ie[(long)c * Np + pidx(nx, ny, q[0], q[1], q[2])];
                        if (qb[b] <= n[b]) s += ie[(long)c * Np + pidx(nx, ny, qb[0], qb[1], qb[2])];
                        if (qc[c] <= n[c]) s += ie[(long)b * Np + pidx(nx, ny, qc[0], qc[1], qc[2])];
                        sh = ih[p] * s;
                    }
                    if (oe) oe[p] = se;
                    if (oh) oh[p] = sh;
                    if (se > best) best = se;
                    if (sh > best) best = sh;
                }
    }
    free(ie); free(ih);
    return best;
}
