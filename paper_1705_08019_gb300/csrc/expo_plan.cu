// expo_plan.cu -- host side of the exponential propagators of the
// homogeneous ParaExp problems (Sec. III-B, "Approximation of the matrix
// exponential"; parameter condition of Sec. III-D).
//
// Nothing here touches the device: the interpolation points, the divided
// differences of exp, the choice of substep and degree, and the real
// coefficients the operator kernels consume are scalars computed once per
// run (and cached per argument set).
//
//  * Spectral interval.  X = dt_CFL A has its spectrum in i[-2, 2]; a substep
//    of q leapfrog steps is exp(c X), c = q dt / dt_CFL.
//  * Points.  Leja: xi_0 = 0 followed by conjugate pairs +-i eta_j; eta_j is
//    the first maximiser over the grid eta = 2l/2^15 of the sum of log
//    distances to the points chosen before.  Taylor: all points 0.
//  * Divided differences d_k = f[xi_0..xi_k] of f(z) = exp(a z): the first
//    column of exp(a Z), Z lower bidiagonal with the points on the diagonal
//    and ones below it (Opitz, 1964), computed by scaling and squaring with
//    a truncated Taylor series.  Taylor points: d_k = a^k / k!.
//  * Condition (per substep, normal A, ||A|| bounded by 2/dt_CFL):
//      max_z |log(p_m(z) e^{-cz})| + u_p H_m <= 2 c tol
//    on z = i 2l/4096, l = 0..4096, for tau = 1 and every output fraction
//    tau = i/q (with tau c in place of c); the smallest m/q wins.
#include <algorithm>
#include <cmath>
#include <complex>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "internal.h"

namespace fitgb {
namespace {

using cplx = std::complex<double>;

constexpr int kEtaGrid = 1 << 15;
constexpr int kSamples = 4096;
constexpr double kCmax = 32.0;
constexpr int kMaxPairs = kExpoMaxDegree / 2;

std::mutex g_mu;
std::vector<double> g_etas;   // eta_1..eta_kMaxPairs once computed
std::map<std::tuple<int, double, double, int>, std::pair<int, int>> g_plans;
std::map<std::tuple<int, int, double>, std::vector<double>> g_coeffs;   // (kind, m, a) -> alpha | gamma | eta2

// Conjugate Leja points: the greedy maximisation of the product of distances
// to the points chosen so far, over the grid of the half segment i[0, 2].
const std::vector<double> &leja_etas() {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_etas.empty()) return g_etas;
    std::vector<double> grid(kEtaGrid + 1), score(kEtaGrid + 1);
    for (int l = 0; l <= kEtaGrid; ++l) {
        grid[l] = 2.0 * (double)l / (double)kEtaGrid;
        score[l] = std::log(grid[l]);   // distance to xi_0 = 0 (-inf at 0)
    }
    std::vector<double> etas;
    for (int p = 0; p < kMaxPairs; ++p) {
        int best = 0;
        for (int l = 1; l <= kEtaGrid; ++l)
            if (score[l] > score[best]) best = l;
        const double eta = grid[best];
        etas.push_back(eta);
        for (int l = 0; l <= kEtaGrid; ++l)
            score[l] = (score[l] + std::log(std::fabs(grid[l] - eta))) + std::log(grid[l] + eta);
    }
    g_etas = etas;
    return g_etas;
}

std::vector<cplx> points(int kind, int m) {
    std::vector<cplx> xi(m + 1, cplx(0.0, 0.0));
    if (kind == FIT_HOMOG_TAYLOR) return xi;
    const std::vector<double> &etas = leja_etas();
    for (int k = 1; k <= m; ++k) {
        const double eta = etas[(k - 1) / 2];
        xi[k] = (k & 1) ? cplx(0.0, eta) : cplx(0.0, -eta);
    }
    return xi;
}

// Lower-triangular complex matrices of order n, row-major.
void lt_mul(int n, const std::vector<cplx> &A, const std::vector<cplx> &B, std::vector<cplx> &C) {
    for (int r = 0; r < n; ++r)
        for (int c = 0; c <= r; ++c) {
            cplx s(0.0, 0.0);
            for (int k = c; k <= r; ++k) s += A[r * n + k] * B[k * n + c];
            C[r * n + c] = s;
        }
}

// d_k = f[xi_0..xi_k] for f(z) = exp(a z), k = 0..m.
std::vector<cplx> divided_differences(int kind, const std::vector<cplx> &xi, double a) {
    const int n = (int)xi.size();
    std::vector<cplx> d(n);
    if (kind == FIT_HOMOG_TAYLOR) {
        double v = 1.0;
        for (int k = 0; k < n; ++k) {
            d[k] = cplx(v, 0.0);
            v = v * a / (double)(k + 1);
        }
        return d;
    }
    double rad = 0.0;
    for (const cplx &z : xi) rad = std::max(rad, std::abs(z));
    const double nrm = std::fabs(a) * (rad + 1.0);   // bound on ||a Z||_1
    int sq = 0;
    while (nrm / std::ldexp(1.0, sq) > 0.5) ++sq;
    const double scale = a / std::ldexp(1.0, sq);
    std::vector<cplx> M(n * n, cplx(0.0, 0.0)), E(n * n, cplx(0.0, 0.0)), T(n * n, cplx(0.0, 0.0)),
        W(n * n, cplx(0.0, 0.0));
    for (int r = 0; r < n; ++r) {
        M[r * n + r] = scale * xi[r];
        if (r > 0) M[r * n + r - 1] = cplx(scale, 0.0);
        E[r * n + r] = cplx(1.0, 0.0);
        T[r * n + r] = cplx(1.0, 0.0);
    }
    // Taylor series of exp(M), ||M|| <= 1/2: 20 terms reach double rounding
    for (int k = 1; k <= 20; ++k) {
        lt_mul(n, T, M, W);
        for (int t = 0; t < n * n; ++t) {
            T[t] = W[t] / (double)k;
            E[t] += T[t];
        }
    }
    for (int s = 0; s < sq; ++s) {
        lt_mul(n, E, E, W);
        E.swap(W);
    }
    for (int k = 0; k < n; ++k) d[k] = E[k * n + 0];
    return d;
}

// err[k] = max over the samples of |log(p_k e^{-cz})| + u_p max_z sum_{l<=k} |d_l w_l(z)|
std::vector<double> errors(const std::vector<cplx> &xi, const std::vector<cplx> &d, double c, double up) {
    const int n = (int)xi.size();
    std::vector<double> out(n, 0.0), dmax(n, 0.0), hmax(n, 0.0);
    for (int l = 0; l <= kSamples; ++l) {
        const cplx z(0.0, 2.0 * (double)l / (double)kSamples);
        const cplx ecz = std::exp(-c * z);
        cplx w(1.0, 0.0), p(0.0, 0.0);
        double hump = 0.0;
        for (int k = 0; k < n; ++k) {
            const cplx term = d[k] * w;
            p += term;
            hump += std::abs(term);
            double delta = std::abs(std::log(p * ecz));
            if (std::isnan(delta)) delta = INFINITY;
            dmax[k] = std::max(dmax[k], delta);
            hmax[k] = std::max(hmax[k], hump);
            w *= z - xi[k];
        }
    }
    for (int k = 0; k < n; ++k) out[k] = dmax[k] + up * hmax[k];
    return out;
}

std::pair<int, int> plan_uncached(int kind, double u, double tol, int precision) {
    const double up = precision == 32 ? std::ldexp(1.0, -24) : std::ldexp(1.0, -53);
    const std::vector<cplx> xi = points(kind, kExpoMaxDegree);
    struct Cand {
        double cost;
        int q, m;
    };
    std::vector<Cand> cands;
    for (int q = 1; q * u <= kCmax; ++q) {
        const double c = q * u;
        const std::vector<double> err = errors(xi, divided_differences(kind, xi, c), c, up);
        for (int m = 2; m <= kExpoMaxDegree; m += 2)
            if (err[m] <= 2.0 * c * tol) {
                cands.push_back({(double)m / q, q, m});
                break;
            }
    }
    std::sort(cands.begin(), cands.end(), [](const Cand &x, const Cand &y) {
        return x.cost < y.cost || (x.cost == y.cost && x.q < y.q);
    });
    bool have = false;
    double best_cost = 0.0;
    int best_q = 0, best_m = 0;
    for (const Cand &cd : cands) {
        if (have && (cd.cost > best_cost || (cd.cost == best_cost && cd.q > best_q))) break;
        const int q = cd.q;
        const double c = q * u;
        int m = cd.m;
        while (m <= kExpoMaxDegree) {
            bool fails = false;
            const std::vector<cplx> sub(xi.begin(), xi.begin() + m + 1);
            for (int i = 1; i < q && !fails; ++i) {
                const double tau = (double)i / q;
                const std::vector<double> err = errors(sub, divided_differences(kind, sub, tau * c), tau * c, up);
                if (err[m] > 2.0 * tau * c * tol) fails = true;
            }
            if (!fails) break;
            m += 2;
        }
        if (m > kExpoMaxDegree) continue;
        const double cost = (double)m / q;
        if (!have || cost < best_cost || (cost == best_cost && q < best_q)) {
            have = true;
            best_cost = cost;
            best_q = q;
            best_m = m;
        }
    }
    if (!have) return {0, 0};
    return {best_q, best_m};
}

}  // namespace

int expo_plan(int kind, double u, double tol, int precision, int *q, int *m) {
    if (kind != FIT_HOMOG_LEJA && kind != FIT_HOMOG_TAYLOR) return FIT_ERR_ARG;
    if (!(u > 0.0) || !std::isfinite(u) || !(tol > 0.0) || !std::isfinite(tol)) return FIT_ERR_ARG;
    if (precision != 32 && precision != 64) return FIT_ERR_ARG;
    const auto key = std::make_tuple(kind, u, tol, precision);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_plans.find(key);
        if (it != g_plans.end()) {
            *q = it->second.first;
            *m = it->second.second;
            return *q > 0 ? FIT_OK : FIT_ERR_ARG;
        }
    }
    const std::pair<int, int> r = plan_uncached(kind, u, tol, precision);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_plans[key] = r;
    }
    *q = r.first;
    *m = r.second;
    return r.first > 0 ? FIT_OK : FIT_ERR_ARG;
}

int expo_pair_coeffs(int kind, int m, double a, double *alpha, double *gamma, double *eta2) {
    if (kind != FIT_HOMOG_LEJA && kind != FIT_HOMOG_TAYLOR) return FIT_ERR_ARG;
    if (m < 2 || m > kExpoMaxDegree || (m & 1) || !std::isfinite(a)) return FIT_ERR_ARG;
    const int J = m / 2;
    const auto key = std::make_tuple(kind, m, a);
    std::vector<double> v;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_coeffs.find(key);
        if (it != g_coeffs.end()) v = it->second;
    }
    if (v.empty()) {
        const std::vector<cplx> xi = points(kind, m);
        const std::vector<cplx> d = divided_differences(kind, xi, a);
        v.resize(3 * J);
        for (int j = 1; j <= J; ++j) {
            const double eta = xi[2 * j - 1].imag();   // xi_{2j-1} = +i eta_j
            // p_{2j} - p_{2j-2} = R_{j-1}(z) ((d_{2j-1} - i eta_j d_{2j}) + d_{2j} z): real for conjugate points
            v[j - 1] = (d[2 * j - 1] - cplx(0.0, eta) * d[2 * j]).real();
            v[J + j - 1] = d[2 * j].real();
            v[2 * J + j - 1] = eta * eta;
        }
        std::lock_guard<std::mutex> lk(g_mu);
        if (g_coeffs.size() > 4096) g_coeffs.clear();
        g_coeffs[key] = v;
    }
    for (int j = 0; j < J; ++j) {
        alpha[j] = v[j];
        gamma[j] = v[J + j];
        eta2[j] = v[2 * J + j];
    }
    return FIT_OK;
}

}  // namespace fitgb

extern "C" {

int fit_expo_plan(int kind, double dt_ratio, double tol, int precision, int *substep, int *degree) {
    if (!substep || !degree) return FIT_ERR_ARG;
    return fitgb::expo_plan(kind, dt_ratio, tol, precision, substep, degree);
}

int fit_expo_coeffs(int kind, int degree, double a, double *alpha, double *gamma, double *eta2) {
    if (!alpha || !gamma || !eta2) return FIT_ERR_ARG;
    return fitgb::expo_pair_coeffs(kind, degree, a, alpha, gamma, eta2);
}

}  // extern "C"
