// Host-side setup math of libpic (FP64): the Appendix C coefficient fit, the Sec. 3
// current-correction taps and the leapfrog stability limit.  Runs once per handle.
#include <cmath>
#include <vector>

#include "pic_internal.h"

namespace pic {

namespace {

typedef long double ld;

// Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_n (extended precision).
void gauss_legendre(int n, std::vector<ld>& x, std::vector<ld>& w) {
    x.assign(n, 0.0L);
    w.assign(n, 0.0L);
    const ld pi = 3.141592653589793238462643383279502884L;
    for (int i = 0; i < (n + 1) / 2; ++i) {
        ld z = std::cos(pi * (i + 0.75L) / (n + 0.5L));
        ld pp = 0.0L, p0 = 1.0L, p1 = z;
        for (int it = 0; it < 100; ++it) {
            p0 = 1.0L;
            p1 = z;
            for (int k = 2; k <= n; ++k) {
                ld p2 = ((2.0L * k - 1.0L) * z * p1 - (k - 1.0L) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            pp = n * (z * p1 - p0) / (z * z - 1.0L);
            ld dz = p1 / pp;
            z -= dz;
            if (std::fabs(dz) < 1e-19L) break;
        }
        p0 = 1.0L;
        p1 = z;
        for (int k = 2; k <= n; ++k) {
            ld p2 = ((2.0L * k - 1.0L) * z * p1 - (k - 1.0L) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        pp = n * (z * p1 - p0) / (z * z - 1.0L);
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0L / ((1.0L - z * z) * pp * pp);
    }
}

// Dense solve with partial pivoting (LU), in place; returns 0 on success.
int solve(std::vector<ld>& A, std::vector<ld>& b, int n) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
        if (A[piv * n + c] == 0.0L) return 1;
        if (piv != c) {
            for (int k = 0; k < n; ++k) std::swap(A[c * n + k], A[piv * n + k]);
            std::swap(b[c], b[piv]);
        }
        for (int r = c + 1; r < n; ++r) {
            ld f = A[r * n + c] / A[c * n + c];
            if (f == 0.0L) continue;
            for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        ld s = b[r];
        for (int k = r + 1; k < n; ++k) s -= A[r * n + k] * b[k];
        b[r] = s / A[r * n + r];
    }
    return 0;
}

}  // namespace

// Appendix C: minimise int_0^1/2 w(k) ([k1]_p - [k1]_target)^2 dk subject to
// sum_l (2l-1) C_l = 1, with [k1]_target = (kappa/pi) sin(pi k / kappa) (Sec. 3) in units of
// k_g = 2 pi/dz, solved through the bordered (Lagrange) system.  The system is very
// ill-conditioned (the high-order sines are nearly dependent where the weight lives), so the
// quadrature and the solve run in extended precision.
// The target is (kappa/pi) sin(pi k/kappa) ([k1]_t, Sec. 3); with CE given (ME coefficients of an
// E-side operator) it is [k1]_t^2 / [k]_E1, the B side of a pair with [k]_E1 [k]_B1 = [k1]_t^2
// (the [k]_E1 != [k]_B1 solvers Sec. 3 allows).
static int fit_target(double kappa, int M, double wk, double n, const double* CE, int ME, double* C) {
    if (M < 1 || M > PIC_MAX_M || !(kappa > 0.0)) return 1;
    if (wk <= 0.0) wk = 0.6;
    if (n <= 0.0) n = 10.0;
    const ld pi = 3.141592653589793238462643383279502884L;
    const int nq = 1000;
    std::vector<ld> gx, gw;
    gauss_legendre(nq, gx, gw);
    const int N = M + 1;
    std::vector<ld> K(N * N, 0.0L), rhs(N, 0.0L);
    for (int q = 0; q < nq; ++q) {
        ld k = 0.25L * (gx[q] + 1.0L);
        ld wq = 0.25L * gw[q] * std::exp(-std::log(2.0L) * std::pow(2.0L * k / (ld)wk, (ld)n));
        ld target = (ld)kappa / pi * std::sin(pi * k / (ld)kappa);
        if (CE) {
            ld ke = 0.0L;                    // [k]_E1 in units of k_g: sum_l C_l sin((2l-1) pi k) / pi
            for (int l = 0; l < ME; ++l) ke += (ld)CE[l] * std::sin((2 * l + 1) * pi * k);
            ke /= pi;
            if (!(std::fabs(ke) > 0.0L)) continue;     // k = 0: no weight in the quadrature
            target = target * target / ke;
        }
        ld s[PIC_MAX_M];
        for (int l = 0; l < M; ++l) s[l] = std::sin((2 * l + 1) * pi * k);
        for (int i = 0; i < M; ++i) {
            for (int j = 0; j < M; ++j) K[i * N + j] += 2.0L / (pi * pi) * wq * s[i] * s[j];
            rhs[i] += 2.0L / pi * wq * s[i] * target;
        }
    }
    for (int j = 0; j < M; ++j) {
        K[j * N + M] = 2.0L * j + 1.0L;
        K[M * N + j] = 2.0L * j + 1.0L;
    }
    rhs[M] = 1.0L;
    if (solve(K, rhs, N)) return 1;
    for (int l = 0; l < M; ++l) C[l] = (double)rhs[l];
    return 0;
}

int fit_coefficients(double kappa, int M, double wk, double n, double* C) {
    return fit_target(kappa, M, wk, n, nullptr, 0, C);
}

int fit_coefficients_b(double kappa, int M, double wk, double n, const double* CE, int ME, double* C) {
    if (!CE || ME < 1 || ME > PIC_MAX_M) return 1;
    return fit_target(kappa, M, wk, n, CE, ME, C);
}

// Sec. 3 correction: taps of the inverse of P(phi) = P_0 + 2 sum_m P_m cos(m phi),
// P_m = sum_{l > m} C_l, sampled on a fine periodic grid (the DFT of 1/P).
int correction_taps(const double* C, int M, int hlen, double* h) {
    if (M < 1 || M > PIC_MAX_M || hlen < 0) return 1;
    double Pm[PIC_MAX_M];
    for (int m = 0; m < M; ++m) {
        double s = 0.0;
        for (int l = m; l < M; ++l) s += C[l];
        Pm[m] = s;
    }
    const int Nf = 8192;
    std::vector<double> inv(Nf);
    for (int q = 0; q < Nf; ++q) {
        double phi = 2.0 * M_PI * q / Nf;
        double P = Pm[0];
        for (int m = 1; m < M; ++m) P += 2.0 * Pm[m] * std::cos(m * phi);
        if (!(std::fabs(P) > 1e-12)) return 1;
        inv[q] = 1.0 / P;
    }
    for (int m = 0; m <= hlen; ++m) {
        double s = 0.0;
        for (int q = 0; q < Nf; ++q) s += inv[q] * std::cos(2.0 * M_PI * (double)m * q / Nf);
        h[hlen + m] = h[hlen - m] = s / Nf;
    }
    return 0;
}

// Leapfrog limit (dt/2)^2 (max [k]_E1 [k]_B1 + sum (2/d_perp)^2) <= 1 (Eq. wave); [k]_E1 = [k]_B1
// for the symmetric stencils.
double cfl_dt_split(int ndim, double dz, double dx, double dy, const double* CE, const double* CB, int M) {
    double pmax = 0.0, pmin = 0.0;
    const int ns = 20001;
    for (int q = 0; q < ns; ++q) {
        double t = 0.5 * M_PI * q / (ns - 1);
        double se = 0.0, sb = 0.0;
        for (int l = 0; l < M; ++l) {
            se += CE[l] * std::sin((2 * l + 1) * t);
            sb += CB[l] * std::sin((2 * l + 1) * t);
        }
        pmax = std::fmax(pmax, se * sb);
        pmin = std::fmin(pmin, se * sb);
    }
    if (pmin < -1e-12 * std::fmax(pmax, 1e-300)) return -1.0;
    double s = pmax * (2.0 / dz) * (2.0 / dz) + (2.0 / dx) * (2.0 / dx);
    if (ndim == 3) s += (2.0 / dy) * (2.0 / dy);
    return 2.0 / std::sqrt(s);
}

double cfl_dt(int ndim, double dz, double dx, double dy, const double* C, int M) {
    return cfl_dt_split(ndim, dz, dx, dy, C, C, M);
}

// k-space solvers: the leapfrog is stable while (dt/2)^2 max_k sum_a [k]_a^2 <= 1, the maximum at
// the Nyquist wavenumber of every axis.  Spectral: [k]_a = pi/h_a there.  [k1]_t along z (Yee
// across): sin^2(pi dt/(2 dz)) + sum_perp (dt/h)^2 <= 1 with dt < dz, increasing in dt: bisection.
// kt = 2 (PSATD): the analytic update is stable for any dt; the particle move allows one cell.
double kspace_cfl_dt(int ndim, int kt, double dz, double dx, double dy) {
    const double hp[2] = {dx, dy};
    const int np = ndim == 3 ? 2 : 1;
    if (kt == 2) {                         // PSATD: one cell per step for the particles
        double h = std::fmin(dz, dx);
        if (ndim == 3) h = std::fmin(h, dy);
        return h;
    }
    if (!kt) {
        double s = (M_PI / dz) * (M_PI / dz);
        for (int a = 0; a < np; ++a) s += (M_PI / hp[a]) * (M_PI / hp[a]);
        return 2.0 / std::sqrt(s);
    }
    auto f = [&](double dt) {
        const double q = std::sin(0.5 * M_PI * dt / dz);
        double v = q * q - 1.0;
        for (int a = 0; a < np; ++a) v += (dt / hp[a]) * (dt / hp[a]);
        return v;
    };
    double lo = 0.0, hi = dz;
    if (f(hi) <= 0.0) return hi;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (f(mid) <= 0.0) lo = mid;
        else hi = mid;
    }
    return lo;
}

}  // namespace pic
