/*
 * FP64 CPU oracle for the relativistic-beam electromagnetic PIC step.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference the CUDA
 * path is checked against.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py load it.  It shares no source with
 * the CUDA library and must never be linked into it.
 *
 * Every routine is a direct loop over the definition it implements:
 *
 *   - Field advance: the discretised Faraday and Ampere laws of Sec. 2.1
 *     (Eq. 1), leapfrogged in time with the symbol [w]_t of Sec. 2.1, the Yee
 *     operators of Sec. 2.2 and the customised axial operators d+/d- of
 *     Appendix C (stencil width 2M, coefficients C_l).  B is advanced by half
 *     steps around the full E step so that E and B live at integer times.
 *   - Gather: the field at a particle is the shape-weighted sum over the
 *     staggered nodes of each component (Sec. 1: "the fields are used to
 *     interpolate forces onto the particles").
 *   - Push: relativistic Boris rotation (leapfrog in time, Sec. 2.1).
 *   - Deposit: charge-conserving (Esirkepov) current from the old and new
 *     positions, which is what Sec. 2.1 requires for Gauss's law (Eq. Gauss)
 *     to be kept by the field advance.
 *   - Current correction for the customised stencil (Sec. 3): J1 <- h * J1
 *     along z, h the impulse response of the inverse of the symbol ratio
 *     P = [k]_custom / [k]_Yee; h is supplied by the caller.
 *   - Current filter along z (the "5 pass" filter the paper uses with its runs and
 *     Table 2): four binomial passes and one compensating pass, on every current component.
 *   - Gauss residual d-.E - rho (Eq. Gauss), charge density, energies.
 *
 * Grid conventions.  Axis 1 is z (index i, contiguous), axis 2 is x (index j),
 * axis 3 is y (index k).  Arrays are [ny][nx][nz] doubles; 2D runs use ny = 1
 * and drop every y derivative.  Staggering: E1 (i+1/2,j,k), E2 (i,j+1/2,k),
 * E3 (i,j,k+1/2), B1 (i,j+1/2,k+1/2), B2 (i+1/2,j,k+1/2), B3 (i+1/2,j+1/2,k);
 * rho and the 2D E3 at nodes.  A field stored at index i of a half-integer
 * axis sits at i+1/2.  Fields are zero outside 0 <= i < nz (open/conducting
 * ends in z) and periodic in x and y.  Positions are in cell units
 * (xi = z/dz, x/dx, y/dy).
 *
 * Parameter blocks (kept flat for ctypes):
 *   ip[0]=ndim ip[1]=nz ip[2]=nx ip[3]=ny ip[4]=M ip[5]=shape (1|2)
 *   ip[6]=periodic_z (0: zero outside z, the PIC runs; 1: periodic, for the
 *         plane-wave dispersion test only; honoured by the field operators)
 *   ip[7]=split (0: one coefficient set C[0..M) for d+ and d-; 1: C[0..M) for the E-side
 *         d+ ([k]_E1, Faraday's law) and C[M..2M) for the B-side d- ([k]_B1, Ampere's and
 *         Gauss's laws): the "[k]_E1 != [k]_B1" option Sec. 3 mentions)
 *   dp[0]=dz dp[1]=dx dp[2]=dy dp[3]=dt
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads of the loops below (OpenMP builds only).  The library starts single-threaded so that
 * every test sees one fixed summation order; the CPU baseline raises it to time all cores.
 * Loops over cells write disjoint outputs; the deposit and the charge density add into shared
 * nodes with atomic updates. */
void or_set_threads(int n) {
#ifdef _OPENMP
    omp_set_num_threads(n < 1 ? 1 : n);
#else
    (void)n;
#endif
}
int or_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
int or_openmp(void) {
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}

typedef struct {
    int ndim, nz, nx, ny, M, shape, periodic_z;
    double dz, dx, dy, dt;
    const double* C;    /* d+ (E side) */
    const double* CB;   /* d- (B side) */
} grid_t;

static grid_t mk(const int* ip, const double* dp, const double* C) {
    grid_t g;
    g.ndim = ip[0]; g.nz = ip[1]; g.nx = ip[2]; g.ny = ip[3];
    g.M = ip[4]; g.shape = ip[5]; g.periodic_z = ip[6];
    g.dz = dp[0]; g.dx = dp[1]; g.dy = dp[2]; g.dt = dp[3];
    g.C = C;
    g.CB = (C && ip[7]) ? C + g.M : C;
    if (g.ndim == 2) g.ny = 1;
    return g;
}

static long ncell(const grid_t* g) { return (long)g->nz * g->nx * g->ny; }

static int wrap(int a, int n) { a %= n; if (a < 0) a += n; return a; }

/* field value with zero outside the z range and periodic x, y */
static double at(const grid_t* g, const double* f, int i, int j, int k) {
    if (g->periodic_z) i = wrap(i, g->nz);
    if (i < 0 || i >= g->nz) return 0.0;
    j = wrap(j, g->nx);
    k = wrap(k, g->ny);
    return f[((long)k * g->nx + j) * g->nz + i];
}

static long lin(const grid_t* g, int i, int j, int k) {
    return ((long)k * g->nx + j) * g->nz + i;
}

/* Appendix C: d+ f_i = sum_l C_l (f_{i+l} - f_{i-l+1}) / dz  (Yee: M=1, C_1=1) */
static double dzp(const grid_t* g, const double* f, int i, int j, int k) {
    double s = 0.0;
    for (int l = 1; l <= g->M; ++l)
        s += g->C[l - 1] * (at(g, f, i + l, j, k) - at(g, f, i - l + 1, j, k));
    return s / g->dz;
}
/* Appendix C: d- f_i = sum_l C_l (f_{i+l-1} - f_{i-l}) / dz, with the B-side coefficients */
static double dzm(const grid_t* g, const double* f, int i, int j, int k) {
    double s = 0.0;
    for (int l = 1; l <= g->M; ++l)
        s += g->CB[l - 1] * (at(g, f, i + l - 1, j, k) - at(g, f, i - l, j, k));
    return s / g->dz;
}
/* transverse operators are always the two-point Yee differences (Sec. 2.2) */
static double dxp(const grid_t* g, const double* f, int i, int j, int k) {
    return (at(g, f, i, j + 1, k) - at(g, f, i, j, k)) / g->dx;
}
static double dxm(const grid_t* g, const double* f, int i, int j, int k) {
    return (at(g, f, i, j, k) - at(g, f, i, j - 1, k)) / g->dx;
}
static double dyp(const grid_t* g, const double* f, int i, int j, int k) {
    if (g->ndim == 2) return 0.0;
    return (at(g, f, i, j, k + 1) - at(g, f, i, j, k)) / g->dy;
}
static double dym(const grid_t* g, const double* f, int i, int j, int k) {
    if (g->ndim == 2) return 0.0;
    return (at(g, f, i, j, k) - at(g, f, i, j, k - 1)) / g->dy;
}

/* Faraday half step B -= (dt/2) d+ x E.  Reads only E, so B updates in place. */
static void faraday_half(const grid_t* g, const double* E, double* B) {
    long N = ncell(g);
    const double *E1 = E, *E2 = E + N, *E3 = E + 2 * N;
    double *B1 = B, *B2 = B + N, *B3 = B + 2 * N;
    double h = 0.5 * g->dt;
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < g->ny; ++k)
        for (int j = 0; j < g->nx; ++j)
            for (int i = 0; i < g->nz; ++i) {
                long c = lin(g, i, j, k);
                double c1 = dxp(g, E3, i, j, k) - dyp(g, E2, i, j, k);
                double c2 = dyp(g, E1, i, j, k) - dzp(g, E3, i, j, k);
                double c3 = dzp(g, E2, i, j, k) - dxp(g, E1, i, j, k);
                B1[c] -= h * c1;
                B2[c] -= h * c2;
                B3[c] -= h * c3;
            }
}

/* Ampere full step E += dt (d- x B - J).  Reads only B and J. */
static void ampere(const grid_t* g, double* E, const double* B, const double* J) {
    long N = ncell(g);
    double *E1 = E, *E2 = E + N, *E3 = E + 2 * N;
    const double *B1 = B, *B2 = B + N, *B3 = B + 2 * N;
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < g->ny; ++k)
        for (int j = 0; j < g->nx; ++j)
            for (int i = 0; i < g->nz; ++i) {
                long c = lin(g, i, j, k);
                double c1 = dxm(g, B3, i, j, k) - dym(g, B2, i, j, k);
                double c2 = dym(g, B1, i, j, k) - dzm(g, B3, i, j, k);
                double c3 = dzm(g, B2, i, j, k) - dxm(g, B1, i, j, k);
                E1[c] += g->dt * (c1 - J[c]);
                E2[c] += g->dt * (c2 - J[N + c]);
                E3[c] += g->dt * (c3 - J[2 * N + c]);
            }
}

/* One field step: B^n -> B^{n+1/2} -> E^{n+1} -> B^{n+1}.  E, B, J are (3,ny,nx,nz). */
void or_field_advance(const int* ip, const double* dp, const double* C,
                      double* E, double* B, const double* J) {
    grid_t g = mk(ip, dp, C);
    faraday_half(&g, E, B);
    ampere(&g, E, B, J);
    faraday_half(&g, E, B);
}

/* Only the Faraday half step or only the Ampere step (used by operator tests). */
void or_faraday_half(const int* ip, const double* dp, const double* C, const double* E, double* B) {
    grid_t g = mk(ip, dp, C);
    faraday_half(&g, E, B);
}
void or_ampere(const int* ip, const double* dp, const double* C, double* E, const double* B, const double* J) {
    grid_t g = mk(ip, dp, C);
    ampere(&g, E, B, J);
}

/* Sec. 3 current correction: J1[i] <- sum_m h[m] J1[i-m], |m| <= hlen, J1 = 0 outside z. */
void or_correct_j1(const int* ip, const double* h, int hlen, double* J) {
    grid_t g = mk(ip, (const double[4]){1, 1, 1, 1}, NULL);
#pragma omp parallel
    {
    double* row = (double*)malloc(sizeof(double) * g.nz);
#pragma omp for collapse(2) schedule(static)
    for (int k = 0; k < g.ny; ++k)
        for (int j = 0; j < g.nx; ++j) {
            double* J1 = J + lin(&g, 0, j, k);
            for (int i = 0; i < g.nz; ++i) {
                double s = 0.0;
                for (int m = -hlen; m <= hlen; ++m) {
                    int src = i - m;
                    if (src >= 0 && src < g.nz) s += h[m + hlen] * J1[src];
                }
                row[i] = s;
            }
            memcpy(J1, row, sizeof(double) * g.nz);
        }
    free(row);
    }
}

/* B-spline particle shapes in cell units: linear (order 1) and quadratic (order 2). */
static double shape(int order, double d) {
    d = fabs(d);
    if (order == 1) return d < 1.0 ? 1.0 - d : 0.0;
    if (d <= 0.5) return 0.75 - d * d;
    if (d < 1.5) return 0.5 * (1.5 - d) * (1.5 - d);
    return 0.0;
}

/* staggering offsets (in cells) of E1..E3, B1..B3 along (z, x, y) */
static const double STAG[6][3] = {
    {0.5, 0.0, 0.0}, {0.0, 0.5, 0.0}, {0.0, 0.0, 0.5},
    {0.0, 0.5, 0.5}, {0.5, 0.0, 0.5}, {0.5, 0.5, 0.0},
};

static double interp(const grid_t* g, const double* f, const double* s, const double* xi) {
    double v = 0.0;
    int a0 = (int)floor(xi[0]) - 2, b0 = (int)floor(xi[1]) - 2;
    int c0 = g->ndim == 3 ? (int)floor(xi[2]) - 2 : 0;
    int cn = g->ndim == 3 ? 5 : 1;
    for (int c = c0; c < c0 + cn; ++c) {
        double wy = g->ndim == 3 ? shape(g->shape, c + s[2] - xi[2]) : 1.0;
        if (wy == 0.0) continue;
        for (int b = b0; b < b0 + 5; ++b) {
            double wx = shape(g->shape, b + s[1] - xi[1]);
            if (wx == 0.0) continue;
            for (int a = a0; a < a0 + 5; ++a) {
                double wz = shape(g->shape, a + s[0] - xi[0]);
                if (wz == 0.0) continue;
                v += wz * wx * wy * at(g, f, a, b, c);
            }
        }
    }
    return v;
}

/* Gather E, B at n particles.  xi (n,3) in cell units; out (n,6) = E1 E2 E3 B1 B2 B3. */
void or_gather(const int* ip, const double* dp, const double* E, const double* B,
               long n, const double* xi, double* out) {
    grid_t g = mk(ip, dp, NULL);
    long N = ncell(&g);
#pragma omp parallel for schedule(static)
    for (long p = 0; p < n; ++p)
        for (int c = 0; c < 6; ++c) {
            const double* f = c < 3 ? E + c * N : B + (c - 3) * N;
            out[p * 6 + c] = interp(&g, f, STAG[c], xi + 3 * p);
        }
}

/* Relativistic Boris push u^{n-1/2} -> u^{n+1/2}; eps = q dt / (2 m). */
void or_boris(long n, const double* eb, double* u, double eps) {
#pragma omp parallel for schedule(static)
    for (long p = 0; p < n; ++p) {
        const double* E = eb + 6 * p;
        const double* B = eb + 6 * p + 3;
        double* v = u + 3 * p;
        double um[3], t[3], s[3], up[3], ul[3];
        for (int d = 0; d < 3; ++d) um[d] = v[d] + eps * E[d];
        double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
        for (int d = 0; d < 3; ++d) t[d] = eps * B[d] / gm;
        double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
        for (int d = 0; d < 3; ++d) s[d] = 2.0 * t[d] / (1.0 + t2);
        up[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
        up[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
        up[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
        ul[0] = um[0] + (up[1] * s[2] - up[2] * s[1]);
        ul[1] = um[1] + (up[2] * s[0] - up[0] * s[2]);
        ul[2] = um[2] + (up[0] * s[1] - up[1] * s[0]);
        for (int d = 0; d < 3; ++d) v[d] = ul[d] + eps * E[d];
    }
}

/* x^{n+1} = x^n + dt u^{n+1/2} / gamma^{n+1/2}, in cell units (no wrapping). */
void or_move(const int* ip, const double* dp, long n, const double* xi0, const double* u, double* xi1) {
    grid_t g = mk(ip, dp, NULL);
    double h[3] = {g.dz, g.dx, g.dy};
#pragma omp parallel for schedule(static)
    for (long p = 0; p < n; ++p) {
        const double* v = u + 3 * p;
        double gam = sqrt(1.0 + v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        for (int d = 0; d < 3; ++d)
            xi1[3 * p + d] = d < g.ndim ? xi0[3 * p + d] + g.dt * v[d] / gam / h[d] : xi0[3 * p + d];
    }
}

/*
 * Esirkepov current deposition for a move xi0 -> xi1 (each |dxi| < 1 cell).
 * 2D: W1 = dS1 (S0_2 + dS2/2), W2 = dS2 (S0_1 + dS1/2),
 *     W3 = S0_1 S0_2 + dS1 S0_2/2 + S0_1 dS2/2 + dS1 dS2/3,
 *     J1 = -(Q/V)(dz/dt) cumsum_z W1, J2 = -(Q/V)(dx/dt) cumsum_x W2, J3 = (Q/V) v3 W3.
 * 3D: W_a = dS_a (S0_b S0_c + dS_b S0_c/2 + S0_b dS_c/2 + dS_b dS_c/3), J_a = -(Q/V)(h_a/dt) cumsum_a W_a.
 * Adds into J (3,ny,nx,nz).  Q = charge of one macro-particle; V the cell volume.
 */
void or_deposit(const int* ip, const double* dp, long n, const double* xi0, const double* xi1,
                const double* u, double Q, double* J) {
    grid_t g = mk(ip, dp, NULL);
    long N = ncell(&g);
    double V = g.ndim == 3 ? g.dz * g.dx * g.dy : g.dz * g.dx;
    double hh[3] = {g.dz, g.dx, g.dy};
    enum { W = 8 };
#pragma omp parallel for schedule(static)
    for (long p = 0; p < n; ++p) {
        const double* a0p = xi0 + 3 * p;
        const double* a1p = xi1 + 3 * p;
        int base[3];
        double S0[3][W], DS[3][W];
        int nd = g.ndim;
        for (int d = 0; d < 3; ++d) {
            base[d] = (int)floor(fmin(a0p[d], a1p[d])) - 3;
            for (int q = 0; q < W; ++q) {
                if (d < nd) {
                    double s0 = shape(g.shape, base[d] + q - a0p[d]);
                    double s1 = shape(g.shape, base[d] + q - a1p[d]);
                    S0[d][q] = s0;
                    DS[d][q] = s1 - s0;
                } else {
                    S0[d][q] = q == 0 ? 1.0 : 0.0;
                    DS[d][q] = 0.0;
                }
            }
        }
        if (nd == 2) base[2] = 0;
        int qy = nd == 3 ? W : 1;
        double gam = sqrt(1.0 + u[3 * p] * u[3 * p] + u[3 * p + 1] * u[3 * p + 1] + u[3 * p + 2] * u[3 * p + 2]);
        double v3 = u[3 * p + 2] / gam;
        for (int a = 0; a < 3; ++a) {
            if (a >= nd) continue;
            int b = (a + 1) % 3, c = (a + 2) % 3;
            if (nd == 2) { b = 1 - a; c = 2; }
            double fac = -Q / V * hh[a] / g.dt;
            /* loop over the two transverse window indices, cumulative sum along a */
            int nb = (b < nd) ? W : 1, nc = (c < nd) ? W : 1;
            for (int ib = 0; ib < nb; ++ib)
                for (int ic = 0; ic < nc; ++ic) {
                    double cum = 0.0;
                    for (int ia = 0; ia < W; ++ia) {
                        double Wv = DS[a][ia] * (S0[b][ib] * S0[c][ic] + 0.5 * DS[b][ib] * S0[c][ic]
                                                 + 0.5 * S0[b][ib] * DS[c][ic] + DS[b][ib] * DS[c][ic] / 3.0);
                        cum += Wv;
                        int idx[3];
                        idx[a] = base[a] + ia; idx[b] = base[b] + ib; idx[c] = base[c] + ic;
                        if (idx[0] < 0 || idx[0] >= g.nz) continue;
                        int jj = wrap(idx[1], g.nx), kk = nd == 3 ? wrap(idx[2], g.ny) : 0;
#pragma omp atomic
                        J[a * N + lin(&g, idx[0], jj, kk)] += fac * cum;
                    }
                }
        }
        if (nd == 2) {
            double fac = Q / V * v3;
            for (int ia = 0; ia < W; ++ia)
                for (int ib = 0; ib < W; ++ib) {
                    double Wv = S0[0][ia] * S0[1][ib] + 0.5 * DS[0][ia] * S0[1][ib]
                              + 0.5 * S0[0][ia] * DS[1][ib] + DS[0][ia] * DS[1][ib] / 3.0;
                    int i = base[0] + ia;
                    if (i < 0 || i >= g.nz) continue;
#pragma omp atomic
                    J[2 * N + lin(&g, i, wrap(base[1] + ib, g.nx), 0)] += fac * Wv;
                }
        }
        (void)qy;
    }
}

/* Charge density at nodes: rho += (Q/V) S(i - xi_z) S(j - xi_x) [S(k - xi_y)]. */
void or_rho(const int* ip, const double* dp, long n, const double* xi, double Q, double* rho) {
    grid_t g = mk(ip, dp, NULL);
    double V = g.ndim == 3 ? g.dz * g.dx * g.dy : g.dz * g.dx;
#pragma omp parallel for schedule(static)
    for (long p = 0; p < n; ++p) {
        const double* x = xi + 3 * p;
        int a0 = (int)floor(x[0]) - 2, b0 = (int)floor(x[1]) - 2;
        int c0 = g.ndim == 3 ? (int)floor(x[2]) - 2 : 0, cn = g.ndim == 3 ? 5 : 1;
        for (int c = c0; c < c0 + cn; ++c) {
            double wy = g.ndim == 3 ? shape(g.shape, c - x[2]) : 1.0;
            for (int b = b0; b < b0 + 5; ++b) {
                double wx = shape(g.shape, b - x[1]);
                for (int a = a0; a < a0 + 5; ++a) {
                    if (a < 0 || a >= g.nz) continue;
                    double w = shape(g.shape, a - x[0]) * wx * wy;
                    if (w == 0.0) continue;
#pragma omp atomic
                    rho[lin(&g, a, wrap(b, g.nx), g.ndim == 3 ? wrap(c, g.ny) : 0)] += Q / V * w;
                }
            }
        }
    }
}

/* Gauss residual at nodes: G = d-_z E1 + d-_x E2 + d-_y E3 - rho (Eq. Gauss). */
void or_gauss(const int* ip, const double* dp, const double* C, const double* E,
              const double* rho, double* G) {
    grid_t g = mk(ip, dp, C);
    long N = ncell(&g);
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < g.ny; ++k)
        for (int j = 0; j < g.nx; ++j)
            for (int i = 0; i < g.nz; ++i) {
                long c = lin(&g, i, j, k);
                G[c] = dzm(&g, E, i, j, k) + dxm(&g, E + N, i, j, k) + dym(&g, E + 2 * N, i, j, k) - rho[c];
            }
}

/* Current filter along z (the "5 pass" filter of Sec. 2.2, 2.3 and Table 2; the paper names it
 * without defining it).  Reading: four passes of the binomial smoother (1/4, 1/2, 1/4) followed
 * by one compensating pass (-5/4, 7/2, -5/4).  Each pass is y_i = w1 (x_{i-1} + x_{i+1}) + w0 x_i
 * over 0 <= i < nz with x = 0 outside that range (open z) or x periodic in z when periodic_z.
 * The k-space symbol of one pass is w0 + 2 w1 cos(k dz), so the whole filter multiplies a
 * Fourier mode by cos^8(k dz/2) (1 + 5 sin^2(k dz/2)).  ncomp arrays of nz*nx*ny doubles. */
void or_filter_z(const int* ip, int ncomp, double* F) {
    static const double w1[5] = {0.25, 0.25, 0.25, 0.25, -1.25};
    static const double w0[5] = {0.5, 0.5, 0.5, 0.5, 3.5};
    grid_t g = mk(ip, (const double[4]){1, 1, 1, 1}, NULL);
    long N = ncell(&g);
#pragma omp parallel
    {
    double* x = (double*)malloc(sizeof(double) * g.nz);
#pragma omp for collapse(3) schedule(static)
    for (int c = 0; c < ncomp; ++c)
        for (int k = 0; k < g.ny; ++k)
            for (int j = 0; j < g.nx; ++j) {
                double* row = F + c * N + lin(&g, 0, j, k);
                for (int p = 0; p < 5; ++p) {
                    memcpy(x, row, sizeof(double) * g.nz);
                    for (int i = 0; i < g.nz; ++i) {
                        int il = i - 1, ir = i + 1;
                        if (g.periodic_z) { il = wrap(il, g.nz); ir = wrap(ir, g.nz); }
                        double xl = (il >= 0 && il < g.nz) ? x[il] : 0.0;
                        double xr = (ir >= 0 && ir < g.nz) ? x[ir] : 0.0;
                        row[i] = w1[p] * (xl + xr) + w0[p] * x[i];
                    }
                }
            }
    free(x);
    }
}

/* Moving window: every field array moves one cell towards -z, the front column becomes zero. */
void or_shift_z(const int* ip, int ncomp, double* F) {
    grid_t g = mk(ip, (const double[4]){1, 1, 1, 1}, NULL);
    long N = ncell(&g);
    for (int c = 0; c < ncomp; ++c)
        for (int k = 0; k < g.ny; ++k)
            for (int j = 0; j < g.nx; ++j) {
                double* row = F + c * N + lin(&g, 0, j, k);
                for (int i = 0; i + 1 < g.nz; ++i) row[i] = row[i + 1];
                row[g.nz - 1] = 0.0;
            }
}
