/*
 * pic.h -- C ABI of the GB300 (sm_103a) relativistic-beam electromagnetic PIC step.
 *
 * The step is the PIC loop of Sec. 1 of arXiv:1910.13529 ("deposit -> advance the
 * fields -> interpolate -> push"), with
 *   - the discretised Faraday and Ampere laws of Sec. 2.1 (Eq. 1) on a staggered grid,
 *     axial derivative either the Yee two-point difference (Sec. 2.2) or the customised
 *     2M-point stencil d+/d- of Sec. 3 and Appendix C;
 *   - charge-conserving (Esirkepov) current deposition, which keeps Gauss's law
 *     (Eq. Gauss) as Sec. 2.1 requires, with linear or quadratic B-spline shapes;
 *   - optionally the current filter along z that the paper runs with ("5 pass filter",
 *     Sec. 2.2, 2.3, Table 2): four (1/4, 1/2, 1/4) passes and one (-5/4, 7/2, -5/4) pass;
 *   - for the customised stencil, the current correction of Sec. 3: J1 <- h * J1 along z,
 *     h the impulse response of 1/P, P(k) = [k]_custom / [k]_Yee;
 *   - field interpolation (gather) and a relativistic Boris push (leapfrog, Sec. 2.1);
 *   - an optional moving window at c along +z with cold-plasma injection.
 *
 * Units: c = 1, lengths in c/omega_p, time in 1/omega_p, Gauss's law d.E = rho.
 *
 * Grid and memory layout (all device arrays are caller-owned, contiguous, FP32):
 *   axis 1 = z (index i, fastest), axis 2 = x (index j), axis 3 = y (index k).
 *   A field array holds 3 components, component-major: F[c][k][j][i], c = 0,1,2,
 *   ny = 1 when ndim == 2.  Staggering: E1 (i+1/2,j,k), E2 (i,j+1/2,k), E3 (i,j,k+1/2),
 *   B1 (i,j+1/2,k+1/2), B2 (i+1/2,j,k+1/2), B3 (i+1/2,j+1/2,k); J like E; rho at nodes.
 *   In 2D, E3 and J3 sit at nodes and B1 at (i,j+1/2), B2 at (i+1/2,j), B3 at (i+1/2,j+1/2).
 *   Fields are zero outside 0 <= i < nz ("open"/conducting z ends) and periodic in x, y (the
 *   k-space solvers, PIC_SOLVER_SPECTRAL, _KT and _PSATD, are periodic along z as well).
 *
 * Particle layout (per species, structure of arrays, capacity cap):
 *   int32 cell[cap]   guarded linear cell index (iz + 1) + (nz + 2) * (ix + nx * iy),
 *                     iz in [-1, nz] (the guard values exist only transiently),
 *                     any negative value marks a dead slot;
 *   float off[ndim][cap]  in-cell offsets in [0, 1) along z, x (, y);
 *   float u[3][cap]   momentum per unit mass u = gamma v;
 *   int32 id[cap]     optional particle identifiers (NULL: none), carried by sort and
 *                     assigned to injected particles.
 *
 * Status and errors: every call returns a pic_status; nothing is thrown across the ABI
 * and the library never exits.  Asynchronous CUDA failures and device-side errors
 * (capacity overflow) are reported by the next synchronising call (pic_diag,
 * pic_get_count, pic_sync).  pic_last_error() gives a one-line description.
 * Calls are ordered on the caller's cudaStream_t (passed as void*); a handle is not
 * thread-safe.
 */
#ifndef PIC_H
#define PIC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pic_t pic_t;

typedef enum {
    PIC_OK = 0,
    PIC_ERR_ARG = 1,       /* invalid argument or configuration */
    PIC_ERR_CFL = 2,       /* dt above the leapfrog stability limit of the chosen stencil */
    PIC_ERR_CUDA = 3,      /* a CUDA runtime call failed */
    PIC_ERR_OOM = 4,       /* device allocation of library scratch failed */
    PIC_ERR_TIMEOUT = 5,   /* a bounded device-side wait gave up */
    PIC_ERR_STATE = 6,     /* call out of order (e.g. deposit before gather_push) */
    PIC_ERR_CAPACITY = 7   /* particle capacity exceeded (injection) */
} pic_status;

/* Field solvers.  YEE and CUSTOM advance E, B by finite differences on the staggered grid (Eq. 1;
 * CUSTOM: the Appendix C axial stencil, Sec. 3), fields zero outside 0 <= i < nz.  SPECTRAL and KT
 * advance the same staggered fields in k space (cuFFT transforms, one update kernel), periodic
 * along every axis, z included:
 *   PIC_SOLVER_SPECTRAL  [k]_a = k_a on every axis (Sec. 2.3);
 *   PIC_SOLVER_KT        [k]_1 = [k1]_t = (2/dt) sin(k1 dt/2) along z exactly, Yee across (the
 *                        operator Sec. 3 proposes, "advanced in k space"): vacuum waves along z
 *                        move at exactly c;
 *   PIC_SOLVER_PSATD     the analytic-time update of Appendix B (Eqs. B1-B2) with k = |k|: each
 *                        staggered component is moved to the nodes by its half-cell phase, updated
 *                        and moved back; modes on the Nyquist plane of an even axis are removed;
 *                        vacuum waves move at exactly c in every direction, for any dt (the
 *                        particle move still limits dt to one cell: dt <= min(dz, dx, dy)).
 * The forward difference from a node to the half-cell point above it has the symbol
 * e^{i k h/2} i [k]_a, the backward one e^{-i k h/2} i [k]_a; the current is scaled per axis by
 * [k]_Yee,a / [k]_a (the k-space Sec. 3 correction) so that Gauss's law with the solver's own
 * backward difference is kept.  Restrictions of the k-space solvers: moving_window = 0; particles
 * still leave at the z ends (keep them away from the ends); M, coef and coef_b are ignored; no
 * pic_adjoint_step, no batches; pic_autotune does nothing; pic_diag/pic_gauss report the residual
 * of the finite-difference divergence, which these solvers do not keep (their own residual is
 * kept to round-off).  A build without cuFFT refuses them (PIC_ERR_ARG).                      */
enum { PIC_SOLVER_YEE = 0, PIC_SOLVER_CUSTOM = 1, PIC_SOLVER_SPECTRAL = 2, PIC_SOLVER_KT = 3, PIC_SOLVER_PSATD = 4 };

/* Current filter along z (pic_config.current_filter).  The paper uses a "5 pass filter" with its
 * runs and with the self-forces of Table 2 and does not define it; PIC_FILTER_5PASS is the reading
 * that reproduces all three filtered self-forces of Table 2: four binomial passes
 * y_i = (x_{i-1} + 2 x_i + x_{i+1}) / 4 and one compensating pass
 * y_i = (-5 x_{i-1} + 14 x_i - 5 x_{i+1}) / 4, each with x = 0 outside 0 <= i < nz; k-space symbol
 * cos^8(k dz/2) (1 + 5 sin^2(k dz/2)).  It acts on J1, J2 and J3 after deposition and before the
 * Sec. 3 correction.                                                                          */
enum { PIC_FILTER_NONE = 0, PIC_FILTER_5PASS = 1 };

#define PIC_MAX_M 16        /* largest customised stencil (Appendix C uses M = 16) */
#define PIC_MAX_HLEN 24     /* current-correction taps kept on each side in FP32 */
#define PIC_MAX_SPECIES 4
#define PIC_DIAG_N 10

/* Indices of pic_diag's output vector. */
enum {
    PIC_DIAG_GAUSS_MAX = 0,   /* max |d-.E - rho - rho_bg| over interior nodes (FP64) */
    PIC_DIAG_GAUSS_RMS = 1,   /* rms of the same */
    PIC_DIAG_RHO_MAX = 2,     /* max |rho| (scale for the residual; filtered with the filter) */
    PIC_DIAG_FIELD_ENERGY = 3,/* (1/2) sum (E^2 + B^2) dV */
    PIC_DIAG_KINETIC = 4,     /* sum w m (gamma - 1) */
    PIC_DIAG_COUNT = 5,       /* live particles, all species */
    PIC_DIAG_STEP = 6,        /* completed steps */
    PIC_DIAG_SHIFTS = 7,      /* moving-window shifts done */
    PIC_DIAG_STATUS = 8,      /* device status word (0 = ok) */
    PIC_DIAG_INTERIOR = 9     /* number of nodes in the residual */
};

/* Zero-initialise a pic_config (memset or "= {0}") before setting fields: every option
 * defaults to off at 0 / NULL (current_filter, coef_b, ...).                               */
typedef struct pic_config {
    int ndim;               /* 2: (z, x); 3: (z, x, y) */
    int nz, nx, ny;         /* cells along z, x, y (ny ignored in 2D); nz, nx >= 2 */
    double dz, dx, dy;      /* cell sizes */
    double dt;              /* time step */
    int solver;             /* PIC_SOLVER_YEE, _CUSTOM, _SPECTRAL, _KT or _PSATD (see above) */
    int M;                  /* customised: number of coefficients C_1..C_M, 1 <= M <= PIC_MAX_M */
    const double* coef;     /* customised: host array of M coefficients; NULL fits them
                               (Appendix C, target [k1]_t = sin(k dt/2)/(dt/2), Sec. 3).  They
                               define d+ and d- alike ([k]_E1 = [k]_B1) unless coef_b is given */
    double fit_wk, fit_n;   /* fit weight exp(-ln2 (2k/w_k1)^n); 0 selects 0.6 and 10 */
    int shape;              /* 1: linear, 2: quadratic B-spline */
    int moving_window;      /* 1: the window moves one cell when n dt >= (s+1) dz */
    int inject_species;     /* species receiving cold plasma in the new column (-1: none) */
    int inject_ppc[3];      /* quiet-start particles per cell along z, x, y for injection */
    double rho_bg;          /* uniform background charge density (Gauss diagnostic only) */
    int sort_every;         /* pic_step sorts particles by cell every sort_every steps (0: never) */
    int current_filter;     /* PIC_FILTER_NONE or PIC_FILTER_5PASS */
    const double* coef_b;   /* NULL, or (customised solver with explicit coef) M coefficients of
                               the B-side operator d- ([k]_B1: Ampere's and Gauss's laws and the
                               Sec. 3 correction), coef then defining only the E-side d+ ([k]_E1,
                               Faraday's law): the [k]_E1 != [k]_B1 solvers Sec. 3 allows, e.g.
                               with [k]_E1 [k]_B1 = [k1]_t^2.  Not supported by pic_adjoint_step. */
    int precision;          /* arithmetic of fields, currents, offsets and momenta: 0 or 32 = FP32
                               (the only one built); any other value is refused with PIC_ERR_ARG.
                               Diagnostics always reduce in FP64. */
} pic_config;

/* ---- handle ------------------------------------------------------------------------
 * pic_create validates cfg, fits the customised coefficients when cfg->coef is NULL,
 * computes the correction taps h (from the B-side coefficients), checks dt against the
 * stability limit
 *   (dt/2)^2 (max_k [k]_E1 [k]_B1 + sum_perp (2/d_perp)^2) <= 1   (Eq. wave, leapfrog, App. C)
 * (PIC_ERR_CFL above it; PIC_ERR_ARG if [k]_E1 [k]_B1 changes sign), and allocates the library's scratch on the current device:
 * the second field buffer of the out-of-place advance, the corrected-J1 buffer, sort and
 * diagnostic workspace.  Device memory: about 7 x 4 x nz nx ny bytes + 8 x nz nx ny.   */
pic_status pic_create(const pic_config* cfg, pic_t** out);
pic_status pic_destroy(pic_t* h);
/* Text of the last error of h (h == NULL: of the last failed pic_create). Never NULL. */
const char* pic_last_error(const pic_t* h);

/* ---- host-only helpers (no GPU needed) ------------------------------------------------
 * Appendix C least-squares fit of C_1..C_M to the Sec. 3 target [k1]_t with kappa = dz/dt,
 * constraint sum (2l-1) C_l = 1 (p = 2), weight w_k1 = wk, order n.  C_out: M doubles.   */
pic_status pic_fit_coefficients(double kappa, int M, double wk, double n, double* C_out);
/* The B side of a split pair (Sec. 3: [k]_E1 != [k]_B1 with [k]_E1 [k]_B1 = [k1]_t^2): the same fit
 * with the target [k1]_t^2 / [k]_E1, [k]_E1 the operator of the ME coefficients CE (CE = {1}: a Yee
 * E side).  The pair keeps the fundamental-zone Cerenkov cancellation of [k]_1 = [k1]_t (the E1
 * numerator [w]_t^2 - [k]_E1 [k]_B1 of Eq. EM); the transverse force E2 - beta B3 then carries the
 * factor [w]_t / [k]_B1 != 1 of Eq. EM.  C_out: M doubles; use as pic_config coef_b with coef = CE
 * (padded with zeros to M).                                                                   */
pic_status pic_fit_coefficients_b(double kappa, int M, double wk, double n, const double* CE, int ME, double* C_out);
/* Sec. 3 correction taps: impulse response of 1/P, P(phi) = sum_l C_l sin((2l-1)phi/2)/sin(phi/2),
 * h_out: 2*hlen+1 doubles, centre at index hlen.  PIC_ERR_ARG if P has a zero.          */
pic_status pic_correction_taps(const double* C, int M, int hlen, double* h_out);
/* Largest stable dt for the given grid and axial stencil (M = 1, C = {1}: Yee).       */
pic_status pic_cfl_dt(int ndim, double dz, double dx, double dy, const double* C, int M, double* dt_out);
/* The same for separate E-side (CE) and B-side (CB) coefficients, M each: the limit of the
 * product [k]_E1 [k]_B1; PIC_ERR_ARG if that product changes sign (no stable dt).         */
pic_status pic_cfl_dt_split(int ndim, double dz, double dx, double dy, const double* CE, const double* CB, int M,
                            double* dt_out);
/* Largest stable dt of a k-space solver (PIC_SOLVER_SPECTRAL, _KT or _PSATD): the leapfrog
 * needs (dt/2)^2 max_k sum_a [k]_a^2 <= 1, reached at the Nyquist wavenumber of every axis;
 * spectral: dt = 2 / sqrt(sum_a (pi/h_a)^2); KT: sin^2(pi dt/(2 dz)) + sum_perp (dt/h)^2 = 1;
 * PSATD: the field update is stable for any dt, the particle move limits it to min(dz, dx, dy).
 * PIC_ERR_ARG for another solver or non-positive sizes.                                   */
pic_status pic_cfl_dt_kspace(int ndim, int solver, double dz, double dx, double dy, double* dt_out);
/* Coefficients and taps a handle uses (C_out: PIC_MAX_M, h_out: 2*PIC_MAX_HLEN+1); C_out is
 * the E-side set.  pic_get_coefficients_b: the B-side set (Cb_out: PIC_MAX_M) and whether it
 * was given separately (split = 1).                                                     */
pic_status pic_get_coefficients(const pic_t* h, double* C_out, int* M, double* h_out, int* hlen);
pic_status pic_get_coefficients_b(const pic_t* h, double* Cb_out, int* split);

/* ---- binding caller-owned device memory ---------------------------------------------
 * E, B, J: device pointers to 3 * ny * nx * nz floats each (layout above).  The library
 * reads and writes E and B in place (after every completed call the current fields are
 * in these arrays) and uses J as the current of the last deposit.                       */
pic_status pic_bind_fields(pic_t* h, float* E, float* B, float* J);
/* Species s (0 <= s < PIC_MAX_SPECIES): arrays of the layout above with capacity cap and
 * n live particles at slots [0, n).  q, m: charge and mass of one physical particle
 * (electron: -1, 1); w: weight, so one macro-particle carries charge q w and the charge
 * density it adds at a node is q w S / (cell volume).  Rebinding replaces the species.  */
pic_status pic_bind_species(pic_t* h, int s, int32_t* cell, float* off, float* u, int32_t* id,
                            int64_t n, int64_t cap, double q, double m, double w);

/* ---- the step (all calls enqueue on stream and return without synchronising) ----------
 * pic_gather_push: for every live particle, apply a pending window shift, interpolate
 *   E^n, B^n at x^n (shape-weighted, staggered), Boris u^{n-1/2} -> u^{n+1/2}, and move
 *   x^{n+1} = x^n + dt u/gamma; the old position is kept in library scratch.
 * pic_deposit: zero J, deposit J^{n+1/2} from the old and new positions (Esirkepov) for all
 *   species, apply the current filter (if configured) to J1, J2, J3 and the Sec. 3 correction
 *   to J1 (customised stencil), and retire particles that left 0 <= z < nz.  Requires a
 *   preceding pic_gather_push (else PIC_ERR_STATE).
 * pic_field_advance: B^{n+1/2} = B^n - dt/2 d+xE^n, E^{n+1} = E^n + dt (d-xB^{n+1/2} - J),
 *   B^{n+1} = B^{n+1/2} - dt/2 d+xE^{n+1} (Eq. 1); completes step n.  If the window is due,
 *   the fields are shifted one cell towards -z, the front column zeroed and the injected
 *   column of cold plasma appended to inject_species.
 * pic_step: nsteps x (gather_push + deposit + field_advance), with the particle part fused
 *   into one kernel per species; sorts by cell every sort_every steps.                  */
pic_status pic_gather_push(pic_t* h, void* stream);
pic_status pic_deposit(pic_t* h, void* stream);
pic_status pic_field_advance(pic_t* h, void* stream);
pic_status pic_step(pic_t* h, int nsteps, void* stream);
/* The current filter of PIC_FILTER_5PASS applied once, in place, to the bound J (J1, J2, J3),
 * whatever cfg.current_filter says; pic_deposit and pic_step run the same kernel after the
 * deposit when the handle is configured with the filter.  Zero current outside 0 <= i < nz. */
pic_status pic_filter_current(pic_t* h, void* stream);
/* Counting sort of every species (dead slots removed; ids follow their particles).  Order: tiles
 * of 8 x 8 (z, x) cells in 2D and 4 x 4 x 4 (z, x, y) cells in 3D in columns along z, columns
 * along x then y; the tile order snakes (z reversed in odd columns, x reversed in odd rows of
 * columns: consecutive tiles are neighbours); cells z-fastest then x then y inside a tile. */
pic_status pic_sort(pic_t* h, void* stream);

/* ---- diagnostics (FP64 on the GPU) ----------------------------------------------------
 * pic_diag fills out[PIC_DIAG_N] (indices above) and synchronises stream.  The Gauss
 * residual d-.E - rho - rho_bg uses the same d- as Ampere's law (customised stencil
 * included) and skips nodes within (M + hlen + 2) cells of the z ends (2 for Yee), plus 5
 * with the current filter.  With the filter, the field advance keeps Gauss's law for the
 * filtered charge, so pic_diag, pic_gauss and pic_gauss_static filter rho along z the same way
 * (in FP64) before taking the residual; pic_rho always returns the unfiltered density.    */
pic_status pic_diag(pic_t* h, double* out, void* stream);
/* rho (FP64, nz*nx*ny doubles, device) of all live particles at the current positions. */
pic_status pic_rho(pic_t* h, double* rho, void* stream);
/* G = d-.E - rho - rho_bg at every node (FP64, device). */
pic_status pic_gauss(pic_t* h, double* G, void* stream);
/* ---- Gauss residual without allocating ----------------------------------------------
 * The paper has no counterpart to this entry point; it is a convenience of this library.
 * pic_gauss needs an FP64 charge-density buffer of nz*nx*ny doubles, which the handle
 * allocates with cudaMalloc.  Some callers cannot allocate at the moment they want the
 * diagnostic: programs that pre-allocate a fixed device-memory budget at start-up and forbid
 * later growth, and time-critical loops that must not call cudaMalloc because it can block
 * until the whole device is idle.  pic_gauss_static computes exactly what pic_gauss computes
 * (G = d-.E - rho - rho_bg, FP64, written to the caller's device array G of nz*nx*ny
 * doubles) but takes its charge-density scratch from one array of PIC_STATIC_RHO_CELLS
 * doubles (8 MiB) compiled into the library; every GPU that loads the library holds that
 * array until the process exits.  The call makes no cudaMalloc, cudaFree or other
 * allocating call.
 *   - Grids with more than PIC_STATIC_RHO_CELLS nodes are refused with PIC_ERR_ARG.
 *   - The handle's device must be current.  pic_create looks up the array's device address
 *     (cudaGetSymbolAddress, with the handle's device current) and keeps it in the handle; with
 *     CUDA's lazy module loading that lookup is also what loads the array onto the device, so
 *     its 8 MiB are placed when the handle is created, not by pic_gauss_static.
 *   - All calls share the single array.  It is cleared at the start of every call, so
 *     results never depend on an earlier call, but two calls that run at the same time on
 *     the GPU (different streams or handles) race on it and give wrong results: order them
 *     on one stream or synchronise between them.                                          */
#define PIC_STATIC_RHO_CELLS (1 << 20)
pic_status pic_gauss_static(pic_t* h, double* G, void* stream);

/* Live-particle count of species s (synchronises stream). */
pic_status pic_get_count(pic_t* h, int s, int64_t* n, void* stream);
/* Completed steps, window shifts, and whether a shift is still pending on the particles. */
pic_status pic_get_state(const pic_t* h, int64_t* step, int64_t* shifts, int* pending_shift);
/* Next id given to an injected particle. */
pic_status pic_get_next_id(const pic_t* h, int64_t* next_id);
/* Restore the counters of a saved run (checkpoint/resume): completed steps, window shifts,
 * whether a shift is pending on the particles, and the next injected particle id.  The
 * fields and particles themselves are the caller's arrays (rebind the species to set counts). */
pic_status pic_set_state(pic_t* h, int64_t step, int64_t shifts, int pending_shift, int64_t next_id);

/* Synchronise stream and report any CUDA or device-side error. */
pic_status pic_sync(pic_t* h, void* stream);

/* ---- kernel timing (CUDA events on the caller's stream) --------------------------------
 * pic_timing(h, 1) starts collecting: every later kernel launch of h is bracketed by a pair
 * of events on its stream and counted, per class below; pic_timing(h, 0) stops.
 * pic_timing_read synchronises stream and returns, per class, the summed event time (ms)
 * and the number of kernel launches since collection started.                           */
enum {
    PIC_T_PARTICLES = 0,   /* gather + push (+ deposit when fused), per species */
    PIC_T_DEPOSIT = 1,     /* unfused deposition and zeroing of J */
    PIC_T_CORRECTION = 2,  /* Sec. 3 current correction (without the filter) */
    PIC_T_FIELDS = 3,      /* field advance (and copies back to the bound arrays) */
    PIC_T_SORT = 4,        /* counting sort */
    PIC_T_WINDOW = 5,      /* injection of the new plasma column */
    PIC_T_DIAG = 6,        /* rho, Gauss residual, reductions */
    PIC_T_FILTER = 7,      /* current filter along z (with the correction, one fused kernel) */
    PIC_TIMING_N = 8
};
pic_status pic_timing(pic_t* h, int enable);
pic_status pic_timing_read(pic_t* h, double* ms, int64_t* launches, void* stream);

/* ---- adjoint of the field step (gradients with respect to the axial coefficients) ---------
 * For a loss L of the fields after some steps, with particle currents that do not depend on the
 * fields (a rigidly moving beam), pic_adjoint_step takes the adjoint (aE, aB) = dL/d(E, B) at
 * the end of one step back to the start of that step and adds the step's contribution to
 * dL/dC_l (the Sec. 3 / Appendix C axial coefficients, including their effect through the
 * Sec. 3 current correction) to grad.  Handles created with coef_b are refused (PIC_ERR_ARG).
 *   E, B:   forward fields at the start of the step (device, 3 nz nx ny floats each);
 *   J:      the (filtered and corrected) current of that step, as pic_step / pic_deposit left
 *           it in J (the filter precedes the correction and does not depend on C);
 *   aE, aB: device, updated in place; grad: device double[M], accumulated (not cleared).
 * The transposed operators use d-x = (d+x)^T (the pair of Appendix C), so the adjoint step is
 * the leapfrog with the roles of d+ and d- exchanged.  Library scratch: 7 nz nx ny floats.  */
pic_status pic_adjoint_step(pic_t* h, const float* E, const float* B, const float* J, float* aE, float* aB,
                            double* grad, void* stream);

/* ---- tile autotuner ----------------------------------------------------------------------
 * pic_autotune times each field-advance tile variant on the handle's bound fields (results go
 * to library scratch; the state is unchanged; synchronises stream) and keeps the fastest for
 * later steps.  The choice is cached per (ndim, stencil class, grid) for the process.
 * pic_get_tuning: chosen variant, per-variant time in ms (0: not timed; ms needs
 * PIC_MAX_TILE_VARIANTS entries) and the number of variants.  2D (z x x): 0 = 128x8,
 * 1 = 256x4, 2 = 64x16, 3 = 256x8 with one cell per thread and stage, 4 = 128x8, 5 = 256x4,
 * 6 = 128x4, 7 = 256x8 register-blocked (four z cells per thread, 128-bit shared loads),
 * 8..11 register-blocked z segments of 448, 384, 960, 192 cells that march along x with the
 * next rows prefetched;
 * 3D (z x x x y): 0 = 64x4x4, 1 = 128x4x2, 2 = 32x8x4, 3..5 the same shapes register-
 * blocked, 6..9 register-blocked columns that march along y (z x x = 128x4 with 256 or 128
 * threads, 128x8, 64x8), 10, 11 the same with the next planes prefetched (128x8 with 512
 * threads, 64x4 with 128).  Without pic_autotune a handle uses 0 for Yee and the register-
 * blocked 128x8 (2D) or y-marching prefetch-ring 128x8 (3D) tile for customised stencils.  */
#define PIC_MAX_TILE_VARIANTS 16
pic_status pic_autotune(pic_t* h, void* stream);
pic_status pic_get_tuning(const pic_t* h, int* variant, double* ms, int* nvariants);
/* Force a field-advance tile variant (0 <= variant < nvariants). */
pic_status pic_set_tuning(pic_t* h, int variant);

/* ---- batched runs: many independent instances per launch --------------------------------
 * A batch holds n independent 2D or 3D runs (no moving window, no sort), each with its own
 * grid, dt, stencil (Yee or customised, own coefficients), shape and one particle species.
 * pic_batch_step advances all of them with one launch per kernel class and step (J zero,
 * gather/push/deposit, filter, correction, field advance per stencil class), recorded once into
 * CUDA graphs (32 steps, replayed while at least 32 remain, and two steps, one per field-buffer
 * parity) and replayed on the caller's stream.  The
 * field advance of a stencil class walks one work list over all its instances' tiles; the first
 * pic_batch_step after binding times the batched tile variants (one cell per thread, register-
 * blocked, and in 2D x-marching z segments) on the bound fields and keeps the fastest per class
 * (that call synchronises the stream).
 * Instance i is an ordinary handle (pic_batch_instance) for binding and diagnostics; bind its
 * fields and species before the first pic_batch_step.  After pic_batch_step returns (on the
 * stream) the bound field arrays of every instance hold the current fields.              */
typedef struct pic_batch_t pic_batch_t;
pic_status pic_batch_create(const pic_config* cfgs, int n, pic_batch_t** out);
pic_status pic_batch_instance(pic_batch_t* b, int i, pic_t** h);
pic_status pic_batch_step(pic_batch_t* b, int nsteps, void* stream);
/* Field-advance variant chosen per stencil class (variant[4]: classes M <= 1, 4, 8, 16; -1 when
 * the class has no instance; 0 one cell per thread, 1 register-blocked, 2 x-marching) and the
 * timed ms of one launch per variant (ms[12], 3 per class; 0 when not timed). */
pic_status pic_batch_get_tuning(const pic_batch_t* b, int* variant, double* ms);
pic_status pic_batch_destroy(pic_batch_t* b);

#ifdef __cplusplus
}
#endif

#endif /* PIC_H */
