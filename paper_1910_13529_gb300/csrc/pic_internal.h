// Internal declarations shared by the CUDA translation units of libpic.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/pic.h"

namespace pic {

// Division by a run-time constant d without an integer divide (Granlund-Montgomery):
// n / d = (t + ((n - t) >> 1)) >> (s - 1), t = umulhi(m, n), for all 32-bit n.
struct FastDiv {
    uint32_t d, m;
    int s;   // -1: d == 1
};

inline FastDiv make_fastdiv(uint32_t d) {
    FastDiv f{d, 0u, -1};
    if (d <= 1) return f;
    int l = 0;
    while ((1ull << l) < d) ++l;
    f.m = (uint32_t)((((1ull << 32) * ((1ull << l) - d)) / d) + 1);
    f.s = l;
    return f;
}

// Grid constants passed by value to every kernel.
struct GridP {
    int ndim;
    int nz, nx, ny;     // cells
    int nzg;            // nz + 2: z extent of the guarded particle cell index
    long long ncell;    // nz * nx * ny
    float dz, dx, dy, dt;
    int shape;          // 1 or 2
    FastDiv div_nzg, div_nx;   // filled by the particle launchers
};

// Axial stencil (Appendix C).  M = 1, C[0] = 1 is the Yee difference.  C: the E-side d+
// (Faraday's law, [k]_E1); Cm: the B-side d- (Ampere's and Gauss's laws, [k]_B1), equal to C
// unless the handle was created with separate B-side coefficients.
struct StencilP {
    int M;
    float C[PIC_MAX_M];
    float Cm[PIC_MAX_M];
};

// Field-advance launch parameters.
struct FieldP {
    GridP g;
    StencilP st;
    const float* Ein;
    const float* Bin;
    const float* J1;     // current components (J1 may be the corrected copy)
    const float* J2;
    const float* J3;
    float* Eout;
    float* Bout;
    int shift;           // 1: write the result one cell towards -z, zero the front column
    int vec4;            // nz % 4 == 0 and every array 16-byte aligned (set by launch_field_advance)
};

// One species' particle arrays and per-species constants.
struct SpeciesP {
    int32_t* cell;
    float* off;          // [ndim][cap]
    float* u;            // [3][cap]
    int32_t* id;         // may be null
    int32_t* count;      // device live-slot extent
    long long cap;
    float eps;           // q dt / (2 m)   (Boris)
    float kz[2], kx[2], ky[2];   // dt/dz, dt/dx, dt/dy as float-float (hi, lo)
    float qv;            // q w / V        (charge density of one macro-particle per unit shape)
    double qv64;
    double wm;           // w m            (kinetic energy)
    int32_t* prev_cell;  // scratch for the unfused path
    float* prev_off;
};

// One instance of a batched run: its grid, its (single) species, its two field buffers.
struct PartInst {
    GridP g;
    SpeciesP sp;
    const float* E[2];   // fields read at even / odd steps
    const float* B[2];
    float* J;
};

// Current correction of one instance (customised stencil).
struct CorrInst {
    GridP g;
    float h[2 * PIC_MAX_HLEN + 1];
    int hlen;
    float* J1;
};

// Current filter of one batched instance (all three components of J).
struct FiltInst {
    GridP g;
    float* J;
    int vec4;            // nz % 4 == 0 and J 16-byte aligned
};

// Device status word bits.
enum : int { STATUS_CAPACITY = 1, STATUS_TIMEOUT = 2 };

// ---- launchers (return cudaGetLastError of the launch) ----
cudaError_t launch_field_advance(const FieldP& p, cudaStream_t s, int variant = 0);
int field_variants(int ndim);
int default_field_variant(int ndim, int M);

// batched: instance tables live in device memory
cudaError_t launch_field_advance_batch(const FieldP* inst, const int* tile_start, int ninst, int total_tiles,
                                       int ndim, int maxm, int parity, cudaStream_t s);
int field_tiles(int ndim, int maxm, int nz, int nx, int ny);
// Batched 2D field advance with the x-marching segments: work[w] = (instance, z0, first row,
// last row + 1); z segments of MARCH2_BATCH_TZ cells.
constexpr int MARCH2_BATCH_TZ = 192;
constexpr int MARCH2_BATCH_XC = 32;
// The same tile list as launch_field_advance_batch with register-blocked tiles.
cudaError_t launch_field_advance_rb_batch(const FieldP* inst, const int* tile_start, int ninst, int total_tiles,
                                          int ndim, int maxm, int parity, cudaStream_t s);
cudaError_t launch_field_advance_march2_batch(const FieldP* inst, const int4* work, int nwork, int maxm, int parity,
                                              cudaStream_t s);
cudaError_t launch_correct_j1_batch(const CorrInst* inst, int ninst, int max_rows, int max_nz, cudaStream_t s);
cudaError_t launch_push_batch(const PartInst* inst, int ninst, int ndim, int shape, long long max_extent, int parity,
                              cudaStream_t s);
cudaError_t launch_zero_j_batch(const PartInst* inst, int ninst, long long max_ncell, cudaStream_t s);
// defer (3D fused mode): library scratch of two lists of 2 + ceil(cap / 256) ints each, their
// first two ints zero on first use: the chunks whose shared-memory boxes do not fit, processed by
// the general and the per-particle kernels, which clear the lists.
cudaError_t launch_push(const GridP& g, const SpeciesP& sp, const float* E, const float* B,
                        float* J, int shift, int mode, long long extent, int* defer, cudaStream_t s);
cudaError_t launch_deposit_unfused(const GridP& g, const SpeciesP& sp, float* J, long long extent,
                                   cudaStream_t s);
// Appends the new column's cold plasma (3D: at the count rounded up to 256, patch-ordered);
// *extent, the host's upper bound of the count, is advanced accordingly.
cudaError_t launch_inject(const GridP& g, const SpeciesP& sp, const int ppc[3], long long next_id,
                          int* status, long long* extent, cudaStream_t s);
long long sort_bins(const GridP& g);
cudaError_t launch_sort(const GridP& g, const SpeciesP& sp, long long extent, int32_t* hist,
                        int32_t* blocksums, int32_t* cell_alt, float* off_alt, float* u_alt,
                        int32_t* id_alt, cudaStream_t s);
cudaError_t launch_rho(const GridP& g, const SpeciesP& sp, int shift, double* rho, long long extent,
                       cudaStream_t s);
cudaError_t launch_gauss(const GridP& g, const StencilP& st, const float* E, const double* rho,
                         double rho_bg, double* G, cudaStream_t s);
cudaError_t launch_diag_reduce(const GridP& g, const StencilP& st, const float* E, const float* B,
                               const double* rho, double rho_bg, int margin, double* acc,
                               cudaStream_t s);
cudaError_t launch_kinetic(const GridP& g, const SpeciesP& sp, long long extent, double* acc,
                           cudaStream_t s);

// ---- current filter and Sec. 3 correction along z (current_kernels.cu) ----
cudaError_t launch_correct_j1(const GridP& g, const float* taps, int hlen, float* J1, cudaStream_t s);
// filter on J1, J2, J3 and the correction on J1 in one launch (J: the three components)
cudaError_t launch_filter_correct(const GridP& g, const float* taps, int hlen, float* J, cudaStream_t s);
bool filter_vec4_ok(const float* J, int nz);
cudaError_t launch_filter_current(const GridP& g, float* J, cudaStream_t s);
cudaError_t launch_filter_rho(const GridP& g, double* rho, cudaStream_t s);
cudaError_t launch_filter_current_batch(const FiltInst* inst, int ninst, long long max_rows3, cudaStream_t s);

// ---- adjoint (adjoint_kernels.cu) ----
cudaError_t launch_curl_plus_update(const GridP& g, const StencilP& st, const float* X, const float* Y, float a,
                                    float* out, cudaStream_t s);
cudaError_t launch_curl_minus_update(const GridP& g, const StencilP& st, const float* X, const float* Y, const float* J,
                                     float a, float b, float* out, cudaStream_t s);
cudaError_t launch_grad_plus(const GridP& g, int M, const float* L, const float* F, double a, double* grad,
                             cudaStream_t s);
cudaError_t launch_grad_minus(const GridP& g, int M, const float* L, const float* F, double a, double* grad,
                              cudaStream_t s);
cudaError_t launch_grad_corr(const GridP& g, int M, const float* W, const float* J1c, double a, double* grad,
                             cudaStream_t s);

// ---- host math (host_math.cpp) ----
int fit_coefficients(double kappa, int M, double wk, double n, double* C);
int fit_coefficients_b(double kappa, int M, double wk, double n, const double* CE, int ME, double* C);
int correction_taps(const double* C, int M, int hlen, double* h);
double cfl_dt(int ndim, double dz, double dx, double dy, const double* C, int M);
// with the E-side (CE) and B-side (CB) symbols: max of their product; -1 if the product is negative
double cfl_dt_split(int ndim, double dz, double dx, double dy, const double* CE, const double* CB, int M);
// k-space field advance (PIC_SOLVER_SPECTRAL, PIC_SOLVER_KT; kspace_kernels.cu).  Status codes:
// 0 ok, 1 error (message in err), 2 device memory.
struct KSpaceState;
bool kspace_available();
int kspace_create(const GridP& g, int solver, double dz, double dx, double dy, double dt, KSpaceState** out,
                  char* err, size_t nerr);
void kspace_destroy(KSpaceState* k);
long long kspace_modes(const KSpaceState* k);
int kspace_advance(KSpaceState* k, const float* Ein, const float* Bin, const float* J, float* Eout, float* Bout,
                   cudaStream_t s, char* err, size_t nerr);
// largest stable dt of the k-space solvers (kt = 0: spectral, 1: [k1]_t along z, 2: PSATD)
double kspace_cfl_dt(int ndim, int kt, double dz, double dx, double dy);

}  // namespace pic
