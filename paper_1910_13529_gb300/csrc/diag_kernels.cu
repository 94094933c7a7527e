// FP64 diagnostics: Gauss residual d-.E - rho - rho_bg (Eq. Gauss of Sec. 2.1, with the same
// axial d- as Ampere's law), field and kinetic energy.  FP32 field values are widened to FP64
// before any arithmetic; reductions accumulate in FP64.
#include <cuda_runtime.h>

#include "pic_internal.h"

namespace pic {

namespace {

__device__ __forceinline__ double ld(const float* f, long long o) { return (double)__ldg(f + o); }

// d-.E at node (i, j, k) in FP64; E is zero outside 0 <= i < nz, periodic in x, y.
__device__ double div_e(const GridP& g, const StencilP& st, const float* E, int i, int j, int k) {
    const long long N = g.ncell;
    const long long row = ((long long)k * g.nx + j) * g.nz;
    double dz = 0.0;
    for (int l = 1; l <= st.M; ++l) {
        int a = i + l - 1, b = i - l;
        double fa = (a >= 0 && a < g.nz) ? ld(E, row + a) : 0.0;
        double fb = (b >= 0 && b < g.nz) ? ld(E, row + b) : 0.0;
        dz += (double)st.Cm[l - 1] * (fa - fb);   // the B-side d- of Ampere's law
    }
    dz /= (double)g.dz;
    int jm = j == 0 ? g.nx - 1 : j - 1;
    double dx = (ld(E + N, row + i) - ld(E + N, ((long long)k * g.nx + jm) * g.nz + i)) / (double)g.dx;
    double dy = 0.0;
    if (g.ndim == 3) {
        int km = k == 0 ? g.ny - 1 : k - 1;
        dy = (ld(E + 2 * N, row + i) - ld(E + 2 * N, ((long long)km * g.nx + j) * g.nz + i)) / (double)g.dy;
    }
    return dz + dx + dy;
}

__global__ void gauss_kernel(GridP g, StencilP st, const float* E, const double* rho, double rho_bg,
                             double* G) {
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.ncell) return;
    int i = (int)(c % g.nz);
    long long r = c / g.nz;
    int j = (int)(r % g.nx), k = (int)(r / g.nx);
    G[c] = div_e(g, st, E, i, j, k) - rho[c] - rho_bg;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// non-negative doubles order like their bit patterns
__device__ __forceinline__ void atomic_max_nonneg(double* a, double v) {
    atomicMax(reinterpret_cast<unsigned long long*>(a), (unsigned long long)__double_as_longlong(v));
}

// acc: [0] max|G| [1] sum G^2 [2] max|rho| [3] sum (E^2+B^2) [4] kinetic [5] interior nodes
//      [6] live particles
__global__ void __launch_bounds__(256) diag_kernel(GridP g, StencilP st, const float* E, const float* B,
                                                   const double* rho, double rho_bg, int margin,
                                                   double* acc) {
    double gmax = 0.0, g2 = 0.0, rmax = 0.0, w = 0.0, cnt = 0.0;
    const long long N = g.ncell;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        int i = (int)(c % g.nz);
        long long r = c / g.nz;
        int j = (int)(r % g.nx), k = (int)(r / g.nx);
        for (int q = 0; q < 3; ++q) {
            double e = ld(E, q * N + c), b = ld(B, q * N + c);
            w += e * e + b * b;
        }
        double rv = rho[c];
        rmax = fmax(rmax, fabs(rv));
        if (i >= margin && i < g.nz - margin) {
            double G = div_e(g, st, E, i, j, k) - rv - rho_bg;
            gmax = fmax(gmax, fabs(G));
            g2 += G * G;
            cnt += 1.0;
        }
    }
    __shared__ double sh[5][8];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    gmax = warp_max(gmax);
    g2 = warp_sum(g2);
    rmax = warp_max(rmax);
    w = warp_sum(w);
    cnt = warp_sum(cnt);
    if (lane == 0) {
        sh[0][wid] = gmax;
        sh[1][wid] = g2;
        sh[2][wid] = rmax;
        sh[3][wid] = w;
        sh[4][wid] = cnt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int nw = blockDim.x >> 5;
        double a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0;
        for (int q = 0; q < nw; ++q) {
            a0 = fmax(a0, sh[0][q]);
            a1 += sh[1][q];
            a2 = fmax(a2, sh[2][q]);
            a3 += sh[3][q];
            a4 += sh[4][q];
        }
        atomic_max_nonneg(acc + 0, a0);
        atomicAdd(acc + 1, a1);
        atomic_max_nonneg(acc + 2, a2);
        atomicAdd(acc + 3, a3);
        atomicAdd(acc + 5, a4);
    }
}

__global__ void __launch_bounds__(256) kinetic_kernel(SpeciesP sp, double* acc) {
    double e = 0.0, alive = 0.0;
    const long long n = *sp.count;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        if (sp.cell[p] < 0) continue;
        double u0 = sp.u[p], u1 = sp.u[sp.cap + p], u2 = sp.u[2 * sp.cap + p];
        e += sqrt(1.0 + u0 * u0 + u1 * u1 + u2 * u2) - 1.0;
        alive += 1.0;
    }
    e = warp_sum(e);
    alive = warp_sum(alive);
    __shared__ double sh[2][8];
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = e;
        sh[1][threadIdx.x >> 5] = alive;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, c = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
            a += sh[0][q];
            c += sh[1][q];
        }
        atomicAdd(acc + 4, a * sp.wm);
        atomicAdd(acc + 6, c);
    }
}

}  // namespace

cudaError_t launch_gauss(const GridP& g, const StencilP& st, const float* E, const double* rho,
                         double rho_bg, double* G, cudaStream_t s) {
    gauss_kernel<<<(unsigned)((g.ncell + 255) / 256), 256, 0, s>>>(g, st, E, rho, rho_bg, G);
    return cudaGetLastError();
}

cudaError_t launch_diag_reduce(const GridP& g, const StencilP& st, const float* E, const float* B,
                               const double* rho, double rho_bg, int margin, double* acc,
                               cudaStream_t s) {
    long long want = (g.ncell + 255) / 256;
    unsigned blocks = (unsigned)(want < 152 * 8 ? want : 152 * 8);
    diag_kernel<<<blocks, 256, 0, s>>>(g, st, E, B, rho, rho_bg, margin, acc);
    return cudaGetLastError();
}

cudaError_t launch_kinetic(const GridP& g, const SpeciesP& sp, long long extent, double* acc,
                           cudaStream_t s) {
    (void)g;
    if (extent <= 0) return cudaSuccess;
    long long want = (extent + 255) / 256;
    unsigned blocks = (unsigned)(want < 152 * 8 ? want : 152 * 8);
    kinetic_kernel<<<blocks, 256, 0, s>>>(sp, acc);
    return cudaGetLastError();
}

}  // namespace pic
