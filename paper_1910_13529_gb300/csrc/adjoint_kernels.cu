// Adjoint of the field advance (Eq. 1 leapfrog with the customised axial stencil of Sec. 3 /
// Appendix C) and of the Sec. 3 current correction, for gradients of a loss with respect to
// the axial coefficients C_l.
//
// Forward step (T = d+ x, S = d- x = T^T, h = dt/2):
//   B' = B - h T E;   E' = E + dt (S B' - J);   B'' = B' - h T E'
// Adjoint (l_E, l_B: adjoints of the step's outputs), with T_l, S_l the parts of T, S carried
// by coefficient l (axial taps l only):
//   g_l += -h <l_B, T_l E'>;  l_E <- l_E - h S l_B
//   g_l += dt <l_E, S_l B'>;  l_B <- l_B + dt T l_E;  l_J1 = -dt l_E1
//   g_l += -h <l_B, T_l E>;   l_E <- l_E - h S l_B
// Correction J1c = P^{-1} J1 (P symmetric, dP/dC_l = the box filter of half-width l-1):
//   g_l += -<P^{-1} l_J1, P_l J1c> = dt <P^{-1} l_E1, P_l J1c>.
// All sums are FP64 block reductions; fields are FP32.
#include <cuda_runtime.h>

#include "pic_internal.h"

namespace pic {

namespace {

__device__ __forceinline__ float fz(const float* f, int nz, long long row, int i) {
    return (i >= 0 && i < nz) ? __ldg(f + row + i) : 0.f;
}

__device__ __forceinline__ int wrapm(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

struct Cell {
    int i, j, k;
    long long c, row;
};

__device__ __forceinline__ Cell cell_of(const GridP& g, long long c) {
    Cell q;
    q.c = c;
    q.i = (int)(c % g.nz);
    long long r = c / g.nz;
    q.j = (int)(r % g.nx);
    q.k = (int)(r / g.nx);
    q.row = c - q.i;
    return q;
}

__device__ __forceinline__ long long rowof(const GridP& g, int j, int k) { return ((long long)k * g.nx + j) * g.nz; }

// axial d+ (sum over taps) and d- at cell i of a row
__device__ __forceinline__ float dzp(const StencilP& st, const float* f, int nz, long long row, int i) {
    float s = 0.f;
    for (int l = 1; l <= st.M; ++l) s += st.C[l - 1] * (fz(f, nz, row, i + l) - fz(f, nz, row, i - l + 1));
    return s;
}
__device__ __forceinline__ float dzm(const StencilP& st, const float* f, int nz, long long row, int i) {
    float s = 0.f;
    for (int l = 1; l <= st.M; ++l) s += st.C[l - 1] * (fz(f, nz, row, i + l - 1) - fz(f, nz, row, i - l));
    return s;
}

// out = X + a T Y  (T = d+ x, output at B positions)
__global__ void curl_plus_update_kernel(GridP g, StencilP st, const float* X, const float* Y, float a, float* out) {
    const long long N = g.ncell;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        Cell q = cell_of(g, c);
        const float* Y1 = Y;
        const float* Y2 = Y + N;
        const float* Y3 = Y + 2 * N;
        const long long rxp = rowof(g, wrapm(q.j + 1, g.nx), q.k);
        const long long ryp = g.ndim == 3 ? rowof(g, q.j, wrapm(q.k + 1, g.ny)) : q.row;
        const float idz = 1.f / g.dz, idx = 1.f / g.dx, idy = g.ndim == 3 ? 1.f / g.dy : 0.f;
        float dxE3 = (__ldg(Y3 + rxp + q.i) - __ldg(Y3 + c)) * idx;
        float dxE1 = (__ldg(Y1 + rxp + q.i) - __ldg(Y1 + c)) * idx;
        float dyE2 = (__ldg(Y2 + ryp + q.i) - __ldg(Y2 + c)) * idy;
        float dyE1 = (__ldg(Y1 + ryp + q.i) - __ldg(Y1 + c)) * idy;
        float dzE3 = dzp(st, Y3, g.nz, q.row, q.i) * idz;
        float dzE2 = dzp(st, Y2, g.nz, q.row, q.i) * idz;
        out[c] = X[c] + a * (dxE3 - dyE2);
        out[N + c] = X[N + c] + a * (dyE1 - dzE3);
        out[2 * N + c] = X[2 * N + c] + a * (dzE2 - dxE1);
    }
}

// out = X + a S Y + b J  (S = d- x, output at E positions); J may be null
__global__ void curl_minus_update_kernel(GridP g, StencilP st, const float* X, const float* Y, const float* J, float a,
                                         float b, float* out) {
    const long long N = g.ncell;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        Cell q = cell_of(g, c);
        const float* Y1 = Y;
        const float* Y2 = Y + N;
        const float* Y3 = Y + 2 * N;
        const long long rxm = rowof(g, wrapm(q.j - 1, g.nx), q.k);
        const long long rym = g.ndim == 3 ? rowof(g, q.j, wrapm(q.k - 1, g.ny)) : q.row;
        const float idz = 1.f / g.dz, idx = 1.f / g.dx, idy = g.ndim == 3 ? 1.f / g.dy : 0.f;
        float dxB3 = (__ldg(Y3 + c) - __ldg(Y3 + rxm + q.i)) * idx;
        float dxB1 = (__ldg(Y1 + c) - __ldg(Y1 + rxm + q.i)) * idx;
        float dyB2 = (__ldg(Y2 + c) - __ldg(Y2 + rym + q.i)) * idy;
        float dyB1 = (__ldg(Y1 + c) - __ldg(Y1 + rym + q.i)) * idy;
        float dzB3 = dzm(st, Y3, g.nz, q.row, q.i) * idz;
        float dzB2 = dzm(st, Y2, g.nz, q.row, q.i) * idz;
        float j1 = J ? J[c] : 0.f, j2 = J ? J[N + c] : 0.f, j3 = J ? J[2 * N + c] : 0.f;
        out[c] = X[c] + a * (dxB3 - dyB2) + b * j1;
        out[N + c] = X[N + c] + a * (dyB1 - dzB3) + b * j2;
        out[2 * N + c] = X[2 * N + c] + a * (dzB2 - dxB1) + b * j3;
    }
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// block sums of acc[0..M) added to grad[0..M) (FP64 atomics)
__device__ __forceinline__ void flush_grad(double* acc, int M, double* grad) {
    __shared__ double part[PIC_MAX_M][8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int l = 0; l < M; ++l) {
        double v = warp_sum_d(acc[l]);
        if (lane == 0) part[l][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < M) {
        double v = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) v += part[threadIdx.x][q];
        atomicAdd(grad + threadIdx.x, v);
    }
}

// grad_l += a * sum [ L2 (-D+_l F3) + L3 (D+_l F2) ],  D+_l f_i = (f_{i+l} - f_{i-l+1}) / dz
__global__ void __launch_bounds__(256) grad_plus_kernel(GridP g, int M, const float* L, const float* F, double a,
                                                        double* grad) {
    const long long N = g.ncell;
    double acc[PIC_MAX_M];
    for (int l = 0; l < M; ++l) acc[l] = 0.0;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        Cell q = cell_of(g, c);
        const double l2 = L[N + c], l3 = L[2 * N + c];
        if (l2 == 0.0 && l3 == 0.0) continue;
        for (int l = 1; l <= M; ++l) {
            double d3 = (double)fz(F + 2 * N, g.nz, q.row, q.i + l) - (double)fz(F + 2 * N, g.nz, q.row, q.i - l + 1);
            double d2 = (double)fz(F + N, g.nz, q.row, q.i + l) - (double)fz(F + N, g.nz, q.row, q.i - l + 1);
            acc[l - 1] += -l2 * d3 + l3 * d2;
        }
    }
    const double s = a / (double)g.dz;
    for (int l = 0; l < M; ++l) acc[l] *= s;
    flush_grad(acc, M, grad);
}

// grad_l += a * sum [ L2 (-D-_l F3) + L3 (D-_l F2) ],  D-_l f_i = (f_{i+l-1} - f_{i-l}) / dz
__global__ void __launch_bounds__(256) grad_minus_kernel(GridP g, int M, const float* L, const float* F, double a,
                                                         double* grad) {
    const long long N = g.ncell;
    double acc[PIC_MAX_M];
    for (int l = 0; l < M; ++l) acc[l] = 0.0;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        Cell q = cell_of(g, c);
        const double l2 = L[N + c], l3 = L[2 * N + c];
        if (l2 == 0.0 && l3 == 0.0) continue;
        for (int l = 1; l <= M; ++l) {
            double d3 = (double)fz(F + 2 * N, g.nz, q.row, q.i + l - 1) - (double)fz(F + 2 * N, g.nz, q.row, q.i - l);
            double d2 = (double)fz(F + N, g.nz, q.row, q.i + l - 1) - (double)fz(F + N, g.nz, q.row, q.i - l);
            acc[l - 1] += -l2 * d3 + l3 * d2;
        }
    }
    const double s = a / (double)g.dz;
    for (int l = 0; l < M; ++l) acc[l] *= s;
    flush_grad(acc, M, grad);
}

// grad_l += a * sum_i W_i (P_l J1c)_i,  (P_l f)_i = sum_{|m| < l} f_{i-m}
__global__ void __launch_bounds__(256) grad_corr_kernel(GridP g, int M, const float* W, const float* J1c, double a,
                                                        double* grad) {
    const long long N = g.ncell;
    double acc[PIC_MAX_M];
    for (int l = 0; l < M; ++l) acc[l] = 0.0;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const double w = W[c];
        if (w == 0.0) continue;
        Cell q = cell_of(g, c);
        double box = fz(J1c, g.nz, q.row, q.i);
        acc[0] += w * box;
        for (int l = 2; l <= M; ++l) {
            box += (double)fz(J1c, g.nz, q.row, q.i - (l - 1)) + (double)fz(J1c, g.nz, q.row, q.i + (l - 1));
            acc[l - 1] += w * box;
        }
    }
    for (int l = 0; l < M; ++l) acc[l] *= a;
    flush_grad(acc, M, grad);
}

inline unsigned gblocks(long long n) {
    long long b = (n + 255) / 256;
    return (unsigned)(b > 152 * 8 ? 152 * 8 : (b < 1 ? 1 : b));
}

}  // namespace

cudaError_t launch_curl_plus_update(const GridP& g, const StencilP& st, const float* X, const float* Y, float a,
                                    float* out, cudaStream_t s) {
    curl_plus_update_kernel<<<gblocks(g.ncell), 256, 0, s>>>(g, st, X, Y, a, out);
    return cudaGetLastError();
}

cudaError_t launch_curl_minus_update(const GridP& g, const StencilP& st, const float* X, const float* Y, const float* J,
                                     float a, float b, float* out, cudaStream_t s) {
    curl_minus_update_kernel<<<gblocks(g.ncell), 256, 0, s>>>(g, st, X, Y, J, a, b, out);
    return cudaGetLastError();
}

cudaError_t launch_grad_plus(const GridP& g, int M, const float* L, const float* F, double a, double* grad,
                             cudaStream_t s) {
    grad_plus_kernel<<<gblocks(g.ncell), 256, 0, s>>>(g, M, L, F, a, grad);
    return cudaGetLastError();
}

cudaError_t launch_grad_minus(const GridP& g, int M, const float* L, const float* F, double a, double* grad,
                              cudaStream_t s) {
    grad_minus_kernel<<<gblocks(g.ncell), 256, 0, s>>>(g, M, L, F, a, grad);
    return cudaGetLastError();
}

cudaError_t launch_grad_corr(const GridP& g, int M, const float* W, const float* J1c, double a, double* grad,
                             cudaStream_t s) {
    grad_corr_kernel<<<gblocks(g.ncell), 256, 0, s>>>(g, M, W, J1c, a, grad);
    return cudaGetLastError();
}

}  // namespace pic
