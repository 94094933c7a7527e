// Field advance (Eq. 1 of Sec. 2.1, Yee operators of Sec. 2.2, customised axial stencil of
// Sec. 3 / Appendix C), for sm_103a.
//
// One kernel performs the whole leapfrog step out of place:
//   B^{n+1/2} = B^n - dt/2 d+ x E^n
//   E^{n+1}   = E^n + dt (d- x B^{n+1/2} - J)
//   B^{n+1}   = B^{n+1/2} - dt/2 d+ x E^{n+1}
// Each CTA owns a TZ x TX (x TY) output tile.  It stages E^n over the tile plus the halo the
// three stages need (3M-2 cells before and after in z, 1 before / 2 after across), computes
// B^{n+1/2} into shared memory over the tile plus the stage-2 halo, updates E in place in
// shared memory, and finishes B^{n+1}; E^n and B^n are read once and E^{n+1}, B^{n+1} written
// once per cell (60 B per cell-update with J), the halos coming from L2.  Writing to the second
// buffer lets the moving-window shift be folded into the store.
#include <cuda_runtime.h>

#include <climits>

#include <cstdint>

#include "pic_internal.h"

namespace pic {

namespace {

template <int NDIM, int MAXM, int TZ, int TX, int TY>
struct Tile {
    static constexpr int L0 = 3 * MAXM - 2;          // E^n halo before the tile (z)
    static constexpr int W0 = TZ + 6 * MAXM - 3;     // E^n z extent
    static constexpr int L1 = 2 * MAXM - 1;          // B^{n+1/2} halo before the tile
    static constexpr int W1 = TZ + 4 * MAXM - 2;     // B^{n+1/2} z extent
    static constexpr int L2 = MAXM - 1;              // E^{n+1} halo before the tile
    static constexpr int W2 = TZ + 2 * MAXM - 1;     // E^{n+1} z extent
    static constexpr int TYe = NDIM == 3 ? TY : 1;
    static constexpr int RX0 = TX + 3, RY0 = NDIM == 3 ? TY + 3 : 1;   // E rows: [-1, T+1]
    static constexpr int RX1 = TX + 2, RY1 = NDIM == 3 ? TY + 2 : 1;   // B rows: [-1, T]
    static constexpr int RX2 = TX + 1, RY2 = NDIM == 3 ? TY + 1 : 1;   // E' rows: [0, T]
    static constexpr int SE = RX0 * RY0 * W0;
    static constexpr int SB = RX1 * RY1 * W1;
    static constexpr size_t smem_bytes = sizeof(float) * 3 * (SE + SB);
};

// periodic index: a mod n in [0, n); an integer division only when a lies more than one period
// outside (grids narrower than a tile)
__device__ __forceinline__ int wrapi(int a, int n) {
    if ((unsigned)a < (unsigned)n) return a;
    if (a < 0 && a >= -n) return a + n;
    if (a >= n && a - n < n) return a - n;
    a %= n;
    return a < 0 ? a + n : a;
}

// One output tile (tz, tx, ty) of the leapfrog field step, shared memory `smem`.
template <int NDIM, int MAXM, int TZ, int TX, int TY>
__device__ __forceinline__ void advance_tile(const FieldP& p, int tz, int tx, int ty, float* smem) {
    using T = Tile<NDIM, MAXM, TZ, TX, TY>;
    float* sE = smem;                 // [3][RY0][RX0][W0]
    float* sB = smem + 3 * T::SE;     // [3][RY1][RX1][W1]

    const GridP& g = p.g;
    const int nz = g.nz, nx = g.nx, ny = g.ny;
    const long long N = g.ncell;
    const int z0 = tz * TZ;
    const int x0 = tx * TX;
    const int y0 = NDIM == 3 ? ty * TY : 0;
    const int M = p.st.M;

    const float dt = g.dt;
    const float hx = 0.5f * dt / g.dx, fx = dt / g.dx;
    const float hy = NDIM == 3 ? 0.5f * dt / g.dy : 0.f, fy = NDIM == 3 ? dt / g.dy : 0.f;
    float Ch[MAXM], Cf[MAXM];      // d+ of the half B steps (E side), d- of the E step (B side)
#pragma unroll
    for (int l = 0; l < MAXM; ++l) {
        Ch[l] = (l < M ? p.st.C[l] : 0.f) * (0.5f * dt / g.dz);
        Cf[l] = (l < M ? p.st.Cm[l] : 0.f) * (dt / g.dz);
    }

    // ---- stage 0: E^n over the full halo -------------------------------------------
    for (int idx = threadIdx.x; idx < T::RY0 * T::RX0 * T::W0; idx += blockDim.x) {
        int col = idx % T::W0;
        int r = idx / T::W0;
        int rx = r % T::RX0, ry = r / T::RX0;
        int gz = z0 + col - T::L0;
        int gx = wrapi(x0 + rx - 1, nx);
        int gy = NDIM == 3 ? wrapi(y0 + ry - 1, ny) : 0;
        float v0 = 0.f, v1 = 0.f, v2 = 0.f;
        if (gz >= 0 && gz < nz) {
            long long o = ((long long)gy * nx + gx) * nz + gz;
            v0 = __ldg(p.Ein + o);
            v1 = __ldg(p.Ein + N + o);
            v2 = __ldg(p.Ein + 2 * N + o);
        }
        sE[idx] = v0;
        sE[T::SE + idx] = v1;
        sE[2 * T::SE + idx] = v2;
    }
    __syncthreads();

    // ---- stage 1: B^{n+1/2} over x in [-1, TX], y in [-1, TY], z in [-L1, TZ+2MAXM-2] ----
    for (int idx = threadIdx.x; idx < T::RY1 * T::RX1 * T::W1; idx += blockDim.x) {
        int col = idx % T::W1;
        int r = idx / T::W1;
        int rx = r % T::RX1, ry = r / T::RX1;
        int z = col - T::L1;
        int gz = z0 + z;
        float b0 = 0.f, b1 = 0.f, b2 = 0.f;
        if (gz >= 0 && gz < nz) {
            int gx = wrapi(x0 + rx - 1, nx);
            int gy = NDIM == 3 ? wrapi(y0 + ry - 1, ny) : 0;
            long long o = ((long long)gy * nx + gx) * nz + gz;
            // E index of the same (x, y, z): rows shift by 0 (both start at -1), cols by MAXM-1
            int e = (ry * T::RX0 + rx) * T::W0 + col + (MAXM - 1);
            const float* E1 = sE;
            const float* E2 = sE + T::SE;
            const float* E3 = sE + 2 * T::SE;
            float dzE2 = 0.f, dzE3 = 0.f;
#pragma unroll
            for (int l = 0; l < MAXM; ++l) {
                dzE2 += Ch[l] * (E2[e + l + 1] - E2[e - l]);
                dzE3 += Ch[l] * (E3[e + l + 1] - E3[e - l]);
            }
            float dxE1 = E1[e + T::W0] - E1[e];
            float dxE3 = E3[e + T::W0] - E3[e];
            float dyE1 = 0.f, dyE2 = 0.f;
            if (NDIM == 3) {
                dyE1 = E1[e + T::RX0 * T::W0] - E1[e];
                dyE2 = E2[e + T::RX0 * T::W0] - E2[e];
            }
            b0 = __ldg(p.Bin + o) - (hx * dxE3 - hy * dyE2);
            b1 = __ldg(p.Bin + N + o) - (hy * dyE1 - dzE3);
            b2 = __ldg(p.Bin + 2 * N + o) - (dzE2 - hx * dxE1);
        }
        sB[idx] = b0;
        sB[T::SB + idx] = b1;
        sB[2 * T::SB + idx] = b2;
    }
    __syncthreads();

    // ---- stage 2: E^{n+1} in place over x in [0, TX], y in [0, TY], z in [-L2, TZ+MAXM-1] ----
    for (int idx = threadIdx.x; idx < T::RY2 * T::RX2 * T::W2; idx += blockDim.x) {
        int col = idx % T::W2;
        int r = idx / T::W2;
        int rx = r % T::RX2, ry = r / T::RX2;     // x = rx, y = ry
        int z = col - T::L2;
        int gz = z0 + z;
        int e = ((NDIM == 3 ? ry + 1 : 0) * T::RX0 + rx + 1) * T::W0 + z + T::L0;
        float n0 = 0.f, n1 = 0.f, n2 = 0.f;
        if (gz >= 0 && gz < nz) {
            int gx = wrapi(x0 + rx, nx);
            int gy = NDIM == 3 ? wrapi(y0 + ry, ny) : 0;
            long long o = ((long long)gy * nx + gx) * nz + gz;
            int b = ((NDIM == 3 ? ry + 1 : 0) * T::RX1 + rx + 1) * T::W1 + z + T::L1;
            const float* B1 = sB;
            const float* B2 = sB + T::SB;
            const float* B3 = sB + 2 * T::SB;
            float dzB2 = 0.f, dzB3 = 0.f;
#pragma unroll
            for (int l = 0; l < MAXM; ++l) {
                dzB2 += Cf[l] * (B2[b + l] - B2[b - l - 1]);
                dzB3 += Cf[l] * (B3[b + l] - B3[b - l - 1]);
            }
            float dxB1 = B1[b] - B1[b - T::W1];
            float dxB3 = B3[b] - B3[b - T::W1];
            float dyB1 = 0.f, dyB2 = 0.f;
            if (NDIM == 3) {
                dyB1 = B1[b] - B1[b - T::RX1 * T::W1];
                dyB2 = B2[b] - B2[b - T::RX1 * T::W1];
            }
            n0 = sE[e] + (fx * dxB3 - fy * dyB2) - dt * __ldg(p.J1 + o);
            n1 = sE[T::SE + e] + (fy * dyB1 - dzB3) - dt * __ldg(p.J2 + o);
            n2 = sE[2 * T::SE + e] + (dzB2 - fx * dxB1) - dt * __ldg(p.J3 + o);
        }
        sE[e] = n0;
        sE[T::SE + e] = n1;
        sE[2 * T::SE + e] = n2;
    }
    __syncthreads();

    // ---- stage 3: B^{n+1} on the tile; store E^{n+1}, B^{n+1} (shifted if the window moves) ----
    for (int idx = threadIdx.x; idx < T::TYe * TX * TZ; idx += blockDim.x) {
        int z = idx % TZ;
        int r = idx / TZ;
        int x = r % TX, y = r / TX;
        int gz = z0 + z, gx = x0 + x, gy = y0 + y;
        if (gz >= nz || gx >= nx || (NDIM == 3 && gy >= ny)) continue;
        int e = ((NDIM == 3 ? y + 1 : 0) * T::RX0 + x + 1) * T::W0 + z + T::L0;
        int b = ((NDIM == 3 ? y + 1 : 0) * T::RX1 + x + 1) * T::W1 + z + T::L1;
        const float* E1 = sE;
        const float* E2 = sE + T::SE;
        const float* E3 = sE + 2 * T::SE;
        float dzE2 = 0.f, dzE3 = 0.f;
#pragma unroll
        for (int l = 0; l < MAXM; ++l) {
            dzE2 += Ch[l] * (E2[e + l + 1] - E2[e - l]);
            dzE3 += Ch[l] * (E3[e + l + 1] - E3[e - l]);
        }
        float dxE1 = E1[e + T::W0] - E1[e];
        float dxE3 = E3[e + T::W0] - E3[e];
        float dyE1 = 0.f, dyE2 = 0.f;
        if (NDIM == 3) {
            dyE1 = E1[e + T::RX0 * T::W0] - E1[e];
            dyE2 = E2[e + T::RX0 * T::W0] - E2[e];
        }
        float b0 = sB[b] - (hx * dxE3 - hy * dyE2);
        float b1 = sB[T::SB + b] - (hy * dyE1 - dzE3);
        float b2 = sB[2 * T::SB + b] - (dzE2 - hx * dxE1);
        long long row = ((long long)gy * nx + gx) * nz;
        int oz = gz - p.shift;
        if (oz >= 0) {
            long long o = row + oz;
            p.Eout[o] = E1[e];
            p.Eout[N + o] = E2[e];
            p.Eout[2 * N + o] = E3[e];
            p.Bout[o] = b0;
            p.Bout[N + o] = b1;
            p.Bout[2 * N + o] = b2;
        }
        if (p.shift && gz == nz - 1) {
            long long o = row + gz;
            p.Eout[o] = 0.f;
            p.Eout[N + o] = 0.f;
            p.Eout[2 * N + o] = 0.f;
            p.Bout[o] = 0.f;
            p.Bout[N + o] = 0.f;
            p.Bout[2 * N + o] = 0.f;
        }
    }
}

// ---- register-blocked tile ---------------------------------------------------------------
// Same three stages, but every thread produces four consecutive z cells of a stage.  The axial
// derivative of those four cells needs 2 MP + 3 consecutive values of the differentiated
// component (MP = MAXM rounded up to 4); the thread reads them as MP / 2 + 1 aligned 128-bit
// shared loads into registers instead of 2 MAXM scalar loads per cell, which cuts the shared-
// memory traffic of the M = 16 stencil about four-fold.  Every halo is a multiple of 4 cells
// and all component rows start on a 16-byte boundary, so with the E windows starting one cell
// below the d+ stencil and the B windows exactly at the d- stencil, every window, every
// same-cell read and every store of the three stages is aligned:
//   B^{n+1/2} on z in [-2 MP, TZ + 2 MP), E^{n+1} on [-MP, TZ + MP), B^{n+1} on [0, TZ),
//   E^n staged on [-3 MP, TZ + 3 MP).
// E^n, B^n and J of the tile are all staged before the first stage (16-byte cp.async copies
// when nz % 4 == 0, so the CTA's global reads are in flight together); B^{n+1/2} overwrites
// B^n in place and E^{n+1} overwrites E^n.
template <int NDIM, int MAXM, int TZ, int TX, int TY>
struct TileRB {
    static constexpr int MP = (MAXM + 3) & ~3;
    static constexpr int H2 = MP, H1 = 2 * MP, H0 = 3 * MP;
    static constexpr int WE = TZ + 2 * H0;            // E row length (floats)
    static constexpr int WB = TZ + 2 * H1;            // B row length
    static constexpr int WJ = TZ + 2 * H2;            // J row length
    static constexpr int TYe = NDIM == 3 ? TY : 1;
    static constexpr int RX0 = TX + 3, RY0 = NDIM == 3 ? TY + 3 : 1;   // E rows: [-1, T+1]
    static constexpr int RX1 = TX + 2, RY1 = NDIM == 3 ? TY + 2 : 1;   // B rows: [-1, T]
    static constexpr int RX2 = TX + 1, RY2 = NDIM == 3 ? TY + 1 : 1;   // E', J rows: [0, T]
    static constexpr int SE = RX0 * RY0 * WE;
    static constexpr int SB = RX1 * RY1 * WB;
    static constexpr int SJ = RX2 * RY2 * WJ;
    static constexpr size_t smem_bytes = sizeof(float) * 3 * (SE + SB + SJ);
    static_assert(TZ % 4 == 0, "the z tile holds whole groups of four cells");
};

__device__ __forceinline__ void lds4(float (&a)[4], const float* s) {
    const float4 v = *reinterpret_cast<const float4*>(s);
    a[0] = v.x;
    a[1] = v.y;
    a[2] = v.z;
    a[3] = v.w;
}

__device__ __forceinline__ void sts4(float* s, const float (&a)[4]) {
    *reinterpret_cast<float4*>(s) = make_float4(a[0], a[1], a[2], a[3]);
}

// 16-byte asynchronous global -> shared copy; valid == false writes zeros (nothing is read,
// src must still be a mapped address).
__device__ __forceinline__ void cp_async16(float* dst, const float* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const int n = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}
// 4-byte copy with zero fill (valid = false reads nothing): rows that are not 16-byte aligned
__device__ __forceinline__ void cp_async4z(float* dst, const float* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const int n = valid ? 4 : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_all;\n" ::: "memory");
}

// Rows of a staged field: `rows` rows of `w` floats (w % 4 == 0) covering z in [zlo, zlo + w)
// of global rows (x0 + rx + dxy, y0 + ry + dxy) (periodic in x, y), components f0, f1, f2
// into dst[c * cstride + r * w + col]; zero outside 0 <= z < nz.
template <int NDIM, int RX>
__device__ __forceinline__ void stage_rows(float* dst, int cstride, const float* __restrict__ f0,
                                           const float* __restrict__ f1, const float* __restrict__ f2, int rows,
                                           int w, int zlo, int x0, int y0, int dxy, const GridP& g, bool vec) {
    const float* f[3] = {f0, f1, f2};
    const int ng = w >> 2;
    for (int it = threadIdx.x; it < rows * ng; it += blockDim.x) {
        const int gi = it % ng, r = it / ng;
        const int rx = r % RX, ry = r / RX;
        const int gz = zlo + 4 * gi;
        const int gx = wrapi(x0 + rx + dxy, g.nx);
        const int gy = NDIM == 3 ? wrapi(y0 + ry + dxy, g.ny) : 0;
        const long long row = ((long long)gy * g.nx + gx) * g.nz;
        float* d = dst + r * w + 4 * gi;
        if (vec) {
            const bool in = gz >= 0 && gz < g.nz;
            const long long o = in ? row + gz : 0;
#pragma unroll
            for (int c = 0; c < 3; ++c) cp_async16(d + c * cstride, f[c] + o, in);
        } else {
            // rows not 16-byte aligned: element copies, asynchronous as well
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const bool in = gz + j >= 0 && gz + j < g.nz;
                    cp_async4z(d + c * cstride + j, f[c] + (in ? row + gz + j : 0), in);
                }
        }
    }
}

// w[k] = f[z - MP + k], k < 2 MP + 4, from the aligned window at s.
//   d+ (E -> B, Appendix C):  d[j] = sum_l C_l (f[z+j+l] - f[z+j-l+1]),  l = 1..M  (E-side C)
//   d- (B -> E):              d[j] = sum_l C_l (f[z+j+l-1] - f[z+j-l])          (B-side Cm)
// mid[j] = f[z+j].  Coefficients beyond M are zero.
template <int MAXM, int MP, bool PLUS>
__device__ __forceinline__ void window_dz(const StencilP& st, const float* s, float (&d)[4], float (&mid)[4]) {
    constexpr int NW = 2 * MP + 4;
    float w[NW];
#pragma unroll
    for (int q = 0; q < NW / 4; ++q) {
        float a[4];
        lds4(a, s + 4 * q);
        w[4 * q] = a[0];
        w[4 * q + 1] = a[1];
        w[4 * q + 2] = a[2];
        w[4 * q + 3] = a[3];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float acc = 0.f;
#pragma unroll
        for (int l = 1; l <= MAXM; ++l) {
            const float df = PLUS ? w[MP + j + l] - w[MP + j - l + 1] : w[MP + j + l - 1] - w[MP + j - l];
            acc = fmaf(PLUS ? st.C[l - 1] : st.Cm[l - 1], df, acc);
        }
        d[j] = acc;
        mid[j] = w[MP + j];
    }
}

template <int NDIM, int MAXM, int TZ, int TX, int TY>
__device__ __forceinline__ void advance_tile_rb(const FieldP& p, int tz, int tx, int ty, float* smem) {
    using T = TileRB<NDIM, MAXM, TZ, TX, TY>;
    constexpr int MP = T::MP, WE = T::WE, WB = T::WB, WJ = T::WJ;
    float* sE = smem;                             // [3][RY0][RX0][WE]
    float* sB = smem + 3 * T::SE;                 // [3][RY1][RX1][WB]
    float* sJ = smem + 3 * (T::SE + T::SB);       // [3][RY2][RX2][WJ]

    const GridP& g = p.g;
    const int nz = g.nz, nx = g.nx, ny = g.ny;
    const long long N = g.ncell;
    const int z0 = tz * TZ, x0 = tx * TX, y0 = NDIM == 3 ? ty * TY : 0;
    const bool vec = p.vec4 != 0;
    const float dt = g.dt;
    const float hz = 0.5f * dt / g.dz, fz = dt / g.dz;
    const float hx = 0.5f * dt / g.dx, fx = dt / g.dx;
    const float hy = NDIM == 3 ? 0.5f * dt / g.dy : 0.f, fy = NDIM == 3 ? dt / g.dy : 0.f;

    // ---- stage 0: E^n (rows from -1), B^n (rows from -1), J (rows from 0) ------------------
    stage_rows<NDIM, T::RX0>(sE, T::SE, p.Ein, p.Ein + N, p.Ein + 2 * N, T::RY0 * T::RX0, WE, z0 - T::H0, x0, y0,
                             -1, g, vec);
    stage_rows<NDIM, T::RX1>(sB, T::SB, p.Bin, p.Bin + N, p.Bin + 2 * N, T::RY1 * T::RX1, WB, z0 - T::H1, x0, y0,
                             -1, g, vec);
    stage_rows<NDIM, T::RX2>(sJ, T::SJ, p.J1, p.J2, p.J3, T::RY2 * T::RX2, WJ, z0 - T::H2, x0, y0, 0, g, vec);
    cp_async_wait_all();
    __syncthreads();

    // ---- stage 1: B^{n+1/2} in place, rows x in [-1, TX] (y in [-1, TY]), z in [-H1, TZ+H1) --
    constexpr int NG1 = WB / 4;
    for (int it = threadIdx.x; it < T::RY1 * T::RX1 * NG1; it += blockDim.x) {
        const int gi = it % NG1, r = it / NG1;
        const int rx = r % T::RX1, ry = r / T::RX1;
        const int z = 4 * gi - T::H1;
        const int gz = z0 + z;
        if (gz + 3 < 0 || gz >= nz) continue;                       // B^n = B^{n+1/2} = 0 there
        const int e = (ry * T::RX0 + rx) * WE + z + T::H0;          // E rows also start at -1
        float d2[4], d3[4], e2[4], e3[4], e1[4], e1x[4], e3x[4];
        float e1y[4] = {0.f, 0.f, 0.f, 0.f}, e2y[4] = {0.f, 0.f, 0.f, 0.f};
        window_dz<MAXM, MP, true>(p.st, sE + T::SE + e - MP, d2, e2);
        window_dz<MAXM, MP, true>(p.st, sE + 2 * T::SE + e - MP, d3, e3);
        lds4(e1, sE + e);
        lds4(e1x, sE + e + WE);
        lds4(e3x, sE + 2 * T::SE + e + WE);
        if (NDIM == 3) {
            lds4(e1y, sE + e + T::RX0 * WE);
            lds4(e2y, sE + T::SE + e + T::RX0 * WE);
        }
        const int cb = r * WB + 4 * gi;
        float b0[4], b1[4], b2[4];
        lds4(b0, sB + cb);
        lds4(b1, sB + T::SB + cb);
        lds4(b2, sB + 2 * T::SB + cb);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool in = gz + j >= 0 && gz + j < nz;
            b0[j] = in ? b0[j] - (hx * (e3x[j] - e3[j]) - hy * (e2y[j] - e2[j])) : 0.f;
            b1[j] = in ? b1[j] - (hy * (e1y[j] - e1[j]) - hz * d3[j]) : 0.f;
            b2[j] = in ? b2[j] - (hz * d2[j] - hx * (e1x[j] - e1[j])) : 0.f;
        }
        sts4(sB + cb, b0);
        sts4(sB + T::SB + cb, b1);
        sts4(sB + 2 * T::SB + cb, b2);
    }
    __syncthreads();

    // ---- stage 2: E^{n+1} in place, rows x in [0, TX] (y in [0, TY]), z in [-H2, TZ+H2) ------
    constexpr int NG2 = WJ / 4;
    for (int it = threadIdx.x; it < T::RY2 * T::RX2 * NG2; it += blockDim.x) {
        const int gi = it % NG2, r = it / NG2;
        const int rx = r % T::RX2, ry = r / T::RX2;
        const int z = 4 * gi - T::H2;
        const int gz = z0 + z;
        if (gz + 3 < 0 || gz >= nz) continue;                       // E^n = E^{n+1} = 0 there
        const int e = ((NDIM == 3 ? (ry + 1) * T::RX0 : 0) + rx + 1) * WE + z + T::H0;
        const int b = ((NDIM == 3 ? (ry + 1) * T::RX1 : 0) + rx + 1) * WB + z + T::H1;
        float d2[4], d3[4], B2[4], B3[4], B1[4], B1x[4], B3x[4];
        float B1y[4] = {0.f, 0.f, 0.f, 0.f}, B2y[4] = {0.f, 0.f, 0.f, 0.f};
        window_dz<MAXM, MP, false>(p.st, sB + T::SB + b - MP, d2, B2);
        window_dz<MAXM, MP, false>(p.st, sB + 2 * T::SB + b - MP, d3, B3);
        lds4(B1, sB + b);
        lds4(B1x, sB + b - WB);
        lds4(B3x, sB + 2 * T::SB + b - WB);
        if (NDIM == 3) {
            lds4(B1y, sB + b - T::RX1 * WB);
            lds4(B2y, sB + T::SB + b - T::RX1 * WB);
        }
        const int cj = r * WJ + 4 * gi;
        float e0[4], e1[4], e2[4], j0[4], j1[4], j2[4];
        lds4(e0, sE + e);
        lds4(e1, sE + T::SE + e);
        lds4(e2, sE + 2 * T::SE + e);
        lds4(j0, sJ + cj);
        lds4(j1, sJ + T::SJ + cj);
        lds4(j2, sJ + 2 * T::SJ + cj);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool in = gz + j >= 0 && gz + j < nz;
            e0[j] = in ? e0[j] + (fx * (B3[j] - B3x[j]) - fy * (B2[j] - B2y[j])) - dt * j0[j] : 0.f;
            e1[j] = in ? e1[j] + (fy * (B1[j] - B1y[j]) - fz * d3[j]) - dt * j1[j] : 0.f;
            e2[j] = in ? e2[j] + (fz * d2[j] - fx * (B1[j] - B1x[j])) - dt * j2[j] : 0.f;
        }
        sts4(sE + e, e0);
        sts4(sE + T::SE + e, e1);
        sts4(sE + 2 * T::SE + e, e2);
    }
    __syncthreads();

    // ---- stage 3: B^{n+1} on the tile; store E^{n+1}, B^{n+1} (shifted if the window moves) --
    constexpr int NG3 = TZ / 4;
    for (int it = threadIdx.x; it < T::TYe * TX * NG3; it += blockDim.x) {
        const int gi = it % NG3, r = it / NG3;
        const int x = r % TX, y = r / TX;
        const int z = 4 * gi;
        const int gz = z0 + z, gx = x0 + x, gy = y0 + y;
        if (gz >= nz || gx >= nx || (NDIM == 3 && gy >= ny)) continue;
        const int e = ((NDIM == 3 ? (y + 1) * T::RX0 : 0) + x + 1) * WE + z + T::H0;
        const int b = ((NDIM == 3 ? (y + 1) * T::RX1 : 0) + x + 1) * WB + z + T::H1;
        float d2[4], d3[4], e2[4], e3[4], e1[4], e1x[4], e3x[4];
        float e1y[4] = {0.f, 0.f, 0.f, 0.f}, e2y[4] = {0.f, 0.f, 0.f, 0.f};
        window_dz<MAXM, MP, true>(p.st, sE + T::SE + e - MP, d2, e2);
        window_dz<MAXM, MP, true>(p.st, sE + 2 * T::SE + e - MP, d3, e3);
        lds4(e1, sE + e);
        lds4(e1x, sE + e + WE);
        lds4(e3x, sE + 2 * T::SE + e + WE);
        if (NDIM == 3) {
            lds4(e1y, sE + e + T::RX0 * WE);
            lds4(e2y, sE + T::SE + e + T::RX0 * WE);
        }
        float b0[4], b1[4], b2[4];
        lds4(b0, sB + b);
        lds4(b1, sB + T::SB + b);
        lds4(b2, sB + 2 * T::SB + b);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            b0[j] -= hx * (e3x[j] - e3[j]) - hy * (e2y[j] - e2[j]);
            b1[j] -= hy * (e1y[j] - e1[j]) - hz * d3[j];
            b2[j] -= hz * d2[j] - hx * (e1x[j] - e1[j]);
        }
        const long long row = ((long long)gy * nx + gx) * nz;
        if (vec && !p.shift) {
            const long long o = row + gz;
            *reinterpret_cast<float4*>(p.Eout + o) = make_float4(e1[0], e1[1], e1[2], e1[3]);
            *reinterpret_cast<float4*>(p.Eout + N + o) = make_float4(e2[0], e2[1], e2[2], e2[3]);
            *reinterpret_cast<float4*>(p.Eout + 2 * N + o) = make_float4(e3[0], e3[1], e3[2], e3[3]);
            *reinterpret_cast<float4*>(p.Bout + o) = make_float4(b0[0], b0[1], b0[2], b0[3]);
            *reinterpret_cast<float4*>(p.Bout + N + o) = make_float4(b1[0], b1[1], b1[2], b1[3]);
            *reinterpret_cast<float4*>(p.Bout + 2 * N + o) = make_float4(b2[0], b2[1], b2[2], b2[3]);
            continue;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gzj = gz + j;
            if (gzj >= nz) break;
            const int oz = gzj - p.shift;
            if (oz >= 0) {
                const long long o = row + oz;
                p.Eout[o] = e1[j];
                p.Eout[N + o] = e2[j];
                p.Eout[2 * N + o] = e3[j];
                p.Bout[o] = b0[j];
                p.Bout[N + o] = b1[j];
                p.Bout[2 * N + o] = b2[j];
            }
            if (p.shift && gzj == nz - 1) {
                const long long o = row + gzj;
                p.Eout[o] = 0.f;
                p.Eout[N + o] = 0.f;
                p.Eout[2 * N + o] = 0.f;
                p.Bout[o] = 0.f;
                p.Bout[N + o] = 0.f;
                p.Bout[2 * N + o] = 0.f;
            }
        }
    }
}

template <int NDIM, int MAXM, int TZ, int TX, int TY>
__global__ void __launch_bounds__(256, 2) field_advance_rb_kernel(FieldP p) {
    extern __shared__ float4 smem4[];
    advance_tile_rb<NDIM, MAXM, TZ, TX, TY>(p, blockIdx.x, blockIdx.y, blockIdx.z, reinterpret_cast<float*>(smem4));
}


// ---- 3D y-marching tile -----------------------------------------------------------------
// A CTA owns a TZ x TX column of x-z planes and walks y over [ya, ya + yc), keeping three E
// planes, two B planes and one J plane in shared memory, register-blocked along z as above.
// For output plane k it stages E^n(k+2), B^n(k+1), J(k+1), then computes
//   B^{n+1/2}(k+1) from E^n(k+1), E^n(k+2);
//   E^{n+1}(k+1)   from B^{n+1/2}(k+1), B^{n+1/2}(k) (in place over E^n(k+1));
//   B^{n+1}(k)     from E^{n+1}(k), E^{n+1}(k+1), B^{n+1/2}(k), and stores E^{n+1}(k), B^{n+1}(k).
// Every plane is read once per CTA plus its x halo, where a tile blocked in x and y re-reads
// and recomputes a (T+3)^2 / T^2 halo.
template <int MAXM, int TZ, int TX>
struct MarchT {
    static constexpr int MP = (MAXM + 3) & ~3;
    static constexpr int H2 = MP, H1 = 2 * MP, H0 = 3 * MP;
    static constexpr int WE = TZ + 2 * H0, WB = TZ + 2 * H1, WJ = TZ + 2 * H2;
    static constexpr int RX0 = TX + 3, RX1 = TX + 2, RX2 = TX + 1;    // E rows [-1, TX+1], B [-1, TX], J [0, TX]
    static constexpr int PE = RX0 * WE, PB = RX1 * WB, PJ = RX2 * WJ;  // one component of one plane
    static constexpr size_t smem_bytes = sizeof(float) * 3 * (3 * PE + 2 * PB + PJ);
    static_assert(TZ % 4 == 0, "the z tile holds whole groups of four cells");
};

// One x-z plane (global y = gy) of components f0..f2: `rows` rows starting at x0 + dx, z in
// [zlo, zlo + w), into dst[c * cstride + r * w + col]; zero outside 0 <= z < nz.
__device__ __forceinline__ void stage_plane(float* dst, int cstride, const float* __restrict__ f0,
                                            const float* __restrict__ f1, const float* __restrict__ f2, int rows,
                                            int w, int zlo, int x0, int dx, int gy, const GridP& g, bool vec) {
    const float* f[3] = {f0, f1, f2};
    const int ng = w >> 2;
    for (int it = threadIdx.x; it < rows * ng; it += blockDim.x) {
        const int gi = it % ng, r = it / ng;
        const int gz = zlo + 4 * gi;
        const long long row = ((long long)gy * g.nx + wrapi(x0 + r + dx, g.nx)) * g.nz;
        float* d = dst + r * w + 4 * gi;
        if (vec) {
            const bool in = gz >= 0 && gz < g.nz;
            const long long o = in ? row + gz : 0;
#pragma unroll
            for (int c = 0; c < 3; ++c) cp_async16(d + c * cstride, f[c] + o, in);
        } else {
            // rows not 16-byte aligned: element copies, asynchronous as well
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const bool in = gz + j >= 0 && gz + j < g.nz;
                    cp_async4z(d + c * cstride + j, f[c] + (in ? row + gz + j : 0), in);
                }
        }
    }
}

// B^{n+1/2} in place over B^n plane b (rows x in [-1, TX]) from E^n planes e (y) and e1 (y+1).
template <int MAXM, int TZ, int TX>
__device__ __forceinline__ void march_bhalf(const FieldP& p, float* b, const float* e, const float* e1, int z0) {
    using T = MarchT<MAXM, TZ, TX>;
    constexpr int MP = T::MP, WE = T::WE, WB = T::WB, PE = T::PE, PB = T::PB, NG = WB / 4;
    const GridP& g = p.g;
    const float hz = 0.5f * g.dt / g.dz, hx = 0.5f * g.dt / g.dx, hy = 0.5f * g.dt / g.dy;
    for (int it = threadIdx.x; it < T::RX1 * NG; it += blockDim.x) {
        const int gi = it % NG, rx = it / NG;
        const int z = 4 * gi - T::H1, gz = z0 + z;
        if (gz + 3 < 0 || gz >= g.nz) continue;                     // B^n = B^{n+1/2} = 0 there
        const int eo = rx * WE + z + T::H0;
        float d2[4], d3[4], E2[4], E3[4], E1[4], E1x[4], E3x[4], E1y[4], E2y[4];
        window_dz<MAXM, MP, true>(p.st, e + PE + eo - MP, d2, E2);
        window_dz<MAXM, MP, true>(p.st, e + 2 * PE + eo - MP, d3, E3);
        lds4(E1, e + eo);
        lds4(E1x, e + eo + WE);
        lds4(E3x, e + 2 * PE + eo + WE);
        lds4(E1y, e1 + eo);
        lds4(E2y, e1 + PE + eo);
        const int bo = rx * WB + 4 * gi;
        float b0[4], b1[4], b2[4];
        lds4(b0, b + bo);
        lds4(b1, b + PB + bo);
        lds4(b2, b + 2 * PB + bo);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool in = gz + j >= 0 && gz + j < g.nz;
            b0[j] = in ? b0[j] - (hx * (E3x[j] - E3[j]) - hy * (E2y[j] - E2[j])) : 0.f;
            b1[j] = in ? b1[j] - (hy * (E1y[j] - E1[j]) - hz * d3[j]) : 0.f;
            b2[j] = in ? b2[j] - (hz * d2[j] - hx * (E1x[j] - E1[j])) : 0.f;
        }
        sts4(b + bo, b0);
        sts4(b + PB + bo, b1);
        sts4(b + 2 * PB + bo, b2);
    }
}

// E^{n+1} in place over E^n plane e (rows x in [0, TX]) from B^{n+1/2} planes b (y), bm (y-1)
// and the J plane j.
template <int MAXM, int TZ, int TX>
__device__ __forceinline__ void march_enew(const FieldP& p, float* e, const float* b, const float* bm,
                                           const float* j, int z0) {
    using T = MarchT<MAXM, TZ, TX>;
    constexpr int MP = T::MP, WE = T::WE, WB = T::WB, WJ = T::WJ, PE = T::PE, PB = T::PB, PJ = T::PJ;
    constexpr int NG = WJ / 4;
    const GridP& g = p.g;
    const float dt = g.dt, fz = dt / g.dz, fx = dt / g.dx, fy = dt / g.dy;
    for (int it = threadIdx.x; it < T::RX2 * NG; it += blockDim.x) {
        const int gi = it % NG, rx = it / NG;
        const int z = 4 * gi - T::H2, gz = z0 + z;
        if (gz + 3 < 0 || gz >= g.nz) continue;                     // E^n = E^{n+1} = 0 there
        const int eo = (rx + 1) * WE + z + T::H0;
        const int bo = (rx + 1) * WB + z + T::H1;
        float d2[4], d3[4], B2[4], B3[4], B1[4], B1x[4], B3x[4], B1y[4], B2y[4];
        window_dz<MAXM, MP, false>(p.st, b + PB + bo - MP, d2, B2);
        window_dz<MAXM, MP, false>(p.st, b + 2 * PB + bo - MP, d3, B3);
        lds4(B1, b + bo);
        lds4(B1x, b + bo - WB);
        lds4(B3x, b + 2 * PB + bo - WB);
        lds4(B1y, bm + bo);
        lds4(B2y, bm + PB + bo);
        const int jo = rx * WJ + 4 * gi;
        float e0[4], e1[4], e2[4], j0[4], j1[4], j2[4];
        lds4(e0, e + eo);
        lds4(e1, e + PE + eo);
        lds4(e2, e + 2 * PE + eo);
        lds4(j0, j + jo);
        lds4(j1, j + PJ + jo);
        lds4(j2, j + 2 * PJ + jo);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const bool in = gz + q >= 0 && gz + q < g.nz;
            e0[q] = in ? e0[q] + (fx * (B3[q] - B3x[q]) - fy * (B2[q] - B2y[q])) - dt * j0[q] : 0.f;
            e1[q] = in ? e1[q] + (fy * (B1[q] - B1y[q]) - fz * d3[q]) - dt * j1[q] : 0.f;
            e2[q] = in ? e2[q] + (fz * d2[q] - fx * (B1[q] - B1x[q])) - dt * j2[q] : 0.f;
        }
        sts4(e + eo, e0);
        sts4(e + PE + eo, e1);
        sts4(e + 2 * PE + eo, e2);
    }
}

// B^{n+1} on the tile rows (x in [0, TX)) of plane gy from E^{n+1} planes e (y), e1 (y+1) and
// B^{n+1/2} plane b; stores E^{n+1}(y) and B^{n+1}(y) (one cell towards -z if the window moves).
template <int MAXM, int TZ, int TX>
__device__ __forceinline__ void march_bnew_store(const FieldP& p, const float* e, const float* e1, const float* b,
                                                 int z0, int x0, int gy, bool vec) {
    using T = MarchT<MAXM, TZ, TX>;
    constexpr int MP = T::MP, WE = T::WE, WB = T::WB, PE = T::PE, PB = T::PB, NG = TZ / 4;
    const GridP& g = p.g;
    const long long N = g.ncell;
    const float hz = 0.5f * g.dt / g.dz, hx = 0.5f * g.dt / g.dx, hy = 0.5f * g.dt / g.dy;
    // shifted 16-byte stores take the next group's first cell from the next lane: the rows of the
    // tile are whole runs of lanes and every warp runs the loop the same number of times
    static_assert(32 % NG == 0 && (TX * NG) % 32 == 0, "tile rows aligned to warps");
    const bool vshift = vec && p.shift;
    for (int it = threadIdx.x; it < TX * NG; it += blockDim.x) {
        const int gi = it % NG, x = it / NG;
        const int z = 4 * gi, gz = z0 + z, gx = x0 + x;
        const bool valid = gz < g.nz && gx < g.nx;
        if (!valid && !vshift) continue;   // (the shifted path computes on every lane: the planes hold
                                           // the whole tile, so the shared reads stay inside them)
        const int eo = (x + 1) * WE + z + T::H0;
        const int bo = (x + 1) * WB + z + T::H1;
        float d2[4], d3[4], E2[4], E3[4], E1[4], E1x[4], E3x[4], E1y[4], E2y[4];
        window_dz<MAXM, MP, true>(p.st, e + PE + eo - MP, d2, E2);
        window_dz<MAXM, MP, true>(p.st, e + 2 * PE + eo - MP, d3, E3);
        lds4(E1, e + eo);
        lds4(E1x, e + eo + WE);
        lds4(E3x, e + 2 * PE + eo + WE);
        lds4(E1y, e1 + eo);
        lds4(E2y, e1 + PE + eo);
        float b0[4], b1[4], b2[4];
        lds4(b0, b + bo);
        lds4(b1, b + PB + bo);
        lds4(b2, b + 2 * PB + bo);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            b0[q] -= hx * (E3x[q] - E3[q]) - hy * (E2y[q] - E2[q]);
            b1[q] -= hy * (E1y[q] - E1[q]) - hz * d3[q];
            b2[q] -= hz * d2[q] - hx * (E1x[q] - E1[q]);
        }
        const long long row = ((long long)gy * g.nx + gx) * g.nz;
        if (vec && !p.shift) {
            const long long o = row + gz;
            *reinterpret_cast<float4*>(p.Eout + o) = make_float4(E1[0], E1[1], E1[2], E1[3]);
            *reinterpret_cast<float4*>(p.Eout + N + o) = make_float4(E2[0], E2[1], E2[2], E2[3]);
            *reinterpret_cast<float4*>(p.Eout + 2 * N + o) = make_float4(E3[0], E3[1], E3[2], E3[3]);
            *reinterpret_cast<float4*>(p.Bout + o) = make_float4(b0[0], b0[1], b0[2], b0[3]);
            *reinterpret_cast<float4*>(p.Bout + N + o) = make_float4(b1[0], b1[1], b1[2], b1[3]);
            *reinterpret_cast<float4*>(p.Bout + 2 * N + o) = make_float4(b2[0], b2[1], b2[2], b2[3]);
            continue;
        }
        if (vshift) {
            // window shift, nz % 4 == 0: output group [gz, gz + 4) takes cells gz + 1 .. gz + 4.  Cell
            // gz + 4 is the next lane's first cell; at the front (gz + 4 == nz) it is the zeroed
            // front column; for the last group of a tile row it belongs to the next tile, whose first
            // lane stores it one cell down (this group's last output), so this lane stores three.
            const unsigned full = 0xffffffffu;
            float nx6[6] = {E1[0], E2[0], E3[0], b0[0], b1[0], b2[0]};
#pragma unroll
            for (int c = 0; c < 6; ++c) nx6[c] = __shfl_down_sync(full, nx6[c], 1);
            if (!valid) continue;
            float* dst[6] = {p.Eout + row, p.Eout + N + row, p.Eout + 2 * N + row,
                             p.Bout + row, p.Bout + N + row, p.Bout + 2 * N + row};
            const float* src[6] = {E1, E2, E3, b0, b1, b2};
            const bool front = gz + 4 >= g.nz;
            if (front || gi != NG - 1) {
#pragma unroll
                for (int c = 0; c < 6; ++c)
                    *reinterpret_cast<float4*>(dst[c] + gz) =
                        make_float4(src[c][1], src[c][2], src[c][3], front ? 0.f : nx6[c]);
            } else {
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    dst[c][gz] = src[c][1];
                    dst[c][gz + 1] = src[c][2];
                    dst[c][gz + 2] = src[c][3];
                }
            }
            if (gi == 0 && gz > 0) {
#pragma unroll
                for (int c = 0; c < 6; ++c) dst[c][gz - 1] = src[c][0];
            }
            continue;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int gzq = gz + q;
            if (gzq >= g.nz) break;
            const int oz = gzq - p.shift;
            if (oz >= 0) {
                const long long o = row + oz;
                p.Eout[o] = E1[q];
                p.Eout[N + o] = E2[q];
                p.Eout[2 * N + o] = E3[q];
                p.Bout[o] = b0[q];
                p.Bout[N + o] = b1[q];
                p.Bout[2 * N + o] = b2[q];
            }
            if (p.shift && gzq == g.nz - 1) {
                const long long o = row + gzq;
                p.Eout[o] = 0.f;
                p.Eout[N + o] = 0.f;
                p.Eout[2 * N + o] = 0.f;
                p.Bout[o] = 0.f;
                p.Bout[N + o] = 0.f;
                p.Bout[2 * N + o] = 0.f;
            }
        }
    }
}

// ---- 2D x-marching rows -------------------------------------------------------------------
// A CTA owns z in [z0, z0 + TZ) and walks x over [xa, xa + xc): every row of B^{n+1/2} and
// E^{n+1} is computed once (no x halo), register-blocked along z as above.  The rows a step
// needs next are copied by cp.async one step ahead into a ring of 4 E, 3 B and 2 J rows:
// for output row k the step computes B^{n+1/2}(k+1) from E^n(k+1), E^n(k+2); E^{n+1}(k+1) from
// B^{n+1/2}(k+1), B^{n+1/2}(k), J(k+1); B^{n+1}(k) from E^{n+1}(k), E^{n+1}(k+1), B^{n+1/2}(k),
// while E^n(k+3), B^n(k+2), J(k+2) land.
template <int MAXM, int TZ>
struct March2T {
    static constexpr int MP = (MAXM + 3) & ~3;
    static constexpr int H2 = MP, H1 = 2 * MP, H0 = 3 * MP;
    static constexpr int WE = TZ + 2 * H0, WB = TZ + 2 * H1, WJ = TZ + 2 * H2;
    static constexpr int SE = 3 * WE, SB = 3 * WB, SJ = 3 * WJ;           // one row, 3 components
    static constexpr size_t smem_bytes = sizeof(float) * (4 * SE + 3 * SB + 2 * SJ);
    static_assert(TZ % 4 == 0, "the z tile holds whole groups of four cells");
};

// B^{n+1/2} in place over the B^n row b from the E^n rows e (x) and e1 (x + 1).
template <int MAXM, int TZ>
__device__ __forceinline__ void march2_bhalf(const FieldP& p, float* b, const float* e, const float* e1, int z0) {
    using T = March2T<MAXM, TZ>;
    constexpr int MP = T::MP, WE = T::WE, WB = T::WB, NG = WB / 4;
    const GridP& g = p.g;
    const float hz = 0.5f * g.dt / g.dz, hx = 0.5f * g.dt / g.dx;
    for (int gi = threadIdx.x; gi < NG; gi += blockDim.x) {
        const int z = 4 * gi - T::H1, gz = z0 + z;
        if (gz + 3 < 0 || gz >= g.nz) continue;                     // B^n = B^{n+1/2} = 0 there
        const int eo = z + T::H0;
        float d2[4], d3[4], E2[4], E3[4], E1[4], E1x[4], E3x[4];
        window_dz<MAXM, MP, true>(p.st, e + WE + eo - MP, d2, E2);
        window_dz<MAXM, MP, true>(p.st, e + 2 * WE + eo - MP, d3, E3);
        lds4(E1, e + eo);
        lds4(E1x, e1 + eo);
        lds4(E3x, e1 + 2 * WE + eo);
        const int bo = 4 * gi;
        float b0[4], b1[4], b2[4];
        lds4(b0, b + bo);
        lds4(b1, b + WB + bo);
        lds4(b2, b + 2 * WB + bo);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool in = gz + j >= 0 && gz + j < g.nz;
            b0[j] = in ? b0[j] - hx * (E3x[j] - E3[j]) : 0.f;
            b1[j] = in ? b1[j] + hz * d3[j] : 0.f;
            b2[j] = in ? b2[j] - (hz * d2[j] - hx * (E1x[j] - E1[j])) : 0.f;
        }
        sts4(b + bo, b0);
        sts4(b + WB + bo, b1);
        sts4(b + 2 * WB + bo, b2);
    }
}

// E^{n+1} in place over the E^n row e from the B^{n+1/2} rows b (x), bm (x - 1) and the J row j.
template <int MAXM, int TZ>
__device__ __forceinline__ void march2_enew(const FieldP& p, float* e, const float* b, const float* bm, const float* j,
                                            int z0) {
    using T = March2T<MAXM, TZ>;
    constexpr int MP = T::MP, WE = T::WE, WB = T::WB, WJ = T::WJ, NG = WJ / 4;
    const GridP& g = p.g;
    const float dt = g.dt, fz = dt / g.dz, fx = dt / g.dx;
    for (int gi = threadIdx.x; gi < NG; gi += blockDim.x) {
        const int z = 4 * gi - T::H2, gz = z0 + z;
        if (gz + 3 < 0 || gz >= g.nz) continue;                     // E^n = E^{n+1} = 0 there
        const int eo = z + T::H0, bo = z + T::H1;
        float d2[4], d3[4], B2[4], B3[4], B1[4], B1x[4], B3x[4];
        window_dz<MAXM, MP, false>(p.st, b + WB + bo - MP, d2, B2);
        window_dz<MAXM, MP, false>(p.st, b + 2 * WB + bo - MP, d3, B3);
        lds4(B1, b + bo);
        lds4(B1x, bm + bo);
        lds4(B3x, bm + 2 * WB + bo);
        const int jo = 4 * gi;
        float e0[4], e1[4], e2[4], j0[4], j1[4], j2[4];
        lds4(e0, e + eo);
        lds4(e1, e + WE + eo);
        lds4(e2, e + 2 * WE + eo);
        lds4(j0, j + jo);
        lds4(j1, j + WJ + jo);
        lds4(j2, j + 2 * WJ + jo);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const bool in = gz + q >= 0 && gz + q < g.nz;
            e0[q] = in ? e0[q] + fx * (B3[q] - B3x[q]) - dt * j0[q] : 0.f;
            e1[q] = in ? e1[q] - fz * d3[q] - dt * j1[q] : 0.f;
            e2[q] = in ? e2[q] + (fz * d2[q] - fx * (B1[q] - B1x[q])) - dt * j2[q] : 0.f;
        }
        sts4(e + eo, e0);
        sts4(e + WE + eo, e1);
        sts4(e + 2 * WE + eo, e2);
    }
}

// B^{n+1} of row gx from the E^{n+1} rows e (x), e1 (x + 1) and the B^{n+1/2} row b; stores
// E^{n+1}(x), B^{n+1}(x) (one cell towards -z if the window moves).
template <int MAXM, int TZ>
__device__ __forceinline__ void march2_bnew_store(const FieldP& p, const float* e, const float* e1, const float* b,
                                                  int z0, int gx, bool vec) {
    using T = March2T<MAXM, TZ>;
    constexpr int MP = T::MP, WE = T::WE, WB = T::WB, NG = TZ / 4;
    const GridP& g = p.g;
    const long long N = g.ncell;
    const float hz = 0.5f * g.dt / g.dz, hx = 0.5f * g.dt / g.dx;
    const long long row = (long long)gx * g.nz;
    for (int gi = threadIdx.x; gi < NG; gi += blockDim.x) {
        const int z = 4 * gi, gz = z0 + z;
        if (gz >= g.nz) continue;
        const int eo = z + T::H0, bo = z + T::H1;
        float d2[4], d3[4], E2[4], E3[4], E1[4], E1x[4], E3x[4];
        window_dz<MAXM, MP, true>(p.st, e + WE + eo - MP, d2, E2);
        window_dz<MAXM, MP, true>(p.st, e + 2 * WE + eo - MP, d3, E3);
        lds4(E1, e + eo);
        lds4(E1x, e1 + eo);
        lds4(E3x, e1 + 2 * WE + eo);
        float b0[4], b1[4], b2[4];
        lds4(b0, b + bo);
        lds4(b1, b + WB + bo);
        lds4(b2, b + 2 * WB + bo);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            b0[q] -= hx * (E3x[q] - E3[q]);
            b1[q] += hz * d3[q];
            b2[q] -= hz * d2[q] - hx * (E1x[q] - E1[q]);
        }
        if (vec && !p.shift) {
            const long long o = row + gz;
            *reinterpret_cast<float4*>(p.Eout + o) = make_float4(E1[0], E1[1], E1[2], E1[3]);
            *reinterpret_cast<float4*>(p.Eout + N + o) = make_float4(E2[0], E2[1], E2[2], E2[3]);
            *reinterpret_cast<float4*>(p.Eout + 2 * N + o) = make_float4(E3[0], E3[1], E3[2], E3[3]);
            *reinterpret_cast<float4*>(p.Bout + o) = make_float4(b0[0], b0[1], b0[2], b0[3]);
            *reinterpret_cast<float4*>(p.Bout + N + o) = make_float4(b1[0], b1[1], b1[2], b1[3]);
            *reinterpret_cast<float4*>(p.Bout + 2 * N + o) = make_float4(b2[0], b2[1], b2[2], b2[3]);
            continue;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int gzq = gz + q;
            if (gzq >= g.nz) break;
            const int oz = gzq - p.shift;
            if (oz >= 0) {
                const long long o = row + oz;
                p.Eout[o] = E1[q];
                p.Eout[N + o] = E2[q];
                p.Eout[2 * N + o] = E3[q];
                p.Bout[o] = b0[q];
                p.Bout[N + o] = b1[q];
                p.Bout[2 * N + o] = b2[q];
            }
            if (p.shift && gzq == g.nz - 1) {
                const long long o = row + gzq;
                p.Eout[o] = 0.f;
                p.Eout[N + o] = 0.f;
                p.Eout[2 * N + o] = 0.f;
                p.Bout[o] = 0.f;
                p.Bout[N + o] = 0.f;
                p.Bout[2 * N + o] = 0.f;
            }
        }
    }
}

__device__ __forceinline__ void cp_async_commit_group() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev_group() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// One z segment [z0, z0 + TZ) of rows xa .. xb - 1 (the body of the x-marching kernels).
template <int MAXM, int TZ>
__device__ __forceinline__ void march2_segment(const FieldP& p, int z0, int xa, int xb, float* sm) {
    using T = March2T<MAXM, TZ>;
    const GridP& g = p.g;
    const long long N = g.ncell;
    const bool vec = p.vec4 != 0;
    auto Eslot = [&](int i) { return sm + i * T::SE; };
    auto Bslot = [&](int i) { return sm + 4 * T::SE + i * T::SB; };
    auto Jslot = [&](int i) { return sm + 4 * T::SE + 3 * T::SB + i * T::SJ; };
    auto stageE = [&](int i, int x) {
        stage_plane(Eslot(i), T::WE, p.Ein, p.Ein + N, p.Ein + 2 * N, 1, T::WE, z0 - T::H0, wrapi(x, g.nx), 0, 0, g,
                    vec);
    };
    auto stageB = [&](int i, int x) {
        stage_plane(Bslot(i), T::WB, p.Bin, p.Bin + N, p.Bin + 2 * N, 1, T::WB, z0 - T::H1, wrapi(x, g.nx), 0, 0, g,
                    vec);
    };
    auto stageJ = [&](int i, int x) {
        stage_plane(Jslot(i), T::WJ, p.J1, p.J2, p.J3, 1, T::WJ, z0 - T::H2, wrapi(x, g.nx), 0, 0, g, vec);
    };
    auto landed_all = [&]() {
        cp_async_wait_all();
        __syncthreads();
    };
    // prologue: B^{n+1/2}(xa-1), B^{n+1/2}(xa), E^{n+1}(xa), and the first prefetch
    stageE(0, xa - 1);
    stageE(1, xa);
    stageB(0, xa - 1);
    landed_all();
    march2_bhalf<MAXM, TZ>(p, Bslot(0), Eslot(0), Eslot(1), z0);
    stageE(2, xa + 1);
    stageB(1, xa);
    stageJ(0, xa);
    landed_all();
    march2_bhalf<MAXM, TZ>(p, Bslot(1), Eslot(1), Eslot(2), z0);
    __syncthreads();
    march2_enew<MAXM, TZ>(p, Eslot(1), Bslot(1), Bslot(0), Jslot(0), z0);
    __syncthreads();
    // E: ec = E^{n+1}(k), en = E^n(k+1), ef = E^n(k+2) (in flight), eg = free
    // B: bc = B^{n+1/2}(k), bf = B^n(k+1) (in flight), bg = free;  J: jf = J(k+1) (in flight), jg = free
    int ec = 1, en = 2, ef = 3, eg = 0, bc = 1, bf = 2, bg = 0, jf = 1, jg = 0;
    stageE(ef, xa + 2);
    stageB(bf, xa + 1);
    stageJ(jf, xa + 1);
    cp_async_commit_group();
    for (int k = xa; k < xb; ++k) {
        // the next step's rows, while this step computes
        stageE(eg, k + 3);
        stageB(bg, k + 2);
        stageJ(jg, k + 2);
        {
            cp_async_commit_group();
            cp_async_wait_prev_group();             // this step's rows (committed one step earlier)
        }
        __syncthreads();
        march2_bhalf<MAXM, TZ>(p, Bslot(bf), Eslot(en), Eslot(ef), z0);
        __syncthreads();
        march2_enew<MAXM, TZ>(p, Eslot(en), Bslot(bf), Bslot(bc), Jslot(jf), z0);
        __syncthreads();
        march2_bnew_store<MAXM, TZ>(p, Eslot(ec), Eslot(en), Bslot(bc), z0, k, vec);
        __syncthreads();
        int t = ec;
        ec = en;
        en = ef;
        ef = eg;
        eg = t;
        t = bc;
        bc = bf;
        bf = bg;
        bg = t;
        t = jf;
        jf = jg;
        jg = t;
    }
    cp_async_wait_all();                   // no copy may outlive the CTA's shared memory
}

template <int MAXM, int TZ, int NT>
__global__ void __launch_bounds__(NT) field_advance_march2_kernel(FieldP p, int xc) {
    extern __shared__ float4 smem4[];
    const int z0 = blockIdx.x * TZ;
    const int xa = blockIdx.y * xc, xb = min(xa + xc, p.g.nx);
    march2_segment<MAXM, TZ>(p, z0, xa, xb, reinterpret_cast<float*>(smem4));
}

// Many independent 2D grids: a persistent grid walks a work list of (instance, z segment, first
// row, last row + 1) items; inst[2 i + parity] holds instance i's parameters for this step's
// buffer direction.  Every item is the x-marching segment of field_advance_march2_kernel.
template <int MAXM, int TZ, int NT>
__global__ void __launch_bounds__(NT) field_advance_march2_batch_kernel(const FieldP* __restrict__ inst,
                                                                        const int4* __restrict__ work, int nwork,
                                                                        int parity) {
    extern __shared__ float4 smem4[];
    __shared__ FieldP sp;
    for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
        const int4 it = work[w];
        __syncthreads();                        // the previous item is done with sp
        if (threadIdx.x == 0) sp = inst[2 * it.x + parity];
        __syncthreads();
        march2_segment<MAXM, TZ>(sp, it.y, it.z, it.w, reinterpret_cast<float*>(smem4));
    }
}

// Ring variant of the y-march: the planes a step needs next (E^n(k+3), B^n(k+2), J(k+2)) are
// copied by cp.async while the step computes, into a ring of 4 E, 3 B and 2 J planes.
template <int MAXM, int TZ, int TX>
struct MarchRingT {
    using P = MarchT<MAXM, TZ, TX>;
    static constexpr size_t smem_bytes = sizeof(float) * 3 * (4 * P::PE + 3 * P::PB + 2 * P::PJ);
};

template <int MAXM, int TZ, int TX, int NT>
__global__ void __launch_bounds__(NT) field_advance_march_ring_kernel(FieldP p, int yc) {
    using T = MarchT<MAXM, TZ, TX>;
    extern __shared__ float4 smem4[];
    float* sm = reinterpret_cast<float*>(smem4);
    const GridP& g = p.g;
    const long long N = g.ncell;
    const bool vec = p.vec4 != 0;
    const int z0 = blockIdx.x * TZ, x0 = blockIdx.y * TX;
    const int ya = blockIdx.z * yc, yb = min(ya + yc, g.ny);
    auto Eslot = [&](int i) { return sm + i * 3 * T::PE; };
    auto Bslot = [&](int i) { return sm + 12 * T::PE + i * 3 * T::PB; };
    auto Jslot = [&](int i) { return sm + 12 * T::PE + 9 * T::PB + i * 3 * T::PJ; };
    auto stageE = [&](int i, int y) {
        stage_plane(Eslot(i), T::PE, p.Ein, p.Ein + N, p.Ein + 2 * N, T::RX0, T::WE, z0 - T::H0, x0, -1,
                    wrapi(y, g.ny), g, vec);
    };
    auto stageB = [&](int i, int y) {
        stage_plane(Bslot(i), T::PB, p.Bin, p.Bin + N, p.Bin + 2 * N, T::RX1, T::WB, z0 - T::H1, x0, -1,
                    wrapi(y, g.ny), g, vec);
    };
    auto stageJ = [&](int i, int y) {
        stage_plane(Jslot(i), T::PJ, p.J1, p.J2, p.J3, T::RX2, T::WJ, z0 - T::H2, x0, 0, wrapi(y, g.ny), g, vec);
    };
    // prologue: B^{n+1/2}(ya-1), B^{n+1/2}(ya), E^{n+1}(ya), then the first prefetch
    stageE(0, ya - 1);
    stageE(1, ya);
    stageE(2, ya + 1);
    stageB(0, ya - 1);
    stageB(1, ya);
    stageJ(0, ya);
    cp_async_wait_all();
    __syncthreads();
    march_bhalf<MAXM, TZ, TX>(p, Bslot(0), Eslot(0), Eslot(1), z0);
    march_bhalf<MAXM, TZ, TX>(p, Bslot(1), Eslot(1), Eslot(2), z0);
    __syncthreads();
    march_enew<MAXM, TZ, TX>(p, Eslot(1), Bslot(1), Bslot(0), Jslot(0), z0);
    __syncthreads();
    // E: ec = E^{n+1}(k), en = E^n(k+1), ef = E^n(k+2) (in flight), eg = free
    // B: bc = B^{n+1/2}(k), bf = B^n(k+1) (in flight), bg = free;  J: jf = J(k+1) (in flight), jg = free
    int ec = 1, en = 2, ef = 3, eg = 0, bc = 1, bf = 2, bg = 0, jf = 1, jg = 0;
    stageE(ef, ya + 2);
    stageB(bf, ya + 1);
    stageJ(jf, ya + 1);
    cp_async_commit_group();
    for (int k = ya; k < yb; ++k) {
        stageE(eg, k + 3);
        stageB(bg, k + 2);
        stageJ(jg, k + 2);
        {
            cp_async_commit_group();
            cp_async_wait_prev_group();             // this step's planes (committed one step earlier)
        }
        __syncthreads();
        march_bhalf<MAXM, TZ, TX>(p, Bslot(bf), Eslot(en), Eslot(ef), z0);
        __syncthreads();
        march_enew<MAXM, TZ, TX>(p, Eslot(en), Bslot(bf), Bslot(bc), Jslot(jf), z0);
        __syncthreads();
        march_bnew_store<MAXM, TZ, TX>(p, Eslot(ec), Eslot(en), Bslot(bc), z0, x0, k, vec);
        __syncthreads();
        int t = ec;
        ec = en;
        en = ef;
        ef = eg;
        eg = t;
        t = bc;
        bc = bf;
        bf = bg;
        bg = t;
        t = jf;
        jf = jg;
        jg = t;
    }
    cp_async_wait_all();
}

template <int MAXM, int TZ, int TX, int NT>
__global__ void __launch_bounds__(NT) field_advance_march_kernel(FieldP p, int yc) {
    using T = MarchT<MAXM, TZ, TX>;
    extern __shared__ float4 smem4[];
    float* sm = reinterpret_cast<float*>(smem4);
    float* const sB0 = sm + 9 * T::PE;
    float* const sJ = sB0 + 6 * T::PB;
    const GridP& g = p.g;
    const long long N = g.ncell;
    const bool vec = p.vec4 != 0;
    const int z0 = blockIdx.x * TZ, x0 = blockIdx.y * TX;
    const int ya = blockIdx.z * yc, yb = min(ya + yc, g.ny);
    auto Eslot = [&](int i) { return sm + i * 3 * T::PE; };
    auto Bslot = [&](int i) { return sB0 + i * 3 * T::PB; };
    auto stageE = [&](int i, int y) {
        stage_plane(Eslot(i), T::PE, p.Ein, p.Ein + N, p.Ein + 2 * N, T::RX0, T::WE, z0 - T::H0, x0, -1,
                    wrapi(y, g.ny), g, vec);
    };
    auto stageB = [&](int i, int y) {
        stage_plane(Bslot(i), T::PB, p.Bin, p.Bin + N, p.Bin + 2 * N, T::RX1, T::WB, z0 - T::H1, x0, -1,
                    wrapi(y, g.ny), g, vec);
    };
    auto stageJ = [&](int y) {
        stage_plane(sJ, T::PJ, p.J1, p.J2, p.J3, T::RX2, T::WJ, z0 - T::H2, x0, 0, wrapi(y, g.ny), g, vec);
    };
    auto landed = [&]() {
        cp_async_wait_all();
        __syncthreads();
    };
    // prologue: B^{n+1/2}(ya-1), B^{n+1/2}(ya), E^{n+1}(ya)
    stageE(0, ya - 1);
    stageE(1, ya);
    stageB(0, ya - 1);
    landed();
    march_bhalf<MAXM, TZ, TX>(p, Bslot(0), Eslot(0), Eslot(1), z0);
    stageE(2, ya + 1);
    stageB(1, ya);
    stageJ(ya);
    landed();
    march_bhalf<MAXM, TZ, TX>(p, Bslot(1), Eslot(1), Eslot(2), z0);
    __syncthreads();
    march_enew<MAXM, TZ, TX>(p, Eslot(1), Bslot(1), Bslot(0), sJ, z0);
    __syncthreads();
    // E slots: ec = E^{n+1}(k), en = E^n(k+1), ef = free; B slots: bc = B^{n+1/2}(k), bf = free
    int ec = 1, en = 2, ef = 0, bc = 1, bf = 0;
    for (int k = ya; k < yb; ++k) {
        stageE(ef, k + 2);
        stageB(bf, k + 1);
        stageJ(k + 1);
        landed();
        march_bhalf<MAXM, TZ, TX>(p, Bslot(bf), Eslot(en), Eslot(ef), z0);
        __syncthreads();
        march_enew<MAXM, TZ, TX>(p, Eslot(en), Bslot(bf), Bslot(bc), sJ, z0);
        __syncthreads();
        march_bnew_store<MAXM, TZ, TX>(p, Eslot(ec), Eslot(en), Bslot(bc), z0, x0, k, vec);
        __syncthreads();
        const int t = ec;
        ec = en;
        en = ef;
        ef = t;
        const int u = bc;
        bc = bf;
        bf = u;
    }
}

template <int NDIM, int MAXM, int TZ, int TX, int TY>
__global__ void __launch_bounds__(256) field_advance_kernel(FieldP p) {
    extern __shared__ float smem[];
    advance_tile<NDIM, MAXM, TZ, TX, TY>(p, blockIdx.x, blockIdx.y, blockIdx.z, smem);
}

// Many independent grids in one launch: block b takes tile b of the concatenated tile list;
// tile_start[i] is the first tile of instance i (tile_start[ninst] = total).  inst[2 i + parity]
// holds instance i's parameters for this step's buffer direction.
template <int NDIM, int MAXM, int TZ, int TX, int TY>
__global__ void __launch_bounds__(256) field_advance_batch_kernel(const FieldP* __restrict__ inst,
                                                                  const int* __restrict__ tile_start, int ninst,
                                                                  int parity) {
    extern __shared__ float smem[];
    __shared__ FieldP sp;
    __shared__ int sidx, slocal;
    if (threadIdx.x == 0) {
        const int t = blockIdx.x;
        int lo = 0, hi = ninst - 1;          // last instance whose first tile is <= t
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (tile_start[mid] <= t) lo = mid; else hi = mid - 1;
        }
        sidx = lo;
        slocal = t - tile_start[lo];
        sp = inst[2 * lo + parity];
    }
    __syncthreads();
    const int ntz = (sp.g.nz + TZ - 1) / TZ, ntx = (sp.g.nx + TX - 1) / TX;
    const int l = slocal;
    const int tz = l % ntz, tx = (l / ntz) % ntx, ty = NDIM == 3 ? l / (ntz * ntx) : 0;
    advance_tile<NDIM, MAXM, TZ, TX, TY>(sp, tz, tx, ty, smem);
}

// The same tile list with the register-blocked tile (advance_tile_rb).
template <int NDIM, int MAXM, int TZ, int TX, int TY>
__global__ void __launch_bounds__(256, 2) field_advance_rb_batch_kernel(const FieldP* __restrict__ inst,
                                                                        const int* __restrict__ tile_start, int ninst,
                                                                        int parity) {
    extern __shared__ float4 smem4[];
    __shared__ FieldP sp;
    __shared__ int slocal;
    if (threadIdx.x == 0) {
        const int t = blockIdx.x;
        int lo = 0, hi = ninst - 1;          // last instance whose first tile is <= t
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (tile_start[mid] <= t) lo = mid; else hi = mid - 1;
        }
        slocal = t - tile_start[lo];
        sp = inst[2 * lo + parity];
    }
    __syncthreads();
    const int ntz = (sp.g.nz + TZ - 1) / TZ, ntx = (sp.g.nx + TX - 1) / TX;
    const int l = slocal;
    const int tz = l % ntz, tx = (l / ntz) % ntx, ty = NDIM == 3 ? l / (ntz * ntx) : 0;
    advance_tile_rb<NDIM, MAXM, TZ, TX, TY>(sp, tz, tx, ty, reinterpret_cast<float*>(smem4));
}

template <int NDIM, int MAXM, int TZ, int TX, int TY>
cudaError_t launch_fa(const FieldP& p, cudaStream_t s) {
    using T = Tile<NDIM, MAXM, TZ, TX, TY>;
    auto k = field_advance_kernel<NDIM, MAXM, TZ, TX, TY>;
    static bool configured = false;   // attribute is per function; setting it twice is harmless
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)T::smem_bytes);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    dim3 grid((p.g.nz + TZ - 1) / TZ, (p.g.nx + TX - 1) / TX, NDIM == 3 ? (p.g.ny + TY - 1) / TY : 1);
    k<<<grid, 256, T::smem_bytes, s>>>(p);
    return cudaGetLastError();
}

template <int NDIM, int MAXM, int TZ, int TX, int TY>
cudaError_t launch_fa_rb(const FieldP& p, cudaStream_t s) {
    using T = TileRB<NDIM, MAXM, TZ, TX, TY>;
    auto k = field_advance_rb_kernel<NDIM, MAXM, TZ, TX, TY>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)T::smem_bytes);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    dim3 grid((p.g.nz + TZ - 1) / TZ, (p.g.nx + TX - 1) / TX, NDIM == 3 ? (p.g.ny + TY - 1) / TY : 1);
    k<<<grid, 256, T::smem_bytes, s>>>(p);
    return cudaGetLastError();
}

// Rows (2D) or planes (3D) per marching chunk: the chunk count that minimises the number of waves
// times the rows a CTA walks (its chunk plus the two its prologue recomputes), chunks of at least
// `minc` rows.  `cols` CTAs march side by side; `slots` CTAs run at once.
inline int march_chunk(int n, int cols, int slots, int minc) {
    int best = n, best_cost = INT_MAX;
    for (int chunks = 1; chunks <= 64; ++chunks) {
        int c = (n + chunks - 1) / chunks;
        if (c < minc) c = minc;
        const long long ctas = (long long)cols * ((n + c - 1) / c);
        const long long waves = (ctas + slots - 1) / slots;
        const long long cost = waves * (c + 2);
        if (cost < best_cost) {
            best_cost = (int)cost;
            best = c;
        }
    }
    return best;
}

template <int MAXM, int TZ, int TX, int NT>
cudaError_t launch_fa_march(const FieldP& p, cudaStream_t s) {
    using T = MarchT<MAXM, TZ, TX>;
    auto k = field_advance_march_kernel<MAXM, TZ, TX, NT>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::smem_bytes);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    // y chunks: about four waves of CTAs over the SMs, each chunk at least 8 planes
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int cols = ((p.g.nz + TZ - 1) / TZ) * ((p.g.nx + TX - 1) / TX);
    int per_sm = (int)((227 * 1024) / (T::smem_bytes + 1024));
    per_sm = per_sm < 1 ? 1 : (per_sm > 2048 / NT ? 2048 / NT : per_sm);
    const int yc = march_chunk(p.g.ny, cols, nsm * per_sm, 8);
    dim3 grid((p.g.nz + TZ - 1) / TZ, (p.g.nx + TX - 1) / TX, (p.g.ny + yc - 1) / yc);
    k<<<grid, NT, T::smem_bytes, s>>>(p, yc);
    return cudaGetLastError();
}

template <int MAXM, int TZ, int NT>
cudaError_t launch_fa_march2(const FieldP& p, cudaStream_t s) {
    using T = March2T<MAXM, TZ>;
    auto k = field_advance_march2_kernel<MAXM, TZ, NT>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::smem_bytes);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    // x chunks: one wave of CTAs over the SMs, each chunk at least 16 rows (the prologue of a
    // chunk recomputes two rows)
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int cols = (p.g.nz + TZ - 1) / TZ;
    int per_sm = (int)((227 * 1024) / (T::smem_bytes + 1024));
    per_sm = per_sm < 1 ? 1 : (per_sm > 2048 / NT ? 2048 / NT : per_sm);
    const int xc = march_chunk(p.g.nx, cols, nsm * per_sm, 16);
    dim3 grid(cols, (p.g.nx + xc - 1) / xc, 1);
    k<<<grid, NT, T::smem_bytes, s>>>(p, xc);
    return cudaGetLastError();
}

template <int MAXM, int TZ, int TX, int NT>
cudaError_t launch_fa_march_ring(const FieldP& p, cudaStream_t s) {
    using T = MarchRingT<MAXM, TZ, TX>;
    auto k = field_advance_march_ring_kernel<MAXM, TZ, TX, NT>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::smem_bytes);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    // y chunks: one wave of CTAs, each chunk at least 8 planes
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int cols = ((p.g.nz + TZ - 1) / TZ) * ((p.g.nx + TX - 1) / TX);
    int per_sm = (int)((227 * 1024) / (T::smem_bytes + 1024));
    per_sm = per_sm < 1 ? 1 : (per_sm > 2048 / NT ? 2048 / NT : per_sm);
    const int yc = march_chunk(p.g.ny, cols, nsm * per_sm, 8);
    dim3 grid((p.g.nz + TZ - 1) / TZ, (p.g.nx + TX - 1) / TX, (p.g.ny + yc - 1) / yc);
    k<<<grid, NT, T::smem_bytes, s>>>(p, yc);
    return cudaGetLastError();
}

template <int NDIM, int MAXM, int TZ, int TX, int TY>
cudaError_t launch_fa_batch(const FieldP* inst, const int* tile_start, int ninst, int total, int parity,
                            cudaStream_t s) {
    using T = Tile<NDIM, MAXM, TZ, TX, TY>;
    auto k = field_advance_batch_kernel<NDIM, MAXM, TZ, TX, TY>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::smem_bytes);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    k<<<(unsigned)total, 256, T::smem_bytes, s>>>(inst, tile_start, ninst, parity);
    return cudaGetLastError();
}

}  // namespace

template <int NDIM, int MAXM, int TZ, int TX, int TY>
cudaError_t launch_fa_rb_batch(const FieldP* inst, const int* tile_start, int ninst, int total, int parity,
                               cudaStream_t s) {
    using T = TileRB<NDIM, MAXM, TZ, TX, TY>;
    auto k = field_advance_rb_batch_kernel<NDIM, MAXM, TZ, TX, TY>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::smem_bytes);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    k<<<(unsigned)total, 256, T::smem_bytes, s>>>(inst, tile_start, ninst, parity);
    return cudaGetLastError();
}

template <int MAXM, int TZ, int NT>
cudaError_t launch_fa_march2_batch(const FieldP* inst, const int4* work, int nwork, int parity, cudaStream_t s) {
    using T = March2T<MAXM, TZ>;
    auto k = field_advance_march2_batch_kernel<MAXM, TZ, NT>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::smem_bytes);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = (int)((227 * 1024) / (T::smem_bytes + 1024));
    per_sm = per_sm < 1 ? 1 : (per_sm > 2048 / NT ? 2048 / NT : per_sm);
    const int grid = nwork < nsm * per_sm ? nwork : nsm * per_sm;
    if (grid <= 0) return cudaSuccess;
    k<<<grid, NT, T::smem_bytes, s>>>(inst, work, nwork, parity);
    return cudaGetLastError();
}

// Tiles of one grid in the batched field advance (same tile shapes as launch_field_advance_batch).
// Batched 2D x-march: z segments of MARCH2_BATCH_TZ cells (64 threads), rows in chunks.
cudaError_t launch_field_advance_march2_batch(const FieldP* inst, const int4* work, int nwork, int maxm, int parity,
                                              cudaStream_t s) {
    if (nwork <= 0) return cudaSuccess;
    if (maxm <= 1) return launch_fa_march2_batch<1, MARCH2_BATCH_TZ, 64>(inst, work, nwork, parity, s);
    if (maxm <= 4) return launch_fa_march2_batch<4, MARCH2_BATCH_TZ, 64>(inst, work, nwork, parity, s);
    if (maxm <= 8) return launch_fa_march2_batch<8, MARCH2_BATCH_TZ, 64>(inst, work, nwork, parity, s);
    return launch_fa_march2_batch<16, MARCH2_BATCH_TZ, 64>(inst, work, nwork, parity, s);
}

int field_tiles(int ndim, int maxm, int nz, int nx, int ny) {
    (void)maxm;
    if (ndim == 2) return ((nz + 127) / 128) * ((nx + 7) / 8);
    return ((nz + 63) / 64) * ((nx + 3) / 4) * ((ny + 3) / 4);
}

cudaError_t launch_field_advance_rb_batch(const FieldP* inst, const int* tile_start, int ninst, int total_tiles,
                                          int ndim, int maxm, int parity, cudaStream_t s) {
    if (ninst <= 0 || total_tiles <= 0) return cudaSuccess;
    if (ndim == 2) {
        if (maxm <= 1) return launch_fa_rb_batch<2, 1, 128, 8, 1>(inst, tile_start, ninst, total_tiles, parity, s);
        if (maxm <= 4) return launch_fa_rb_batch<2, 4, 128, 8, 1>(inst, tile_start, ninst, total_tiles, parity, s);
        if (maxm <= 8) return launch_fa_rb_batch<2, 8, 128, 8, 1>(inst, tile_start, ninst, total_tiles, parity, s);
        return launch_fa_rb_batch<2, 16, 128, 8, 1>(inst, tile_start, ninst, total_tiles, parity, s);
    }
    if (maxm <= 1) return launch_fa_rb_batch<3, 1, 64, 4, 4>(inst, tile_start, ninst, total_tiles, parity, s);
    if (maxm <= 4) return launch_fa_rb_batch<3, 4, 64, 4, 4>(inst, tile_start, ninst, total_tiles, parity, s);
    if (maxm <= 8) return launch_fa_rb_batch<3, 8, 64, 4, 4>(inst, tile_start, ninst, total_tiles, parity, s);
    return launch_fa_rb_batch<3, 16, 64, 4, 4>(inst, tile_start, ninst, total_tiles, parity, s);
}

cudaError_t launch_field_advance_batch(const FieldP* inst, const int* tile_start, int ninst, int total_tiles,
                                       int ndim, int maxm, int parity, cudaStream_t s) {
    if (ninst <= 0 || total_tiles <= 0) return cudaSuccess;
    if (ndim == 2) {
        if (maxm <= 1) return launch_fa_batch<2, 1, 128, 8, 1>(inst, tile_start, ninst, total_tiles, parity, s);
        if (maxm <= 4) return launch_fa_batch<2, 4, 128, 8, 1>(inst, tile_start, ninst, total_tiles, parity, s);
        if (maxm <= 8) return launch_fa_batch<2, 8, 128, 8, 1>(inst, tile_start, ninst, total_tiles, parity, s);
        return launch_fa_batch<2, 16, 128, 8, 1>(inst, tile_start, ninst, total_tiles, parity, s);
    }
    if (maxm <= 1) return launch_fa_batch<3, 1, 64, 4, 4>(inst, tile_start, ninst, total_tiles, parity, s);
    if (maxm <= 4) return launch_fa_batch<3, 4, 64, 4, 4>(inst, tile_start, ninst, total_tiles, parity, s);
    if (maxm <= 8) return launch_fa_batch<3, 8, 64, 4, 4>(inst, tile_start, ninst, total_tiles, parity, s);
    return launch_fa_batch<3, 16, 64, 4, 4>(inst, tile_start, ninst, total_tiles, parity, s);
}

// Tile variants the autotuner chooses from.  2D: (TZ, TX); 3D: (TZ, TX, TY); rb = register-
// blocked tile (four z cells per thread).
//   2D: 0 = 128 x 8, 1 = 256 x 4, 2 = 64 x 16, 3 = 256 x 8,
//       4 = rb 128 x 8, 5 = rb 256 x 4, 6 = rb 128 x 4, 7 = rb 256 x 8,
//       8 = x-march z 448 (128 threads), 9 = x-march z 384 (128 threads),
//       10 = x-march z 960 (256 threads), 11 = x-march z 192 (64 threads)
//   3D: 0 = 64 x 4 x 4, 1 = 128 x 4 x 2, 2 = 32 x 8 x 4,
//       3 = rb 64 x 4 x 4, 4 = rb 128 x 4 x 2, 5 = rb 32 x 8 x 4,
//       6 = y-march 128 x 4 (256 threads), 7 = y-march 128 x 4 (128 threads),
//       8 = y-march 128 x 8 (256 threads), 9 = y-march 64 x 8 (256 threads),
//       10 = y-march with prefetch ring 128 x 8 (512 threads), 11 = ring 64 x 4 (128 threads)
int field_variants(int ndim) { return ndim == 2 ? 12 : 12; }

// Variant used before (or without) pic_autotune: the register-blocked tile for the customised
// stencils, the scalar tile for Yee.
int default_field_variant(int ndim, int M) {
    if (M <= 1) return 0;
    return ndim == 2 ? 4 : 10;
}

namespace {
template <int NDIM, int MAXM>
cudaError_t launch_fa_variant(const FieldP& p, int v, cudaStream_t s) {
    if (NDIM == 2) {
        switch (v) {
            case 1: return launch_fa<2, MAXM, 256, 4, 1>(p, s);
            case 2: return launch_fa<2, MAXM, 64, 16, 1>(p, s);
            case 3: return launch_fa<2, MAXM, 256, 8, 1>(p, s);
            case 4: return launch_fa_rb<2, MAXM, 128, 8, 1>(p, s);
            case 5: return launch_fa_rb<2, MAXM, 256, 4, 1>(p, s);
            case 6: return launch_fa_rb<2, MAXM, 128, 4, 1>(p, s);
            case 7: return launch_fa_rb<2, MAXM, 256, 8, 1>(p, s);
            case 8: return launch_fa_march2<MAXM, 448, 128>(p, s);
            case 9: return launch_fa_march2<MAXM, 384, 128>(p, s);
            case 10: return launch_fa_march2<MAXM, 960, 256>(p, s);
            case 11: return launch_fa_march2<MAXM, 192, 64>(p, s);
            default: return launch_fa<2, MAXM, 128, 8, 1>(p, s);
        }
    }
    switch (v) {
        case 1: return launch_fa<3, MAXM, 128, 4, 2>(p, s);
        case 2: return launch_fa<3, MAXM, 32, 8, 4>(p, s);
        case 3: return launch_fa_rb<3, MAXM, 64, 4, 4>(p, s);
        case 4: return launch_fa_rb<3, MAXM, 128, 4, 2>(p, s);
        case 5: return launch_fa_rb<3, MAXM, 32, 8, 4>(p, s);
        case 6: return launch_fa_march<MAXM, 128, 4, 256>(p, s);
        case 7: return launch_fa_march<MAXM, 128, 4, 128>(p, s);
        case 8: return launch_fa_march<MAXM, 128, 8, 256>(p, s);
        case 9: return launch_fa_march<MAXM, 64, 8, 256>(p, s);
        case 10: return launch_fa_march_ring<MAXM, 128, 8, 512>(p, s);
        case 11: return launch_fa_march_ring<MAXM, 64, 4, 128>(p, s);
        default: return launch_fa<3, MAXM, 64, 4, 4>(p, s);
    }
}

bool aligned16(const void* q) { return ((uintptr_t)q & 15) == 0; }
}  // namespace

cudaError_t launch_field_advance(const FieldP& p_in, cudaStream_t s, int variant) {
    FieldP p = p_in;
    p.vec4 = (p.g.nz % 4 == 0) && aligned16(p.Ein) && aligned16(p.Bin) && aligned16(p.J1) && aligned16(p.J2) &&
             aligned16(p.J3) && aligned16(p.Eout) && aligned16(p.Bout);
    const int M = p.st.M;
    if (p.g.ndim == 2) {
        if (M <= 1) return launch_fa_variant<2, 1>(p, variant, s);
        if (M <= 4) return launch_fa_variant<2, 4>(p, variant, s);
        if (M <= 8) return launch_fa_variant<2, 8>(p, variant, s);
        return launch_fa_variant<2, 16>(p, variant, s);
    }
    if (M <= 1) return launch_fa_variant<3, 1>(p, variant, s);
    if (M <= 4) return launch_fa_variant<3, 4>(p, variant, s);
    if (M <= 8) return launch_fa_variant<3, 8>(p, variant, s);
    return launch_fa_variant<3, 16>(p, variant, s);
}

}  // namespace pic
