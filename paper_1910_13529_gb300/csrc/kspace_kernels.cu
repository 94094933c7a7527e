// k-space field advance: the spectral solver of Sec. 2.3 ([k]_a = k_a), the operator of Sec. 3
// applied exactly in k space ([k]_1 = [k1]_t along z, Yee across), and PSATD (Appendix B).
//
// The fields stay on the staggered grid of the finite-difference solver and are periodic along
// every axis.  Per step: forward real-to-complex transforms of E, B, J (cuFFT, three components per
// call), one update kernel over the k-space modes, inverse transforms of E and B.  For each axis the
// host tabulates, per FFT index, the forward-difference symbol d+ = e^{i k h/2} i [k](k) (the
// backward one is d- = e^{-i k h/2} i [k](k), the same numbers with the real part negated) and the
// current ratio [k]_Yee / [k], which makes the scaled current obey the continuity equation of this
// solver's d- (the k-space form of the Sec. 3 correction), so Gauss's law d-.E = rho is kept.
// Update, per mode, in the order of Eq. 1:
//   B -= dt/2 curl+ E;   E += dt (curl- B - J ratio);   B -= dt/2 curl+ E;
//   (curl F)_1 = d_x F3 - d_y F2,  (curl F)_2 = d_y F1 - d_z F3,  (curl F)_3 = d_z F2 - d_x F1,
// E and B scaled by 1/(nz nx ny) for the unnormalised inverse transform.  Memory per mode: 9 complex
// values read, 6 written.
#include "pic_internal.h"

#include <cmath>
#include <cstdio>
#include <vector>

#ifdef PIC_HAVE_CUFFT
#include <cufft.h>
#endif

namespace pic {

struct KSpaceState {
    GridP g;
    int solver = 0;
    long long nk = 0;          // modes: (nz/2 + 1) nx ny
    int nzk = 0;
    float2* buf = nullptr;     // E, B, J in k space: 9 nk complex values
    float4* tab = nullptr;     // per axis and index, z then x then y: spectral/KT (d+ re, d+ im,
                               // [k]_Yee / [k], 0); PSATD (cos(k h/2), sin(k h/2), k, ratio or -1)
#ifdef PIC_HAVE_CUFFT
    cufftHandle r2c = 0, c2r = 0;
    bool have_r2c = false, have_c2r = false;
#endif
};

bool kspace_available() {
#ifdef PIC_HAVE_CUFFT
    return true;
#else
    return false;
#endif
}

namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cfma(float s, float2 a, float2 b) {     // b + s a
    return make_float2(fmaf(s, a.x, b.x), fmaf(s, a.y, b.y));
}

// curl with the per-axis symbols dz, dx, dy
__device__ __forceinline__ void ccurl(float2 dz, float2 dx, float2 dy, const float2 (&F)[3], float2 (&out)[3]) {
    out[0] = csub(cmul(dx, F[2]), cmul(dy, F[1]));
    out[1] = csub(cmul(dy, F[0]), cmul(dz, F[2]));
    out[2] = csub(cmul(dz, F[1]), cmul(dx, F[0]));
}

__global__ void __launch_bounds__(256) kspace_update_kernel(float2* __restrict__ Ek, float2* __restrict__ Bk,
                                                            const float2* __restrict__ Jk,
                                                            const float4* __restrict__ tab, int nzk, int nx,
                                                            long long nk, float dt, float scale) {
    const float4* tz = tab;
    const float4* tx = tab + nzk;
    const float4* ty = tab + nzk + nx;
    for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < nk;
         m += (long long)gridDim.x * blockDim.x) {
        const int iz = (int)(m % nzk);
        const long long r = m / nzk;
        const int ix = (int)(r % nx), iy = (int)(r / nx);
        const float4 a = __ldg(tz + iz), b = __ldg(tx + ix), c = __ldg(ty + iy);
        const float2 pz = make_float2(a.x, a.y), px = make_float2(b.x, b.y), py = make_float2(c.x, c.y);
        const float2 mz = make_float2(-a.x, a.y), mx = make_float2(-b.x, b.y), my = make_float2(-c.x, c.y);
        const float ratio[3] = {a.z, b.z, c.z};
        float2 E[3], B[3], J[3], t[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            E[q] = Ek[q * nk + m];
            B[q] = Bk[q * nk + m];
            J[q] = Jk[q * nk + m];
        }
        ccurl(pz, px, py, E, t);
#pragma unroll
        for (int q = 0; q < 3; ++q) B[q] = cfma(-0.5f * dt, t[q], B[q]);
        ccurl(mz, mx, my, B, t);
#pragma unroll
        for (int q = 0; q < 3; ++q) E[q] = cfma(dt, csub(t[q], make_float2(ratio[q] * J[q].x, ratio[q] * J[q].y)), E[q]);
        ccurl(pz, px, py, E, t);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            B[q] = cfma(-0.5f * dt, t[q], B[q]);
            Ek[q * nk + m] = make_float2(E[q].x * scale, E[q].y * scale);
            Bk[q * nk + m] = make_float2(B[q].x * scale, B[q].y * scale);
        }
    }
}

// PSATD (Appendix B, Eqs. B1-B2) per mode, k = |k|, c = cos(k dt), s = sin(k dt):
//   E <- c E + i s khat x B - (s/k) J + (1 - c) khat (khat.E) + (s/k - dt) khat (khat.J)
//   B <- c B - i s khat x E + i (1 - c)/k khat x J            (both from the old E, B)
// on collocated values: each staggered component is multiplied by e^{-i k_a h_a/2} for every axis a
// along which it sits half a cell up (E1 z, E2 x, E3 y; B1 x y, B2 z y, B3 z x; J like E), updated
// and multiplied back.  Tables per axis and index: (cos(k h/2), sin(k h/2), k, [k]_Yee / k), the
// last negative on the Nyquist plane of an even axis, whose modes are removed.  At k = 0:
// E <- E - dt J, B unchanged.
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 ci(float2 a) { return make_float2(-a.y, a.x); }          // i a
__device__ __forceinline__ float2 cscale(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }

__global__ void __launch_bounds__(256) psatd_update_kernel(float2* __restrict__ Ek, float2* __restrict__ Bk,
                                                           const float2* __restrict__ Jk,
                                                           const float4* __restrict__ tab, int nzk, int nx,
                                                           long long nk, float dt, float scale) {
    const float4* tz = tab;
    const float4* tx = tab + nzk;
    const float4* ty = tab + nzk + nx;
    for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < nk;
         m += (long long)gridDim.x * blockDim.x) {
        const int iz = (int)(m % nzk);
        const long long r = m / nzk;
        const int ix = (int)(r % nx), iy = (int)(r / nx);
        const float4 a = __ldg(tz + iz), b = __ldg(tx + ix), c = __ldg(ty + iy);
        if (a.w < 0.f || b.w < 0.f || c.w < 0.f) {          // Nyquist plane: removed
#pragma unroll
            for (int q = 0; q < 3; ++q) Ek[q * nk + m] = Bk[q * nk + m] = make_float2(0.f, 0.f);
            continue;
        }
        // e^{-i k h/2} per axis (z, x, y)
        const float2 ph[3] = {make_float2(a.x, -a.y), make_float2(b.x, -b.y), make_float2(c.x, -c.y)};
        const float2 pE[3] = {ph[0], ph[1], ph[2]};
        const float2 pB[3] = {cmul(ph[1], ph[2]), cmul(ph[0], ph[2]), cmul(ph[0], ph[1])};
        const float ratio[3] = {a.w, b.w, c.w};
        float2 E[3], B[3], J[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            E[q] = cmul(Ek[q * nk + m], pE[q]);
            B[q] = cmul(Bk[q * nk + m], pB[q]);
            J[q] = cscale(ratio[q], cmul(Jk[q * nk + m], pE[q]));
        }
        const float kv[3] = {a.z, b.z, c.z};
        const float kn = sqrtf(kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2]);
        float2 En[3], Bn[3];
        if (kn == 0.f) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                En[q] = cfma(-dt, J[q], E[q]);
                Bn[q] = B[q];
            }
        } else {
            float S, C;
            sincosf(kn * dt, &S, &C);
            const float kh[3] = {kv[0] / kn, kv[1] / kn, kv[2] / kn};
            const float sk = S / kn, omck = (1.f - C) / kn;
            auto cross = [&](const float2 (&f)[3], float2 (&o)[3]) {
                o[0] = make_float2(kh[1] * f[2].x - kh[2] * f[1].x, kh[1] * f[2].y - kh[2] * f[1].y);
                o[1] = make_float2(kh[2] * f[0].x - kh[0] * f[2].x, kh[2] * f[0].y - kh[0] * f[2].y);
                o[2] = make_float2(kh[0] * f[1].x - kh[1] * f[0].x, kh[0] * f[1].y - kh[1] * f[0].y);
            };
            float2 kxB[3], kxE[3], kxJ[3];
            cross(B, kxB);
            cross(E, kxE);
            cross(J, kxJ);
            const float2 kE = make_float2(kh[0] * E[0].x + kh[1] * E[1].x + kh[2] * E[2].x,
                                          kh[0] * E[0].y + kh[1] * E[1].y + kh[2] * E[2].y);
            const float2 kJ = make_float2(kh[0] * J[0].x + kh[1] * J[1].x + kh[2] * J[2].x,
                                          kh[0] * J[0].y + kh[1] * J[1].y + kh[2] * J[2].y);
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                float2 e = cscale(C, E[q]);
                e = cadd(e, cscale(S, ci(kxB[q])));
                e = cfma(-sk, J[q], e);
                e = cfma((1.f - C) * kh[q], kE, e);
                e = cfma((sk - dt) * kh[q], kJ, e);
                En[q] = e;
                float2 bq = cscale(C, B[q]);
                bq = cfma(-S, ci(kxE[q]), bq);
                bq = cadd(bq, cscale(omck, ci(kxJ[q])));
                Bn[q] = bq;
            }
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            Ek[q * nk + m] = cscale(scale, cmul(En[q], cconj(pE[q])));
            Bk[q * nk + m] = cscale(scale, cmul(Bn[q], cconj(pB[q])));
        }
    }
}

// [k](k) of an axis: spectral k; [k1]_t along z for KT; Yee (2/h) sin(k h/2) otherwise
double axis_symbol(int solver, int axis, double k, double h, double dt) {
    if (solver == PIC_SOLVER_SPECTRAL) return k;
    if (solver == PIC_SOLVER_KT && axis == 0) return 2.0 / dt * std::sin(0.5 * k * dt);
    return 2.0 / h * std::sin(0.5 * k * h);
}

void fill_axis(std::vector<float4>& out, int solver, int axis, int n, double h, double dt, bool half, bool absent) {
    const int cnt = half ? n / 2 + 1 : n;
    for (int j = 0; j < cnt; ++j) {
        if (absent) {                                  // 2D: no y axis
            out.push_back(solver == PIC_SOLVER_PSATD ? make_float4(1.f, 0.f, 0.f, 1.f) : make_float4(0.f, 0.f, 1.f, 0.f));
            continue;
        }
        const int jj = (half || j <= (n - 1) / 2) ? j : j - n;
        const double k = 2.0 * M_PI * jj / (n * h);
        if (solver == PIC_SOLVER_PSATD) {
            const double th = 0.5 * k * h;
            const bool nyq = n % 2 == 0 && j == n / 2;
            const double ratio = k == 0.0 ? 1.0 : (2.0 / h * std::sin(th)) / k;
            out.push_back(make_float4((float)std::cos(th), (float)std::sin(th), (float)k, nyq ? -1.f : (float)ratio));
            continue;
        }
        const double kap = axis_symbol(solver, axis, k, h, dt);
        const double yee = 2.0 / h * std::sin(0.5 * k * h);
        const double th = 0.5 * k * h;
        const double ratio = kap == 0.0 ? 1.0 : yee / kap;
        out.push_back(make_float4((float)(-kap * std::sin(th)), (float)(kap * std::cos(th)), (float)ratio, 0.f));
    }
}

}  // namespace

int kspace_create(const GridP& g, int solver, double dz, double dx, double dy, double dt, KSpaceState** out,
                  char* err, size_t nerr) {
    *out = nullptr;
#ifndef PIC_HAVE_CUFFT
    (void)g; (void)solver; (void)dz; (void)dx; (void)dy; (void)dt;
    snprintf(err, nerr, "k-space solvers need cuFFT, which this build does not have");
    return 1;
#else
    KSpaceState* k = new KSpaceState();
    k->g = g;
    k->solver = solver;
    k->nzk = g.nz / 2 + 1;
    k->nk = (long long)k->nzk * g.nx * g.ny;
    std::vector<float4> tab;
    fill_axis(tab, solver, 0, g.nz, dz, dt, true, false);
    fill_axis(tab, solver, 1, g.nx, dx, dt, false, false);
    fill_axis(tab, solver, 2, g.ny, dy, dt, false, g.ndim == 2);
    cudaError_t e = cudaMalloc(&k->buf, sizeof(float2) * 9 * k->nk);
    if (e == cudaSuccess) e = cudaMalloc(&k->tab, sizeof(float4) * tab.size());
    if (e == cudaSuccess) e = cudaMemcpy(k->tab, tab.data(), sizeof(float4) * tab.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        snprintf(err, nerr, "k-space buffers: %s", cudaGetErrorString(e));
        kspace_destroy(k);
        return 2;
    }
    int n3[3] = {g.ny, g.nx, g.nz}, n2[2] = {g.nx, g.nz};
    const int rank = g.ndim == 3 ? 3 : 2;
    int* n = rank == 3 ? n3 : n2;
    cufftResult r = cufftPlanMany(&k->r2c, rank, n, nullptr, 1, 0, nullptr, 1, 0, CUFFT_R2C, 3);
    k->have_r2c = r == CUFFT_SUCCESS;
    if (r == CUFFT_SUCCESS) {
        r = cufftPlanMany(&k->c2r, rank, n, nullptr, 1, 0, nullptr, 1, 0, CUFFT_C2R, 3);
        k->have_c2r = r == CUFFT_SUCCESS;
    }
    if (r != CUFFT_SUCCESS) {
        snprintf(err, nerr, "cuFFT plan creation failed (%d)", (int)r);
        kspace_destroy(k);
        return r == CUFFT_ALLOC_FAILED ? 2 : 1;
    }
    *out = k;
    return 0;
#endif
}

void kspace_destroy(KSpaceState* k) {
    if (!k) return;
#ifdef PIC_HAVE_CUFFT
    if (k->have_r2c) cufftDestroy(k->r2c);
    if (k->have_c2r) cufftDestroy(k->c2r);
#endif
    if (k->buf) cudaFree(k->buf);
    if (k->tab) cudaFree(k->tab);
    delete k;
}

long long kspace_modes(const KSpaceState* k) { return k ? k->nk : 0; }

// Ein, Bin, J (three components each, [c][y][x][z]) -> Eout, Bout.  Out-of-place real-to-complex
// transforms leave their input unchanged; the complex-to-real ones overwrite the k-space buffer.
int kspace_advance(KSpaceState* k, const float* Ein, const float* Bin, const float* J, float* Eout, float* Bout,
                   cudaStream_t s, char* err, size_t nerr) {
#ifndef PIC_HAVE_CUFFT
    (void)k; (void)Ein; (void)Bin; (void)J; (void)Eout; (void)Bout; (void)s;
    snprintf(err, nerr, "k-space solvers need cuFFT, which this build does not have");
    return 1;
#else
    float2* Ek = k->buf;
    float2* Bk = Ek + 3 * k->nk;
    float2* Jk = Bk + 3 * k->nk;
    cufftResult r = cufftSetStream(k->r2c, s);
    if (r == CUFFT_SUCCESS) r = cufftSetStream(k->c2r, s);
    if (r == CUFFT_SUCCESS)
        r = cufftExecR2C(k->r2c, const_cast<cufftReal*>(Ein), reinterpret_cast<cufftComplex*>(Ek));
    if (r == CUFFT_SUCCESS)
        r = cufftExecR2C(k->r2c, const_cast<cufftReal*>(Bin), reinterpret_cast<cufftComplex*>(Bk));
    if (r == CUFFT_SUCCESS)
        r = cufftExecR2C(k->r2c, const_cast<cufftReal*>(J), reinterpret_cast<cufftComplex*>(Jk));
    if (r != CUFFT_SUCCESS) {
        snprintf(err, nerr, "cuFFT forward transform failed (%d)", (int)r);
        return 1;
    }
    const GridP& g = k->g;
    const long long blocks = (k->nk + 255) / 256;
    const unsigned nb = (unsigned)(blocks < 152 * 8 ? (blocks < 1 ? 1 : blocks) : 152 * 8);
    const float scale = (float)(1.0 / ((double)g.nz * g.nx * g.ny));
    if (k->solver == PIC_SOLVER_PSATD)
        psatd_update_kernel<<<nb, 256, 0, s>>>(Ek, Bk, Jk, k->tab, k->nzk, g.nx, k->nk, g.dt, scale);
    else
        kspace_update_kernel<<<nb, 256, 0, s>>>(Ek, Bk, Jk, k->tab, k->nzk, g.nx, k->nk, g.dt, scale);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(err, nerr, "k-space update kernel: %s", cudaGetErrorString(e));
        return 1;
    }
    r = cufftExecC2R(k->c2r, reinterpret_cast<cufftComplex*>(Ek), reinterpret_cast<cufftReal*>(Eout));
    if (r == CUFFT_SUCCESS)
        r = cufftExecC2R(k->c2r, reinterpret_cast<cufftComplex*>(Bk), reinterpret_cast<cufftReal*>(Bout));
    if (r != CUFFT_SUCCESS) {
        snprintf(err, nerr, "cuFFT inverse transform failed (%d)", (int)r);
        return 1;
    }
    return 0;
#endif
}

}  // namespace pic
