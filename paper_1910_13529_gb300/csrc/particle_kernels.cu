// Particle kernels for sm_103a: field gather, relativistic Boris push, position update and
// charge-conserving (Esirkepov) current deposition (Sec. 1 PIC loop; Sec. 2.1 requires the
// deposition to conserve charge so that Gauss's law holds), plus counting sort, moving-window
// injection and the FP64 charge density used by the diagnostics.
//
// Positions are (integer cell, FP32 offset in [0,1)) so that precision does not degrade with
// the distance from the origin.  Shape factors of a position are always computed from its own
// offset and placed into the deposition window by an integer shift, which makes the "new"
// shape of one step bit-identical to the "old" shape of the next: charge is conserved to FP32
// round-off per step with no drift from re-rounded positions.
#include <cuda_runtime.h>

#include <climits>
#include <type_traits>

#include "pic_internal.h"

namespace pic {

namespace {

// ---------------------------------------------------------------- shapes ----
// Weights of the K nodes a position touches, first node at cell + rel.
template <int SHAPE>
struct Shape;

template <>
struct Shape<1> {                         // linear B-spline: S(d) = 1 - |d|
    static constexpr int K = 2;
    template <typename R>
    __device__ static __forceinline__ int w(R o, R* W) {
        W[0] = R(1) - o;
        W[1] = o;
        return 0;
    }
};

template <>
struct Shape<2> {                         // quadratic B-spline centred on the nearest node
    static constexpr int K = 3;
    template <typename R>
    __device__ static __forceinline__ int w(R o, R* W) {
        int up = o >= R(0.5);
        R d = o - (R)up;                  // in [-1/2, 1/2)
        R a = R(0.5) - d, b = R(0.5) + d;
        W[0] = R(0.5) * a * a;
        W[1] = R(0.75) - d * d;
        W[2] = R(0.5) * b * b;
        return up - 1;
    }
};

// weights for a component staggered by half a cell along this axis: shift the position by -1/2
template <int SHAPE>
__device__ __forceinline__ int half_weights(int cell, float o, float* W) {
    if (o >= 0.5f) return cell + Shape<SHAPE>::w(o - 0.5f, W);
    return cell - 1 + Shape<SHAPE>::w(o + 0.5f, W);
}

// periodic wrap of an index at most one period outside [0, n)
__device__ __forceinline__ int wrapi(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f) {
    if (f.s < 0) return n;
    uint32_t t = __umulhi(f.m, n);
    return (t + ((n - t) >> 1)) >> (f.s - 1);
}

// magic-number constants of the grid's divisors, computed on the device (batched instances)
__device__ __forceinline__ FastDiv make_fastdiv_device(uint32_t d) {
    FastDiv f{d, 0u, -1};
    if (d <= 1) return f;
    int l = 32 - __clz(d - 1);
    f.m = (uint32_t)((((1ull << 32) * ((1ull << l) - d)) / d) + 1);
    f.s = l;
    return f;
}

__device__ __forceinline__ GridP prep_device(GridP g) {
    g.div_nzg = make_fastdiv_device((uint32_t)g.nzg);
    g.div_nx = make_fastdiv_device((uint32_t)g.nx);
    return g;
}

struct Pos {
    int iz, ix, iy;
    float oz, ox, oy;
};

__device__ __forceinline__ void decode(const GridP& g, int cell, int& izg, int& ix, int& iy) {
    uint32_t r = fdiv((uint32_t)cell, g.div_nzg);
    izg = cell - (int)r * g.nzg;
    uint32_t q = fdiv(r, g.div_nx);
    ix = (int)r - (int)q * g.nx;
    iy = (int)q;
}

__device__ __forceinline__ int encode(const GridP& g, int iz, int ix, int iy) {
    return (iz + 1) + g.nzg * (ix + g.nx * iy);
}

// ---------------------------------------------------------------- gather ----
// sum_a,b(,c) Wz[a] Wx[b] (Wy[c]) F[row(b, c) + bz + a]; rows are precomputed z-row offsets
template <int NDIM, int SHAPE>
__device__ __forceinline__ float interp(const GridP& g, const float* __restrict__ F, int bz, const float* Wz,
                                        const int* rows, const float* Wx, const float* Wy) {
    constexpr int K = Shape<SHAPE>::K;
    float acc = 0.f;
#pragma unroll
    for (int c = 0; c < (NDIM == 3 ? K : 1); ++c) {
        float wy = NDIM == 3 ? Wy[c] : 1.f;
#pragma unroll
        for (int b = 0; b < K; ++b) {
            const float* row = F + rows[c * K + b];
            float racc = 0.f;
#pragma unroll
            for (int a = 0; a < K; ++a) {
                int gz = bz + a;
                if ((unsigned)gz < (unsigned)g.nz) racc += Wz[a] * __ldg(row + gz);
            }
            acc += (wy * Wx[b]) * racc;
        }
    }
    return acc;
}

// z-row offsets of the K (x K) rows a stencil starting at (bx, by) touches
template <int NDIM, int K>
__device__ __forceinline__ void row_offsets(const GridP& g, int bx, int by, int* rows) {
#pragma unroll
    for (int c = 0; c < (NDIM == 3 ? K : 1); ++c) {
        int yy = NDIM == 3 ? wrapi(by + c, g.ny) * g.nx : 0;
#pragma unroll
        for (int b = 0; b < K; ++b) rows[c * K + b] = (yy + wrapi(bx + b, g.nx)) * g.nz;
    }
}

// E1..E3, B1..B3 at the particle (staggering: E1 z+, E2 x+, E3 y+ (3D) / node (2D),
// B1 x+ y+, B2 z+ y+, B3 z+ x+; "+" = half cell).
template <int NDIM, int SHAPE>
__device__ __forceinline__ void gather(const GridP& g, const float* __restrict__ E,
                                       const float* __restrict__ B, const Pos& p, float* eb) {
    constexpr int K = Shape<SHAPE>::K;
    constexpr int R = NDIM == 3 ? K * K : K;
    float Wzn[K], Wzh[K], Wxn[K], Wxh[K], Wyn[K], Wyh[K];
    int bzn = p.iz + Shape<SHAPE>::w(p.oz, Wzn);
    int bzh = half_weights<SHAPE>(p.iz, p.oz, Wzh);
    int bxn = p.ix + Shape<SHAPE>::w(p.ox, Wxn);
    int bxh = half_weights<SHAPE>(p.ix, p.ox, Wxh);
    int byn = 0, byh = 0;
    if (NDIM == 3) {
        byn = p.iy + Shape<SHAPE>::w(p.oy, Wyn);
        byh = half_weights<SHAPE>(p.iy, p.oy, Wyh);
    }
    const int N = (int)g.ncell;
    int rnn[R], rhn[R];            // x node / x half rows, y node
    row_offsets<NDIM, K>(g, bxn, byn, rnn);
    row_offsets<NDIM, K>(g, bxh, byn, rhn);
    eb[0] = interp<NDIM, SHAPE>(g, E, bzh, Wzh, rnn, Wxn, Wyn);
    eb[1] = interp<NDIM, SHAPE>(g, E + N, bzn, Wzn, rhn, Wxh, Wyn);
    eb[5] = interp<NDIM, SHAPE>(g, B + 2 * N, bzh, Wzh, rhn, Wxh, Wyn);
    if (NDIM == 3) {
        int rnh[R], rhh[R];        // y half rows
        row_offsets<NDIM, K>(g, bxn, byh, rnh);
        row_offsets<NDIM, K>(g, bxh, byh, rhh);
        eb[2] = interp<NDIM, SHAPE>(g, E + 2 * N, bzn, Wzn, rnh, Wxn, Wyh);
        eb[3] = interp<NDIM, SHAPE>(g, B, bzn, Wzn, rhh, Wxh, Wyh);
        eb[4] = interp<NDIM, SHAPE>(g, B + N, bzh, Wzh, rnh, Wxn, Wyh);
    } else {
        eb[2] = interp<NDIM, SHAPE>(g, E + 2 * N, bzn, Wzn, rnn, Wxn, Wyn);
        eb[3] = interp<NDIM, SHAPE>(g, B, bzn, Wzn, rhn, Wxh, Wyn);
        eb[4] = interp<NDIM, SHAPE>(g, B + N, bzh, Wzh, rnn, Wxn, Wyn);
    }
}

// ---------------------------------------------------------------- push ----
// The rotation factors use the approximate reciprocal square root and divide (a few ulp); the
// momentum they produce is still within FP32 round-off of the exact rotation, while positions
// take their accuracy from the float-float displacement below.
__device__ __forceinline__ void boris(float eps, const float* eb, float* u) {
    float um0 = u[0] + eps * eb[0], um1 = u[1] + eps * eb[1], um2 = u[2] + eps * eb[2];
    float f = eps * rsqrtf(1.f + um0 * um0 + um1 * um1 + um2 * um2);     // eps / gamma^-
    float t0 = f * eb[3], t1 = f * eb[4], t2 = f * eb[5];
    float tt = t0 * t0 + t1 * t1 + t2 * t2;
    float sf = __fdividef(2.f, 1.f + tt);
    float s0 = sf * t0, s1 = sf * t1, s2 = sf * t2;
    float up0 = um0 + (um1 * t2 - um2 * t1);
    float up1 = um1 + (um2 * t0 - um0 * t2);
    float up2 = um2 + (um0 * t1 - um1 * t0);
    float ul0 = um0 + (up1 * s2 - up2 * s1);
    float ul1 = um1 + (up2 * s0 - up0 * s2);
    float ul2 = um2 + (up0 * s1 - up1 * s0);
    u[0] = ul0 + eps * eb[0];
    u[1] = ul1 + eps * eb[1];
    u[2] = ul2 + eps * eb[2];
}

// Error-free transforms (Knuth TwoSum, FMA TwoProd) for float-float arithmetic.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = a * b;
    e = fmaf(a, b, -p);
}

// gamma = sqrt(1 + |u|^2) as an unevaluated float-float sum gh + gl; rg ~ 1/gh (approximate:
// every use below corrects or tolerates its few-ulp error).
__device__ __forceinline__ void gamma_ff(const float* u, float& gh, float& gl, float& rg) {
    float sh = 1.f, sl = 0.f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float ph, pl, t, e;
        two_prod(u[d], u[d], ph, pl);
        two_sum(sh, ph, t, e);
        sh = t;
        sl += e + pl;
    }
    float t = sh + sl;
    sl = sl - (t - sh);
    sh = t;
    gh = sqrtf(sh);
    rg = __fdividef(1.f, gh);
    gl = (fmaf(-gh, gh, sh) + sl) * (0.5f * rg);
}

// Displacement u_a dt / (gamma h_a) in cells as dh + dl (k = dt/h_a given as kh + kl).  Computed
// to ~1e-13 relative so that the per-step FP32 rounding of the offset is the only error left:
// rounding to nearest of o + (dh + dl) is unbiased, while a once-rounded FP32 increment would
// drift by the same fraction of an ulp every step.
__device__ __forceinline__ void displacement(float ua, float gh, float gl, float rg, float kh, float kl, float& dh,
                                             float& dl) {
    // the exact FMA residual ua - qh gh corrects whatever rounding qh = ua rg carries
    float qh = ua * rg;
    float ql = (fmaf(-qh, gh, ua) - qh * gl) * rg;
    dh = qh * kh;
    dl = fmaf(qh, kh, -dh) + (qh * kl + ql * kh);
}

// o + (dh + dl) -> new cell and offset in [0, 1), with one rounding of the exact sum.
__device__ __forceinline__ void advance_axis(int& i, float& o, float dh, float dl) {
    float s, e;
    two_sum(o, dh, s, e);
    float t = s + (e + dl);
    float fl = floorf(t);
    float r, re;
    two_sum(s, -fl, r, re);                   // exact: fl is an integer near s
    t = r + (e + dl + re);
    int di = (int)fl;
    if (t < 0.f) {                            // the rounded sum sat within round-off of fl
        t += 1.f;
        di -= 1;
    }
    if (t >= 1.f) {
        t -= 1.f;
        di += 1;
    }
    i += di;
    o = t;
}

// ---------------------------------------------------------------- deposit ----
// Current accumulators: add(component, node z, node x, node y, value) with x, y not yet wrapped.
struct GlobalAcc {
    const GridP* g;
    float* J;
    __device__ __forceinline__ void add(int c, int gz, int gx, int gy, float v) const {
        if (gz < 0 || gz >= g->nz) return;
        int o = (wrapi(gy, g->ny) * g->nx + wrapi(gx, g->nx)) * g->nz + gz;
        atomicAdd(J + c * (int)g->ncell + o, v);
    }
};
// Old-position weights w0 (first node b0) and the new position (i1, o1) -> the deposition
// window: S0 = old weights and DS = new - old, both placed in the K + 1 nodes from the lower
// of the two supports (returned).
template <int SHAPE>
__device__ __forceinline__ int axis_weights_from(int b0, const float* w0, int i1, float o1, float* S0, float* DS) {
    constexpr int K = Shape<SHAPE>::K;
    constexpr int KW = K + 1;
    float w1[K];
    const int b1 = i1 + Shape<SHAPE>::w(o1, w1);
    const bool sh0 = b0 > b1, sh1 = b1 > b0;
#pragma unroll
    for (int k = 0; k < KW; ++k) {
        const float a0 = k < K ? w0[k] : 0.f, a1 = k >= 1 ? w0[k - 1] : 0.f;
        const float c0 = k < K ? w1[k] : 0.f, c1 = k >= 1 ? w1[k - 1] : 0.f;
        const float a = sh0 ? a1 : a0;
        const float c = sh1 ? c1 : c0;
        S0[k] = a;
        DS[k] = c - a;
    }
    return min(b0, b1);
}

template <int SHAPE>
__device__ __forceinline__ int axis_weights(int i0, float o0, int i1, float o1, float* S0, float* DS) {
    constexpr int K = Shape<SHAPE>::K;
    constexpr int KW = K + 1;
    float w0[K], w1[K];
    const int b0 = i0 + Shape<SHAPE>::w(o0, w0);
    const int b1 = i1 + Shape<SHAPE>::w(o1, w1);
    // the supports start at most one node apart: place each at offset 0 or 1 of the window
    const bool sh0 = b0 > b1, sh1 = b1 > b0;
#pragma unroll
    for (int k = 0; k < KW; ++k) {
        const float a0 = k < K ? w0[k] : 0.f, a1 = k >= 1 ? w0[k - 1] : 0.f;
        const float c0 = k < K ? w1[k] : 0.f, c1 = k >= 1 ? w1[k - 1] : 0.f;
        const float a = sh0 ? a1 : a0;
        const float c = sh1 ? c1 : c0;
        S0[k] = a;
        DS[k] = c - a;
    }
    return min(b0, b1);
}

// Esirkepov current of one particle moving p0 -> p1 (|displacement| < 1 cell per axis).
// 2D: W1 = dSz (S0x + dSx/2), W2 = dSx (S0z + dSz/2), W3 = S0z S0x + dSz S0x/2 + S0z dSx/2 + dSz dSx/3.
// 3D: W_a = dS_a (S0_b S0_c + dS_b S0_c/2 + S0_b dS_c/2 + dS_b dS_c/3).
// J_a = -(q w/V)(h_a/dt) cumsum_a W_a; 2D J3 = (q w/V) v3 W3.
template <int NDIM, int SHAPE, typename Acc>
__device__ __forceinline__ void deposit(const GridP& g, float qv, float v3, const Pos& p0, const Pos& p1,
                                        const Acc& acc) {
    constexpr int KW = Shape<SHAPE>::K + 1;
    float S0z[KW], DSz[KW], S0x[KW], DSx[KW], S0y[KW], DSy[KW];
    const int bz = axis_weights<SHAPE>(p0.iz, p0.oz, p1.iz, p1.oz, S0z, DSz);
    const int bx = axis_weights<SHAPE>(p0.ix, p0.ox, p1.ix, p1.ox, S0x, DSx);
    const int by = NDIM == 3 ? axis_weights<SHAPE>(p0.iy, p0.oy, p1.iy, p1.oy, S0y, DSy) : 0;
    const float f1 = -qv * g.dz / g.dt, f2 = -qv * g.dx / g.dt;
    if (NDIM == 2) {
#pragma unroll
        for (int b = 0; b < KW; ++b) {           // J1: cumulative along z
            float tx = S0x[b] + 0.5f * DSx[b];
            float cum = 0.f;
#pragma unroll
            for (int a = 0; a < KW - 1; ++a) {
                cum += DSz[a] * tx;
                if (cum != 0.f) acc.add(0, bz + a, bx + b, 0, f1 * cum);
            }
        }
#pragma unroll
        for (int a = 0; a < KW; ++a) {           // J2: cumulative along x; J3
            float tz = S0z[a] + 0.5f * DSz[a];
            float cum = 0.f;
#pragma unroll
            for (int b = 0; b < KW; ++b) {
                if (b < KW - 1) {
                    cum += DSx[b] * tz;
                    if (cum != 0.f) acc.add(1, bz + a, bx + b, 0, f2 * cum);
                }
                float w3 = S0z[a] * S0x[b] + 0.5f * DSz[a] * S0x[b] + 0.5f * S0z[a] * DSx[b]
                         + (1.f / 3.f) * DSz[a] * DSx[b];
                if (w3 != 0.f) acc.add(2, bz + a, bx + b, 0, qv * v3 * w3);
            }
        }
    } else {
        const float f3 = -qv * g.dy / g.dt;
#pragma unroll
        for (int c = 0; c < KW; ++c)
#pragma unroll
            for (int b = 0; b < KW; ++b) {       // J1 along z
                float t = S0x[b] * S0y[c] + 0.5f * DSx[b] * S0y[c] + 0.5f * S0x[b] * DSy[c]
                        + (1.f / 3.f) * DSx[b] * DSy[c];
                float cum = 0.f;
#pragma unroll
                for (int a = 0; a < KW - 1; ++a) {
                    cum += DSz[a] * t;
                    if (cum != 0.f) acc.add(0, bz + a, bx + b, by + c, f1 * cum);
                }
            }
#pragma unroll
        for (int a = 0; a < KW; ++a) {
#pragma unroll
            for (int c = 0; c < KW; ++c) {       // J2 along x
                float t = S0z[a] * S0y[c] + 0.5f * DSz[a] * S0y[c] + 0.5f * S0z[a] * DSy[c]
                        + (1.f / 3.f) * DSz[a] * DSy[c];
                float cum = 0.f;
#pragma unroll
                for (int b = 0; b < KW - 1; ++b) {
                    cum += DSx[b] * t;
                    if (cum != 0.f) acc.add(1, bz + a, bx + b, by + c, f2 * cum);
                }
            }
#pragma unroll
            for (int b = 0; b < KW; ++b) {       // J3 along y
                float t = S0z[a] * S0x[b] + 0.5f * DSz[a] * S0x[b] + 0.5f * S0z[a] * DSx[b]
                        + (1.f / 3.f) * DSz[a] * DSx[b];
                float cum = 0.f;
#pragma unroll
                for (int c = 0; c < KW - 1; ++c) {
                    cum += DSy[c] * t;
                    if (cum != 0.f) acc.add(2, bz + a, bx + b, by + c, f3 * cum);
                }
            }
        }
    }
}

// ---------------------------------------------------------------- kernels ----
enum { MODE_FUSED = 0, MODE_PUSH_ONLY = 1 };

// Gather, Boris, move one particle and store its new state.  Returns false for an empty,
// retired or out-of-window slot.  p0/p1: old and new positions (p1.ix, p1.iy unwrapped).
template <int NDIM, int SHAPE, int MODE>
__device__ __forceinline__ bool advance_one(const GridP& g, const SpeciesP& sp, const float* __restrict__ E,
                                            const float* __restrict__ B, int shift, long long p, long long cap,
                                            Pos& p0, Pos& p1, float& v3) {
    int cell = sp.cell[p];
    if (cell < 0) {
        if (MODE == MODE_PUSH_ONLY) sp.prev_cell[p] = -1;
        return false;
    }
    int izg;
    decode(g, cell, izg, p0.ix, p0.iy);
    p0.iz = izg - 1 - shift;
    if (p0.iz < 0 || p0.iz >= g.nz) {      // left through the back of the window (or stale)
        sp.cell[p] = -1;
        if (MODE == MODE_PUSH_ONLY) sp.prev_cell[p] = -1;
        return false;
    }
    p0.oz = sp.off[p];
    p0.ox = sp.off[cap + p];
    p0.oy = NDIM == 3 ? sp.off[2 * cap + p] : 0.f;
    float u[3] = {sp.u[p], sp.u[cap + p], sp.u[2 * cap + p]};

    float eb[6];
    gather<NDIM, SHAPE>(g, E, B, p0, eb);
    boris(sp.eps, eb, u);

    float gh, gl, rg;
    gamma_ff(u, gh, gl, rg);
    float dzh, dzl, dxh, dxl, dyh = 0.f, dyl = 0.f;
    displacement(u[0], gh, gl, rg, sp.kz[0], sp.kz[1], dzh, dzl);
    displacement(u[1], gh, gl, rg, sp.kx[0], sp.kx[1], dxh, dxl);
    if (NDIM == 3) displacement(u[2], gh, gl, rg, sp.ky[0], sp.ky[1], dyh, dyl);
    // |v| < c and dt below the stability limit keep every move under one cell; anything else
    // (a non-finite field or momentum) retires the particle instead of indexing outside.
    if (!(fabsf(dzh) < 1.f && fabsf(dxh) < 1.f && fabsf(dyh) < 1.f)) {
        sp.cell[p] = -1;
        if (MODE == MODE_PUSH_ONLY) sp.prev_cell[p] = -1;
        return false;
    }
    p1 = p0;
    advance_axis(p1.iz, p1.oz, dzh, dzl);
    advance_axis(p1.ix, p1.ox, dxh, dxl);
    if (NDIM == 3) advance_axis(p1.iy, p1.oy, dyh, dyl);
    v3 = u[2] * rg;

    int wx = wrapi(p1.ix, g.nx);
    int wy = NDIM == 3 ? wrapi(p1.iy, g.ny) : 0;
    if (MODE == MODE_PUSH_ONLY) {
        sp.prev_cell[p] = encode(g, p0.iz, p0.ix, p0.iy);
        sp.prev_off[p] = p0.oz;
        sp.prev_off[cap + p] = p0.ox;
        if (NDIM == 3) sp.prev_off[2 * cap + p] = p0.oy;
        sp.cell[p] = encode(g, p1.iz, wx, wy);     // iz in [-1, nz]: guarded encoding
    } else {
        sp.cell[p] = (p1.iz >= 0 && p1.iz < g.nz) ? encode(g, p1.iz, wx, wy) : -1;
    }
    sp.off[p] = p1.oz;
    sp.off[cap + p] = p1.ox;
    if (NDIM == 3) sp.off[2 * cap + p] = p1.oy;
    sp.u[p] = u[0];
    sp.u[cap + p] = u[1];
    sp.u[2 * cap + p] = u[2];
    return true;
}

// Gather + push only; the old positions are kept for pic_deposit.
template <int NDIM, int SHAPE>
__global__ void __launch_bounds__(256) push_kernel(GridP g, SpeciesP sp, const float* __restrict__ E,
                                                   const float* __restrict__ B, int shift) {
    const long long n = *sp.count;
    const long long cap = sp.cap;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        Pos p0, p1;
        float v3;
        advance_one<NDIM, SHAPE, MODE_PUSH_ONLY>(g, sp, E, B, shift, p, cap, p0, p1, v3);
    }
}

// Particles per chunk of the fused kernels (one per thread).
constexpr int FUSED_T = 256;

// ---------------------------------------------------------------- 2D fused kernel ----
// Specialised 2D gather + push + Esirkepov for cell-sorted particles.  Per chunk of FUSED_T
// particles (one per thread):
//  1. the fields of the chunk's gather footprint are staged in shared memory (coalesced z rows,
//     zero outside the z range), so the 6 x K^2 interpolation loads are shared-memory loads;
//  2. the 2D Esirkepov weights are separable products of per-axis vectors:
//       J1(a,b) = f1 Cz[a] Tx[b],  J2(a,b) = f2 Tz[a] Cx[b],
//       J3(a,b) = qv v3 (S0z[a] (S0x[b] + dSx[b]/2) + dSz[a] (S0x[b]/2 + dSx[b]/3)),
//     with Cz = cumsum dSz, Tx = S0x + dSx/2 (and z <-> x);
//  3. the chunk's current is summed in a shared-memory box in 32-bit fixed point (native
//     integer atomics); when more than 8 lanes of a warp share a deposition window (dense
//     beams) runs of consecutive lanes are summed by a segmented warp reduction first, so that
//     one lane per run issues the atomic; the box is added to J with float4 atomics.
// Boxes larger than the shared-memory caps fall back to global loads / global atomics.
constexpr int F_CAP = 6 * 1024;    // field box floats (6 components)
constexpr int J_CAP = 3 * 1024;    // current box floats (3 components)
constexpr int SMEM_2D = F_CAP + J_CAP;

// 4-byte asynchronous global -> shared copy (the next chunk's particle data)
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
// 16- and 4-byte copies with zero fill (valid = false reads nothing and writes zeros): field
// groups of a staged box, cells outside 0 <= z < nz read as zero
__device__ __forceinline__ void cp_async16z(void* dst, const void* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async4z(void* dst, const void* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all_p() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// floor(i / d) for 0 <= i < 2^22 from r = 1/d rounded to nearest: (i + 1/2) r is within
// (i + 1/2) 2^-23 / d of (i + 1/2) / d, which lies at least 1/(2d) from an integer.
__device__ __forceinline__ int box_div(int i, float r) { return (int)(((float)i + 0.5f) * r); }

// Runs of consecutive lanes with the same deposition window (cell-sorted particles of a dense
// beam): a segmented warp sum lets only the first lane of each run add the run's total.
struct SegReduce {
    bool same[5];       // lane + 2^k belongs to the same run
    bool head;          // first lane of its run: adds the run's total
    int steps;          // warp-uniform: ceil(log2(longest run)), 0 when no lanes share a window
    __device__ __forceinline__ int sum(int v) const {
        int t;
        if (steps > 0) { t = __shfl_down_sync(0xffffffffu, v, 1);  if (same[0]) v += t; }
        if (steps > 1) { t = __shfl_down_sync(0xffffffffu, v, 2);  if (same[1]) v += t; }
        if (steps > 2) { t = __shfl_down_sync(0xffffffffu, v, 4);  if (same[2]) v += t; }
        if (steps > 3) { t = __shfl_down_sync(0xffffffffu, v, 8);  if (same[3]) v += t; }
        if (steps > 4) { t = __shfl_down_sync(0xffffffffu, v, 16); if (same[4]) v += t; }
        return v;
    }
};

__device__ __forceinline__ SegReduce make_segments(unsigned long long key) {
    const int lane = threadIdx.x & 31;
    unsigned long long prev = __shfl_up_sync(0xffffffffu, key, 1);
    SegReduce r;
    r.head = lane == 0 || prev != key;
    const unsigned heads = __ballot_sync(0xffffffffu, r.head);
    // run length of a head: distance to the next head (or to the end of the warp)
    const unsigned above = lane < 31 ? (heads >> (lane + 1)) : 0u;
    const int len = r.head ? (above ? __ffs(above) : 32 - lane) : 0;
    const int maxlen = __reduce_max_sync(0xffffffffu, len);
    r.steps = maxlen <= 1 ? 0 : 32 - __clz(maxlen - 1);
    const int run = __popc(heads & (0xffffffffu >> (31 - lane)));     // heads at or below this lane
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        int o = 1 << k;
        int other = __shfl_down_sync(0xffffffffu, run, o);
        r.same[k] = lane + o < 32 && other == run;
    }
    return r;
}

// block-wide min/max of lo/hi (two axes) into box[4]; all threads call
__device__ __forceinline__ void box_reduce(int* box, int lz, int hz, int lx, int hx) {
    const int lane = threadIdx.x & 31;
    int a = __reduce_min_sync(0xffffffffu, lz), b = __reduce_max_sync(0xffffffffu, hz);
    int c = __reduce_min_sync(0xffffffffu, lx), d = __reduce_max_sync(0xffffffffu, hx);
    if (lane == 0 && a != INT_MAX) {
        atomicMin(box + 0, a);
        atomicMax(box + 1, b);
        atomicMin(box + 2, c);
        atomicMax(box + 3, d);
    }
}

// Field box of a chunk, rows of fzl (a multiple of 4) floats along z, fvol = fxl fzl nodes:
//   P1[fvol] float2 = (E1, B2): half cell along z, node along x  -> weights (Wzh, Wxn)
//   P2[fvol] float2 = (E2, B1): node along z, half cell along x  -> weights (Wzn, Wxh)
//   S3[fvol] = E3 (node, node),  T3[fvol] = B3 (half, half)
// Components that share a stencil are interpolated together with packed FP32 FMAs.
template <int K>
__device__ __forceinline__ float2 tile_interp2(const float2* __restrict__ f, int zl, int z, int x, const float (&Wz)[K],
                                               const float (&Wx)[K]) {
    const float2* r = f + x * zl + z;
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int b = 0; b < K; ++b) {
        float2 t = make_float2(0.f, 0.f);
#pragma unroll
        for (int a = 0; a < K; ++a) t = __ffma2_rn(make_float2(Wz[a], Wz[a]), r[a], t);
        acc = __ffma2_rn(make_float2(Wx[b], Wx[b]), t, acc);
        r += zl;
    }
    return acc;
}

// E3 and B3 (different stencils) as one packed chain: .x = E3, .y = B3.
template <int K>
__device__ __forceinline__ float2 tile_interp_e3b3(const float* __restrict__ S3, const float* __restrict__ T3, int zl,
                                                   int za, int xa, int zb, int xb, const float (&Wza)[K],
                                                   const float (&Wxa)[K], const float (&Wzb)[K],
                                                   const float (&Wxb)[K]) {
    const float* r = S3 + xa * zl + za;
    const float* q = T3 + xb * zl + zb;
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int b = 0; b < K; ++b) {
        float2 t = make_float2(0.f, 0.f);
#pragma unroll
        for (int a = 0; a < K; ++a) t = __ffma2_rn(make_float2(Wza[a], Wzb[a]), make_float2(r[a], q[a]), t);
        acc = __ffma2_rn(make_float2(Wxa[b], Wxb[b]), t, acc);
        r += zl;
        q += zl;
    }
    return acc;
}

// Cells gz..gz+3 of a field row into a (zero outside 0 <= z < nz); vec: 16-byte groups.
__device__ __forceinline__ float4 load_group(const float* __restrict__ row, int gz, int nz, bool vec) {
    if (vec && gz >= 0 && gz + 3 < nz) return __ldg(reinterpret_cast<const float4*>(row + gz));
    float4 a;
    a.x = (unsigned)gz < (unsigned)nz ? __ldg(row + gz) : 0.f;
    a.y = (unsigned)(gz + 1) < (unsigned)nz ? __ldg(row + gz + 1) : 0.f;
    a.z = (unsigned)(gz + 2) < (unsigned)nz ? __ldg(row + gz + 2) : 0.f;
    a.w = (unsigned)(gz + 3) < (unsigned)nz ? __ldg(row + gz + 3) : 0.f;
    return a;
}

__device__ __forceinline__ bool aligned16(const void* q) { return ((uintptr_t)q & 15) == 0; }

template <int SHAPE>
__device__ __forceinline__ void push_deposit_2d_chunks(const GridP& g, const SpeciesP& sp,
                                                       const float* __restrict__ E, const float* __restrict__ B,
                                                       float* __restrict__ J, int shift, long long chunk0,
                                                       long long stride, float* sF, float* sJ, int* box) {
    constexpr int K = Shape<SHAPE>::K;
    constexpr int KW = K + 1;
    const long long n = *sp.count;
    const long long cap = sp.cap;
    const int N = (int)g.ncell;
    const bool fvec = (g.nz & 3) == 0 && aligned16(E) && aligned16(B);
    const bool jvec = (g.nz & 3) == 0 && aligned16(J);
    for (long long base = chunk0 * FUSED_T; base < n; base += stride * FUSED_T) {
        if (threadIdx.x < 5) box[threadIdx.x] = threadIdx.x == 4 ? 0 : (threadIdx.x & 1) ? INT_MIN : INT_MAX;
        __syncthreads();
        const long long p = base + threadIdx.x;
        // ---- load and decode ----
        bool ok = false;
        Pos p0;
        float u[3] = {0.f, 0.f, 0.f};
        if (p < n) {
            int cell = sp.cell[p];
            if (cell >= 0) {
                int izg;
                decode(g, cell, izg, p0.ix, p0.iy);
                p0.iz = izg - 1 - shift;
                if (p0.iz >= 0 && p0.iz < g.nz) {
                    ok = true;
                    p0.oz = sp.off[p];
                    p0.ox = sp.off[cap + p];
                    p0.oy = 0.f;
                    u[0] = sp.u[p];
                    u[1] = sp.u[cap + p];
                    u[2] = sp.u[2 * cap + p];
                } else {
                    sp.cell[p] = -1;
                }
            }
        }
        // ---- gather weights and the chunk's boxes ----
        float Wzn[K], Wzh[K], Wxn[K], Wxh[K];
        int bzn = 0, bzh = 0, bxn = 0, bxh = 0;
        if (ok) {
            bzn = p0.iz + Shape<SHAPE>::w(p0.oz, Wzn);
            bzh = half_weights<SHAPE>(p0.iz, p0.oz, Wzh);
            bxn = p0.ix + Shape<SHAPE>::w(p0.ox, Wxn);
            bxh = half_weights<SHAPE>(p0.ix, p0.ox, Wxh);
        }
        box_reduce(box, ok ? min(bzn, bzh) : INT_MAX, ok ? max(bzn, bzh) + K - 1 : INT_MIN,
                   ok ? min(bxn, bxh) : INT_MAX, ok ? max(bxn, bxh) + K - 1 : INT_MIN);
        __syncthreads();
        const bool any = box[0] != INT_MAX;
        // field box: z aligned down to a multiple of 4, rows padded to whole groups
        const int fz0 = any ? (box[0] & ~3) : 0, fx0 = box[2];
        const int fzl = any ? ((box[1] + 1 - fz0 + 3) & ~3) : 0, fxl = any ? box[3] - box[2] + 1 : 0;
        const int fvol = fzl * fxl;
        const bool ftile = any && 6 * fvol <= F_CAP && fxl <= g.nx + 2 * K;
        // current box: every deposition window lies within one node below and two above the
        // gather stencils (the move is under one cell per axis)
        const int jz0 = any ? ((box[0] - 1) & ~3) : 0, jx0 = box[2] - 1;
        const int jzl = any ? ((box[1] + 3 - jz0 + 3) & ~3) : 0, jxl = any ? box[3] - box[2] + 4 : 0;
        const int jvol = jzl * jxl;
        const bool jtile = any && 3 * jvol <= J_CAP && jxl <= g.nx + 2 * KW;
        float2* P1 = reinterpret_cast<float2*>(sF);
        float2* P2 = P1 + fvol;
        float* S3 = sF + 4 * fvol;
        float* T3 = S3 + fvol;
        if (ftile) {
            const int ng = fzl >> 2;
            const float rg = 1.f / (float)ng, rx = 1.f / (float)fxl;
            for (int i = threadIdx.x; i < 3 * fxl * ng; i += FUSED_T) {
                const int r = box_div(i, rg), zg = i - r * ng;
                const int pc = box_div(r, rx), x = r - pc * fxl;
                const long long row = (long long)wrapi(fx0 + x, g.nx) * g.nz;
                const int gz = fz0 + 4 * zg;
                const int o = x * fzl + 4 * zg;
                // pc = 0: (E1, B2), 1: (E2, B1), 2: E3, B3
                const float* fa = E + pc * N + row;
                const float* fb = B + (pc == 0 ? N : pc == 1 ? 0 : 2 * N) + row;
                const float4 a = load_group(fa, gz, g.nz, fvec), b = load_group(fb, gz, g.nz, fvec);
                if (pc < 2) {
                    float4* d = reinterpret_cast<float4*>((pc == 0 ? P1 : P2) + o);
                    d[0] = make_float4(a.x, b.x, a.y, b.y);
                    d[1] = make_float4(a.z, b.z, a.w, b.w);
                } else {
                    *reinterpret_cast<float4*>(S3 + o) = a;
                    *reinterpret_cast<float4*>(T3 + o) = b;
                }
            }
        }
        if (jtile)
            for (int i = threadIdx.x; i < (3 * jvol) >> 2; i += FUSED_T)
                reinterpret_cast<float4*>(sJ)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();
        // ---- gather (staggering: E1 z+, E2 x+, E3 node, B1 x+, B2 z+, B3 z+ x+) ----
        float eb[6];
        if (ok) {
            if (ftile) {
                const float2 q1 = tile_interp2<K>(P1, fzl, bzh - fz0, bxn - fx0, Wzh, Wxn);
                const float2 q2 = tile_interp2<K>(P2, fzl, bzn - fz0, bxh - fx0, Wzn, Wxh);
                const float2 q3 = tile_interp_e3b3<K>(S3, T3, fzl, bzn - fz0, bxn - fx0, bzh - fz0, bxh - fx0, Wzn,
                                                      Wxn, Wzh, Wxh);
                eb[0] = q1.x;
                eb[4] = q1.y;
                eb[1] = q2.x;
                eb[3] = q2.y;
                eb[2] = q3.x;
                eb[5] = q3.y;
            } else {
                gather<2, SHAPE>(g, E, B, p0, eb);
            }
        }
        // ---- push and move ----
        Pos p1 = p0;
        float v3 = 0.f;
        if (ok) {
            boris(sp.eps, eb, u);
            float gh, gl, rg;
            gamma_ff(u, gh, gl, rg);
            float dzh, dzl, dxh, dxl;
            displacement(u[0], gh, gl, rg, sp.kz[0], sp.kz[1], dzh, dzl);
            displacement(u[1], gh, gl, rg, sp.kx[0], sp.kx[1], dxh, dxl);
            if (!(fabsf(dzh) < 1.f && fabsf(dxh) < 1.f)) {
                ok = false;
                sp.cell[p] = -1;
            } else {
                advance_axis(p1.iz, p1.oz, dzh, dzl);
                advance_axis(p1.ix, p1.ox, dxh, dxl);
                v3 = u[2] * rg;
                const int wx = wrapi(p1.ix, g.nx);
                sp.cell[p] = (p1.iz >= 0 && p1.iz < g.nz) ? encode(g, p1.iz, wx, 0) : -1;
                sp.off[p] = p1.oz;
                sp.off[cap + p] = p1.ox;
                sp.u[p] = u[0];
                sp.u[cap + p] = u[1];
                sp.u[2 * cap + p] = u[2];
            }
        }
        // ---- deposition ----
        float S0z[KW], DSz[KW], S0x[KW], DSx[KW];
        int bz = 0, bx = 0;
        if (ok) {
            bz = axis_weights_from<SHAPE>(bzn, Wzn, p1.iz, p1.oz, S0z, DSz);
            bx = axis_weights_from<SHAPE>(bxn, Wxn, p1.ix, p1.ox, S0x, DSx);
        } else {
#pragma unroll
            for (int k = 0; k < KW; ++k) S0z[k] = DSz[k] = S0x[k] = DSx[k] = 0.f;
        }
        // J1(a,b) = Cz[a] Tx[b], J2(a,b) = Tz[a] Cx[b], J3(a,b) = S0z[a] Ax[b] + DSz[a] Bx[b] with
        // Cz = f1 cumsum dSz, Cx = f2 cumsum dSx, T = S0 + dS/2, Ax = f3 Tx, Bx = f3 (S0x/2 + dSx/3).
        const float f1 = -sp.qv * g.dz / g.dt, f2 = -sp.qv * g.dx / g.dt, f3 = sp.qv * v3;
        float cz[KW], cx[KW];
        float mb = fabsf(f3);         // bound of every contribution of this particle (below)
        {
            float az = 0.f, ax = 0.f;
#pragma unroll
            for (int k = 0; k < KW; ++k) {
                az += DSz[k];
                ax += DSx[k];
                cz[k] = az;
                cx[k] = ax;
                mb = fmaxf(mb, fmaxf(fabsf(f1 * az), fabsf(f2 * ax)));
            }
        }
        // The shared current box accumulates in 32-bit fixed point: integer shared atomics are
        // single instructions, where FP32 ones retry on every conflicting lane, and integer sums
        // reduce across a warp in one instruction.  Tz, Tx and the 2D J3 weight
        // (S0z S0x + S1z S1x)/3 + (S0z S1x + S1z S0x)/6 lie in [0, 1], so no contribution
        // exceeds mb = max(|Cz|, |Cx|, |f3|).  With 2^(e-1) <= max mb < 2^e over the chunk, the
        // scale s = 2^(22-e) keeps every scaled contribution (and each of the two products of
        // J3) below 2^22, where adding 1.5 2^23 rounds it to an integer in the low mantissa
        // bits, and every node sum of at most FUSED_T particles below 2^30.  The rounding step
        // is below 2^-21 of the chunk's largest contribution.
        if (jtile) {
            const unsigned wm = __reduce_max_sync(0xffffffffu, ok ? __float_as_uint(mb) : 0u);
            if ((threadIdx.x & 31) == 0 && wm) atomicMax(reinterpret_cast<unsigned*>(box + 4), wm);
        }
        __syncthreads();
        const int mbits = box[4];
        const int sexp = min(275 - (mbits >> 23), 253);       // biased exponent of s
        const float fs = __int_as_float(sexp << 23), inv_s = __int_as_float((254 - sexp) << 23);
        int* const iJ = reinterpret_cast<int*>(sJ);
        if (any && jtile && mbits != 0) {
            const float g1 = f1 * fs, g2 = f2 * fs, g3 = f3 * fs;
            float2 CT[KW], TC[KW];        // (s Cz, Tz)[a], (Tx, s Cx)[b]
            float Ax[KW], Bx[KW];         // s Ax, s Bx
#pragma unroll
            for (int k = 0; k < KW; ++k) {
                CT[k] = make_float2(g1 * cz[k], S0z[k] + 0.5f * DSz[k]);
                const float tx = S0x[k] + 0.5f * DSx[k];
                TC[k] = make_float2(tx, g2 * cx[k]);
                Ax[k] = g3 * tx;
                Bx[k] = g3 * (0.5f * S0x[k] + (1.f / 3.f) * DSx[k]);
            }
            // Lanes sharing a window hit the same nodes.  With at most 8 lanes per window anywhere
            // in the warp every live lane adds its own values (at most 8-way address conflicts,
            // serialised by the shared-memory pipe); otherwise (dense beams) runs of consecutive
            // lanes are summed first and one lane per run adds the total.  Empty slots have unique
            // keys.
            const unsigned long long key = ok ? (((unsigned long long)(bz + 4) << 32) | (unsigned)(bx + 4))
                                              : (0xFFFFFFFF00000000ull | (unsigned)threadIdx.x);
            const int gmax = __reduce_max_sync(0xffffffffu, __popc(__match_any_sync(0xffffffffu, key)));
            int* s0 = iJ + (bx - jx0) * jzl + (bz - jz0);
            const float MAGIC = 12582912.f;           // 1.5 2^23
            // no lane of the warp changed its support node along an axis: the last window node along
            // it has S0 = dS = 0 and the last cumulative sum along it is zero; skip those deposits
            const bool uz = __any_sync(0xffffffffu, S0z[KW - 1] != 0.f || DSz[KW - 1] != 0.f);
            const bool ux = __any_sync(0xffffffffu, S0x[KW - 1] != 0.f || DSx[KW - 1] != 0.f);
            auto terms = [&](auto&& put) {
#pragma unroll
                for (int b = 0; b < KW; ++b)
#pragma unroll
                    for (int a = 0; a < KW; ++a) {
                        // J1 (a < KW-1): zero at the last cumulative z sum or the last x node;
                        // J2 (b < KW-1): at the last cumulative x sum or the last z node;
                        // J3: at the last z node or the last x node
                        const bool k1 = !((a == KW - 2 && !uz) || (b == KW - 1 && !ux));
                        const bool k2 = !((b == KW - 2 && !ux) || (a == KW - 1 && !uz));
                        const bool k3 = !((a == KW - 1 && !uz) || (b == KW - 1 && !ux));
                        const int o = b * jzl + a;
                        if (a < KW - 1 && b < KW - 1) {
                            if (k1 || k2) {
                                const float2 v = __ffma2_rn(CT[a], TC[b], make_float2(MAGIC, MAGIC));
                                if (k1) put(o, v.x);
                                if (k2) put(jvol + o, v.y);
                            }
                        } else if (a < KW - 1) {
                            if (k1) put(o, fmaf(CT[a].x, TC[b].x, MAGIC));
                        } else if (b < KW - 1) {
                            if (k2) put(jvol + o, fmaf(CT[a].y, TC[b].y, MAGIC));
                        }
                        if (k3) put(2 * jvol + o, fmaf(S0z[a], Ax[b], fmaf(DSz[a], Bx[b], MAGIC)));
                    }
            };
            if (gmax <= 8) {
                if (ok) terms([&](int o, float biased) { atomicAdd(s0 + o, __float_as_int(biased) - 0x4B400000); });
            } else {
                const SegReduce seg = make_segments(key);
                terms([&](int o, float biased) {
                    const int v = seg.sum(__float_as_int(biased) - 0x4B400000);
                    if (seg.head && ok && v != 0) atomicAdd(s0 + o, v);
                });
            }
        } else if (any && !jtile && ok) {
            // box too large for shared memory: FP32 atomics straight to J
#pragma unroll
            for (int b = 0; b < KW; ++b) {
                const int row = wrapi(bx + b, g.nx) * g.nz;
                const float tx = S0x[b] + 0.5f * DSx[b];
                const float ax = f3 * tx, bxv = f3 * (0.5f * S0x[b] + (1.f / 3.f) * DSx[b]);
#pragma unroll
                for (int a = 0; a < KW; ++a) {
                    const int gz = bz + a;
                    if ((unsigned)gz >= (unsigned)g.nz) continue;
                    float* d = J + row + gz;
                    float v;
                    if (a < KW - 1 && (v = f1 * cz[a] * tx) != 0.f) atomicAdd(d, v);
                    if (b < KW - 1 && (v = (S0z[a] + 0.5f * DSz[a]) * f2 * cx[b]) != 0.f) atomicAdd(d + N, v);
                    if ((v = fmaf(S0z[a], ax, DSz[a] * bxv)) != 0.f) atomicAdd(d + 2 * N, v);
                }
            }
        }
        __syncthreads();
        if (jtile && mbits != 0) {
            // box -> J in 16-byte groups (one vector atomic per group inside the grid)
            const int ng = jzl >> 2;
            const float rg = 1.f / (float)ng, rx = 1.f / (float)jxl;
            for (int i = threadIdx.x; i < 3 * jxl * ng; i += FUSED_T) {
                const int4 q = reinterpret_cast<const int4*>(iJ)[i];
                if ((q.x | q.y | q.z | q.w) == 0) continue;
                const float4 v = make_float4((float)q.x * inv_s, (float)q.y * inv_s, (float)q.z * inv_s,
                                             (float)q.w * inv_s);
                const int r = box_div(i, rg), zg = i - r * ng;
                const int c = box_div(r, rx), x = r - c * jxl;
                const int gz = jz0 + 4 * zg;
                float* dst = J + c * N + wrapi(jx0 + x, g.nx) * g.nz + gz;
                if (jvec && gz >= 0 && gz + 3 < g.nz) {
                    atomicAdd(reinterpret_cast<float4*>(dst), v);
                } else {
                    if ((unsigned)gz < (unsigned)g.nz && q.x) atomicAdd(dst, v.x);
                    if ((unsigned)(gz + 1) < (unsigned)g.nz && q.y) atomicAdd(dst + 1, v.y);
                    if ((unsigned)(gz + 2) < (unsigned)g.nz && q.z) atomicAdd(dst + 2, v.z);
                    if ((unsigned)(gz + 3) < (unsigned)g.nz && q.w) atomicAdd(dst + 3, v.w);
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- 3D fused kernel ----
// The 3D counterpart of push_deposit_2d_chunks: per chunk of FUSED_T cell-sorted particles the
// gather footprint is staged in shared memory, components are interpolated in pairs with packed
// FP32 FMAs, and the 3D Esirkepov current
//   J1(a,b,c) = Cz[a] Txy(b,c), J2(a,b,c) = Cx[b] Tzy(a,c), J3(a,b,c) = Cy[c] Tzx(a,b),
//   C_d = -(q w/V)(h_d/dt) cumsum dS_d,  T_uv = S0_u (S0_v + dS_v/2) + dS_u (S0_v/2 + dS_v/3)
// is accumulated in a 32-bit fixed-point box as in 2D (T_uv lies in [0, 1], so |C_d| bounds
// every contribution).
//
// Both shared-memory boxes have compile-time strides, so every interpolation load and every
// deposit address is a base register plus an immediate, and the staging index arithmetic uses
// constant divisors.  A chunk of 256 particles sorted in 4 x 4 x 4-cell tiles spans at most three
// tiles of a uniform 2-per-cell plasma (chunk and tile boundaries do not line up); three tiles
// along z, whatever their alignment to the 4-cell groups after window shifts, need at most 18 x 7 x 7
// field nodes and 21 x 10 x 10 current nodes.  A chunk whose boxes do not fit (a tile row ends
// inside it, sparse regions, particles injected since the last sort) takes the general path.  The current box is cleared once when the
// CTA starts and then by the flush that empties it, so a chunk does not clear it again.
// Field rows hold up to 20 z nodes, current rows up to 24: with row pitches of 20 and 24 words the
// cells of a sorted warp (4 along z, 4 along x) fall on distinct shared-memory banks (a pitch of
// 16 would put x and x + 2 on the same banks).
constexpr int FZ3 = 20, FZP3 = 20, FX3 = 8, FY3 = 8;     // field box per component: [y][x][z]
constexpr int FV3 = FZP3 * FX3 * FY3;
constexpr int JZ3 = 24, JZP3 = 24, JX3 = 10, JY3 = 10;   // current box per component: [y][x][z]
constexpr int JV3 = JZP3 * JX3 * JY3;
constexpr int PF3 = 7;                           // prefetched words per particle (cell, 3 offsets, 3 momenta)
constexpr int SMEM_3D = 6 * FV3 + 3 * JV3 + 2 * PF3 * FUSED_T;
static_assert((3 * JV3) % 4 == 0 && FZP3 % 4 == 0 && JZP3 % 4 == 0, "16-byte groups");

// i / d for the box extents d = 1..32 as (i m_d) >> 16 with m_d = ceil(2^16 / d): the product
// exceeds i / d by i e / (2^16 d), e = d m_d - 2^16 < d, which keeps it below the next integer
// (at least 1/d above i / d) while i e < 2^16, i.e. for every i < 2048 (checked below).
struct Inv16 {
    unsigned m[33];
};
constexpr Inv16 make_inv16() {
    Inv16 t{};
    for (int d = 1; d <= 32; ++d) t.m[d] = 65535u / (unsigned)d + 1u;
    return t;
}
constexpr bool inv16_exact() {
    const Inv16 t = make_inv16();
    for (unsigned d = 1; d <= 32; ++d)
        for (unsigned i = 0; i < 2048; ++i)
            if (((i * t.m[d]) >> 16) != i / d) return false;
    return true;
}
static_assert(inv16_exact(), "reciprocal division table");
__constant__ Inv16 kInv16 = make_inv16();
__device__ __forceinline__ int qdiv(int i, unsigned m) { return (int)(((unsigned)i * m) >> 16); }

// .x = sum Wza Wxa Wya Fa, .y = sum Wzb Wxb Wyb Fb over K^3 nodes of the fixed-stride field box;
// oa, ob: offsets of the two stencil origins.
template <int K>
__device__ __forceinline__ float2 tile_interp3_fixed(const float* __restrict__ Fa, const float (&Wza)[K],
                                                     const float (&Wxa)[K], const float (&Wya)[K],
                                                     const float* __restrict__ Fb, const float (&Wzb)[K],
                                                     const float (&Wxb)[K], const float (&Wyb)[K]) {
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int c = 0; c < K; ++c) {
        float2 tc = make_float2(0.f, 0.f);
#pragma unroll
        for (int b = 0; b < K; ++b) {
            const float* ra = Fa + (c * FX3 + b) * FZP3;
            const float* rb = Fb + (c * FX3 + b) * FZP3;
            float2 t = make_float2(0.f, 0.f);
#pragma unroll
            for (int a = 0; a < K; ++a) t = __ffma2_rn(make_float2(Wza[a], Wzb[a]), make_float2(ra[a], rb[a]), t);
            tc = __ffma2_rn(make_float2(Wxa[b], Wxb[b]), t, tc);
        }
        acc = __ffma2_rn(make_float2(Wya[c], Wyb[c]), tc, acc);
    }
    return acc;
}

constexpr int F_CAP3 = 10240;      // general path: field box floats (6 components)
constexpr int J_CAP3 = 11264;      // general path: current box ints (3 components)

// Global-memory gather and deposition for chunks whose boxes do not fit the shared-memory
// tiles.  Kept out of line: inlined, their registers would be reserved by the whole kernel.
template <int SHAPE>
__device__ __noinline__ void gather3_global(const GridP g, const float* __restrict__ E, const float* __restrict__ B,
                                            const Pos p0, float* eb) {
    gather<3, SHAPE>(g, E, B, p0, eb);
}
template <int SHAPE>
__device__ __noinline__ void deposit3_global(const GridP g, float qv, const Pos p0, const Pos p1, float* J) {
    GlobalAcc acc{&g, J};
    deposit<3, SHAPE>(g, qv, 0.f, p0, p1, acc);
}

// DEFER: a chunk whose boxes do not fit is appended to defer[2..] (count in defer[0]) for the
// general kernel, or to defer2[2..] for the per-particle kernel when even the general path's boxes
// would not hold it; without DEFER it takes the out-of-line global-memory path here.
template <int SHAPE, bool DEFER>
__device__ __forceinline__ void push_deposit_3d_chunks(const GridP& g, const SpeciesP& sp,
                                                       const float* __restrict__ E, const float* __restrict__ B,
                                                       float* __restrict__ J, int shift, long long chunk0,
                                                       long long stride, float* sF, float* sJ, int* box,
                                                       int* __restrict__ defer, int* __restrict__ defer2) {
    constexpr int K = Shape<SHAPE>::K;
    constexpr int KW = K + 1;
    const long long n = *sp.count;
    const long long cap = sp.cap;
    const int N = (int)g.ncell;
    const bool fvec = (g.nz & 3) == 0 && aligned16(E) && aligned16(B);
    const bool jvec = (g.nz & 3) == 0 && aligned16(J);
    int* const iJ = reinterpret_cast<int*>(sJ);
    float* const pfb = sJ + 3 * JV3;                  // [2][PF3][FUSED_T]
    auto prefetch = [&](long long b, int buf) {
        const long long q = b + threadIdx.x;
        if (q < n) {
            float* d = pfb + buf * PF3 * FUSED_T + threadIdx.x;
            cp_async4(d, sp.cell + q);
            cp_async4(d + FUSED_T, sp.off + q);
            cp_async4(d + 2 * FUSED_T, sp.off + cap + q);
            cp_async4(d + 3 * FUSED_T, sp.off + 2 * cap + q);
            cp_async4(d + 4 * FUSED_T, sp.u + q);
            cp_async4(d + 5 * FUSED_T, sp.u + cap + q);
            cp_async4(d + 6 * FUSED_T, sp.u + 2 * cap + q);
        }
        cp_async_commit();
    };
    int buf = 0;
    prefetch(chunk0 * FUSED_T, 0);
    // box[0..6] and box[7..13] serve alternate chunks: no barrier at the top of the loop or after
    // the flush.  The current box starts cleared.
    if (threadIdx.x < 14) {
        const int q = threadIdx.x % 7;
        box[threadIdx.x] = q == 6 ? 0 : (q & 1) ? INT_MIN : INT_MAX;
    }
    for (int i = threadIdx.x; i < (3 * JV3) / 4; i += FUSED_T)
        reinterpret_cast<int4*>(iJ)[i] = make_int4(0, 0, 0, 0);
    __syncthreads();
    int cur = 0;
    for (long long base = chunk0 * FUSED_T; base < n; base += stride * FUSED_T, buf ^= 1, cur ^= 7) {
        int* const bc = box + cur;
        if (threadIdx.x < 7) box[(cur ^ 7) + threadIdx.x] = threadIdx.x == 6 ? 0 : (threadIdx.x & 1) ? INT_MIN : INT_MAX;
        prefetch(base + stride * FUSED_T, buf ^ 1);
        cp_async_wait_prev();                      // this thread's words of this chunk
        const long long p = base + threadIdx.x;
        const float* mine = pfb + buf * PF3 * FUSED_T + threadIdx.x;
        // ---- load and decode ----
        bool ok = false;
        Pos p0;
        float u[3] = {0.f, 0.f, 0.f};
        if (p < n) {
            int cell = __float_as_int(mine[0]);
            if (cell >= 0) {
                int izg;
                decode(g, cell, izg, p0.ix, p0.iy);
                p0.iz = izg - 1 - shift;
                if (p0.iz >= 0 && p0.iz < g.nz) {
                    ok = true;
                    p0.oz = mine[FUSED_T];
                    p0.ox = mine[2 * FUSED_T];
                    p0.oy = mine[3 * FUSED_T];
                    u[0] = mine[4 * FUSED_T];
                    u[1] = mine[5 * FUSED_T];
                    u[2] = mine[6 * FUSED_T];
                } else {
                    sp.cell[p] = -1;
                }
            }
        }
        // ---- gather weights and the chunk's boxes ----
        float Wzn[K], Wzh[K], Wxn[K], Wxh[K], Wyn[K], Wyh[K];
        int bzn = 0, bzh = 0, bxn = 0, bxh = 0, byn = 0, byh = 0;
        if (ok) {
            bzn = p0.iz + Shape<SHAPE>::w(p0.oz, Wzn);
            bzh = half_weights<SHAPE>(p0.iz, p0.oz, Wzh);
            bxn = p0.ix + Shape<SHAPE>::w(p0.ox, Wxn);
            bxh = half_weights<SHAPE>(p0.ix, p0.ox, Wxh);
            byn = p0.iy + Shape<SHAPE>::w(p0.oy, Wyn);
            byh = half_weights<SHAPE>(p0.iy, p0.oy, Wyh);
        }
        box_reduce(bc, ok ? min(bzn, bzh) : INT_MAX, ok ? max(bzn, bzh) + K - 1 : INT_MIN,
                   ok ? min(bxn, bxh) : INT_MAX, ok ? max(bxn, bxh) + K - 1 : INT_MIN);
        {
            const int c = __reduce_min_sync(0xffffffffu, ok ? min(byn, byh) : INT_MAX);
            const int d = __reduce_max_sync(0xffffffffu, ok ? max(byn, byh) + K - 1 : INT_MIN);
            if ((threadIdx.x & 31) == 0 && c != INT_MAX) {
                atomicMin(bc + 4, c);
                atomicMax(bc + 5, d);
            }
        }
        __syncthreads();
        const bool any = bc[0] != INT_MAX;
        const int fz0 = bc[0] & ~3, fx0 = bc[2], fy0 = bc[4];
        const int fzl = bc[1] + 1 - fz0, fxl = bc[3] - bc[2] + 1, fyl = bc[5] - bc[4] + 1;
        const bool ftile = any && fzl <= FZ3 && fxl <= FX3 && fyl <= FY3;
        // every deposition window lies within one node below and two above the gather stencils
        const int jz0 = (bc[0] - 1) & ~3, jx0 = bc[2] - 1, jy0 = bc[4] - 1;
        const int jzl = bc[1] + 3 - jz0, jxl = bc[3] - bc[2] + 4, jyl = bc[5] - bc[4] + 4;
        const bool jtile = any && jzl <= JZ3 && jxl <= JX3 && jyl <= JY3;
        if (DEFER && any && !(ftile && jtile)) {
            // boxes the general path holds in shared memory (its own rounding of the z extents) go to
            // the general kernel's list, the rest (the plasma injected since the last sort: one
            // long row of cells) to the per-particle kernel's list
            const int gfz = (bc[1] + 1 - fz0 + 3) & ~3, gjz = (bc[1] + 3 - jz0 + 3) & ~3;
            const bool general = 6 * gfz * fxl * fyl <= F_CAP3 && fxl <= g.nx + 2 * K && fyl <= g.ny + 2 * K &&
                                 3 * gjz * jxl * jyl <= J_CAP3 && jxl <= g.nx + 2 * KW && jyl <= g.ny + 2 * KW;
            int* list = general ? defer : defer2;
            if (threadIdx.x == 0) list[2 + atomicAdd(list, 1)] = (int)(base / FUSED_T);
            __syncthreads();                       // everyone has read this chunk's box words
            continue;
        }
        // groups (c, y, x, z4) of the [c][y][x][z] box, only those inside the used extents, copied
        // asynchronously (all of a thread's groups in flight at once); z groups start at multiples of
        // 4, so with nz % 4 == 0 a group lies wholly inside or wholly outside 0 <= z < nz
        const int ngz = ftile ? (fzl + 3) >> 2 : 0;
        const unsigned mgz = ftile ? kInv16.m[ngz] : 0u, mfx = ftile ? kInv16.m[fxl] : 0u,
                       mfy = ftile ? kInv16.m[fyl] : 0u;
        const int nstage = 6 * fyl * fxl * ngz;
        auto staged = [&](auto&& f) {
#pragma unroll 2
            for (int i = threadIdx.x; i < nstage; i += FUSED_T) {
                const int r = qdiv(i, mgz), zg = i - r * ngz;
                const int r2 = qdiv(r, mfx), x = r - r2 * fxl;
                const int c = qdiv(r2, mfy), y = r2 - c * fyl;
                f(c, x, y, zg);
            }
        };
        static_assert(6 * FY3 * FX3 * (FZ3 / 4) < 2048 && FX3 <= 32 && FY3 <= 32 && FZ3 / 4 <= 32, "qdiv range");
        if (ftile) {
            staged([&](int c, int x, int y, int zg) {
                const long long row = ((long long)wrapi(fy0 + y, g.ny) * g.nx + wrapi(fx0 + x, g.nx)) * g.nz;
                const float* f = (c < 3 ? E + c * N : B + (c - 3) * N) + row;
                float* d = sF + c * FV3 + (y * FX3 + x) * FZP3 + 4 * zg;
                const int gz = fz0 + 4 * zg;
                if (fvec) {
                    const bool in = gz >= 0 && gz < g.nz;
                    cp_async16z(d, f + (in ? gz : 0), in);
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const bool in = (unsigned)(gz + j) < (unsigned)g.nz;
                        cp_async4z(d + j, f + (in ? gz + j : 0), in);
                    }
                }
            });
        }
        cp_async_commit();
        cp_async_wait_all_p();                     // the box (and the next chunk's particle words)
        // a particle at rest in zero fields stays at rest and carries no current: a chunk with no
        // moving particle reads its staged groups back to see whether they are all zero
        const bool moving = ok && (u[0] != 0.f || u[1] != 0.f || u[2] != 0.f);
        bool live = __syncthreads_or(moving);
        if (!live && ftile) {
            unsigned fbits = 0u;
            staged([&](int c, int x, int y, int zg) {
                const float4 v = *reinterpret_cast<const float4*>(sF + c * FV3 + (y * FX3 + x) * FZP3 + 4 * zg);
                fbits |= __float_as_uint(v.x) | __float_as_uint(v.y) | __float_as_uint(v.z) | __float_as_uint(v.w);
            });
            live = __syncthreads_or(fbits != 0u);
        }
        if (!live && ftile) {
            // a quiet chunk (every particle at rest, every field of its footprint zero): nothing
            // moves and no current flows; only a pending window shift is applied to the cells,
            // and the rest of the chunk runs with every particle switched off
            if (shift && ok) sp.cell[p] = encode(g, p0.iz, p0.ix, p0.iy);
            ok = false;
        }
        // ---- gather (E1 z+, E2 x+, E3 y+, B1 x+ y+, B2 z+ y+, B3 z+ x+) ----
        float eb[6];
        if (ok) {
            if (ftile) {
                auto at = [&](int comp, int z, int x, int y) {
                    return sF + comp * FV3 + ((y - fy0) * FX3 + (x - fx0)) * FZP3 + (z - fz0);
                };
                const float2 q1 = tile_interp3_fixed<K>(at(0, bzh, bxn, byn), Wzh, Wxn, Wyn, at(4, bzh, bxn, byh), Wzh,
                                                        Wxn, Wyh);                            // E1, B2
                const float2 q2 = tile_interp3_fixed<K>(at(1, bzn, bxh, byn), Wzn, Wxh, Wyn, at(3, bzn, bxh, byh), Wzn,
                                                        Wxh, Wyh);                            // E2, B1
                const float2 q3 = tile_interp3_fixed<K>(at(2, bzn, bxn, byh), Wzn, Wxn, Wyh, at(5, bzh, bxh, byn), Wzh,
                                                        Wxh, Wyn);                            // E3, B3
                eb[0] = q1.x;
                eb[4] = q1.y;
                eb[1] = q2.x;
                eb[3] = q2.y;
                eb[2] = q3.x;
                eb[5] = q3.y;
            } else if (!DEFER) {
                gather3_global<SHAPE>(g, E, B, p0, eb);
            }
        }
        // ---- push and move ----
        Pos p1 = p0;
        if (ok) {
            boris(sp.eps, eb, u);
            float gh, gl, rg;
            gamma_ff(u, gh, gl, rg);
            float dzh, dzl, dxh, dxl, dyh, dyl;
            displacement(u[0], gh, gl, rg, sp.kz[0], sp.kz[1], dzh, dzl);
            displacement(u[1], gh, gl, rg, sp.kx[0], sp.kx[1], dxh, dxl);
            displacement(u[2], gh, gl, rg, sp.ky[0], sp.ky[1], dyh, dyl);
            if (!(fabsf(dzh) < 1.f && fabsf(dxh) < 1.f && fabsf(dyh) < 1.f)) {
                ok = false;
                sp.cell[p] = -1;
            } else {
                advance_axis(p1.iz, p1.oz, dzh, dzl);
                advance_axis(p1.ix, p1.ox, dxh, dxl);
                advance_axis(p1.iy, p1.oy, dyh, dyl);
                const int wx = wrapi(p1.ix, g.nx), wy = wrapi(p1.iy, g.ny);
                sp.cell[p] = (p1.iz >= 0 && p1.iz < g.nz) ? encode(g, p1.iz, wx, wy) : -1;
                sp.off[p] = p1.oz;
                sp.off[cap + p] = p1.ox;
                sp.off[2 * cap + p] = p1.oy;
                sp.u[p] = u[0];
                sp.u[cap + p] = u[1];
                sp.u[2 * cap + p] = u[2];
            }
        }
        // ---- deposition ----
        float S0z[KW], DSz[KW], S0x[KW], DSx[KW], S0y[KW], DSy[KW];
        int bz = 0, bx = 0, by = 0;
        if (ok) {
            bz = axis_weights_from<SHAPE>(bzn, Wzn, p1.iz, p1.oz, S0z, DSz);
            bx = axis_weights_from<SHAPE>(bxn, Wxn, p1.ix, p1.ox, S0x, DSx);
            by = axis_weights_from<SHAPE>(byn, Wyn, p1.iy, p1.oy, S0y, DSy);
        } else {
#pragma unroll
            for (int k = 0; k < KW; ++k) S0z[k] = DSz[k] = S0x[k] = DSx[k] = S0y[k] = DSy[k] = 0.f;
        }
        const float f1 = -sp.qv * g.dz / g.dt, f2 = -sp.qv * g.dx / g.dt, f3 = -sp.qv * g.dy / g.dt;
        float cz[KW], cx[KW], cy[KW];
        float mb = 0.f;
        {
            float az = 0.f, ax = 0.f, ay = 0.f;
#pragma unroll
            for (int k = 0; k < KW; ++k) {
                az += DSz[k];
                ax += DSx[k];
                ay += DSy[k];
                cz[k] = az;
                cx[k] = ax;
                cy[k] = ay;
                mb = fmaxf(mb, fmaxf(fabsf(f1 * az), fmaxf(fabsf(f2 * ax), fabsf(f3 * ay))));
            }
        }
        // fixed-point scale of the chunk (see push_deposit_2d_chunks): s = 2^(22-e), max mb < 2^e
        if (jtile) {
            const unsigned wm = __reduce_max_sync(0xffffffffu, ok ? __float_as_uint(mb) : 0u);
            if ((threadIdx.x & 31) == 0 && wm) atomicMax(reinterpret_cast<unsigned*>(bc + 6), wm);
        }
        __syncthreads();
        const int mbits = bc[6];
        const int sexp = min(275 - (mbits >> 23), 253);
        const float fs = __int_as_float(sexp << 23), inv_s = __int_as_float((254 - sexp) << 23);
        if (jtile && mbits != 0) {
#pragma unroll
            for (int k = 0; k < KW; ++k) {
                cz[k] *= f1 * fs;
                cx[k] *= f2 * fs;
                cy[k] *= f3 * fs;
            }
            // P = S0 + dS/2 and Q = S0/2 + dS/3 of an axis, formed where they are used
            auto P_ = [](float s0, float ds) { return fmaf(0.5f, ds, s0); };
            auto Q_ = [](float s0, float ds) { return fmaf(1.f / 3.f, ds, 0.5f * s0); };
            // Every lane adds its own deposits, also where many lanes of a warp share a window (the
            // dense beam): the shared-memory atomic unit serialises equal addresses, which costs less
            // than summing over the lanes of a window first (measured on the beam in plasma).
            int* s0 = iJ + ((by - jy0) * JX3 + (bx - jx0)) * JZP3 + (bz - jz0);
            const float MAGIC = 12582912.f;           // 1.5 2^23
            // When no lane of the warp changes its support node along an axis, the last node of the
            // window along that axis has S0 = dS = 0: every product with it is zero, and so is the
            // last cumulative sum along that axis (the dS sum to zero).  Those deposits are skipped
            // for the whole warp (the skipped values are exactly zero).
            const bool uz = __any_sync(0xffffffffu, S0z[KW - 1] != 0.f || DSz[KW - 1] != 0.f);
            const bool ux = __any_sync(0xffffffffu, S0x[KW - 1] != 0.f || DSx[KW - 1] != 0.f);
            const bool uy = __any_sync(0xffffffffu, S0y[KW - 1] != 0.f || DSy[KW - 1] != 0.f);
            // one component at a time: fewer values live at once
            auto terms = [&](auto&& put) {
#pragma unroll
                for (int c = 0; c < KW; ++c) {
                    if (c == KW - 1 && !uy) continue;
                    const float py = P_(S0y[c], DSy[c]), qy = Q_(S0y[c], DSy[c]);
#pragma unroll
                    for (int b = 0; b < KW; ++b) {
                        if (b == KW - 1 && !ux) continue;
                        const float t = fmaf(S0x[b], py, DSx[b] * qy);
#pragma unroll
                        for (int a = 0; a < KW - 1; ++a) {
                            if (a == KW - 2 && !uz) continue;
                            put((c * JX3 + b) * JZP3 + a, fmaf(cz[a], t, MAGIC));
                        }
                    }
#pragma unroll
                    for (int a = 0; a < KW; ++a) {
                        if (a == KW - 1 && !uz) continue;
                        const float t = fmaf(S0z[a], py, DSz[a] * qy);
#pragma unroll
                        for (int b = 0; b < KW - 1; ++b) {
                            if (b == KW - 2 && !ux) continue;
                            put(JV3 + (c * JX3 + b) * JZP3 + a, fmaf(cx[b], t, MAGIC));
                        }
                    }
                }
#pragma unroll
                for (int b = 0; b < KW; ++b) {
                    if (b == KW - 1 && !ux) continue;
                    const float px = P_(S0x[b], DSx[b]), qx = Q_(S0x[b], DSx[b]);
#pragma unroll
                    for (int a = 0; a < KW; ++a) {
                        if (a == KW - 1 && !uz) continue;
                        const float t = fmaf(S0z[a], px, DSz[a] * qx);
#pragma unroll
                        for (int c = 0; c < KW - 1; ++c) {
                            if (c == KW - 2 && !uy) continue;
                            put(2 * JV3 + (c * JX3 + b) * JZP3 + a, fmaf(cy[c], t, MAGIC));
                        }
                    }
                }
            };
            if (ok) terms([&](int o, float biased) { atomicAdd(s0 + o, __float_as_int(biased) - 0x4B400000); });
        } else if (!DEFER && any && !jtile && ok) {
            deposit3_global<SHAPE>(g, sp.qv, p0, p1, J);
        }
        __syncthreads();
        if (jtile && mbits != 0) {
            // box -> J in 16-byte groups (one vector atomic per group inside the grid); the groups
            // are cleared as they are read, for the next chunk
            const int ng = (jzl + 3) >> 2;
            const unsigned mg = kInv16.m[ng], mjx = kInv16.m[jxl], mjy = kInv16.m[jyl];
            static_assert(3 * JY3 * JX3 * (JZ3 / 4) < 2048 && JX3 <= 32 && JY3 <= 32 && JZ3 / 4 <= 32, "qdiv range");
            for (int i = threadIdx.x; i < 3 * jyl * jxl * ng; i += FUSED_T) {
                const int r = qdiv(i, mg), zg = i - r * ng;
                const int r2 = qdiv(r, mjx), x = r - r2 * jxl;
                const int c = qdiv(r2, mjy), y = r2 - c * jyl;
                int4* grp = reinterpret_cast<int4*>(iJ + c * JV3 + (y * JX3 + x) * JZP3) + zg;
                const int4 q = *grp;
                if ((q.x | q.y | q.z | q.w) == 0) continue;
                *grp = make_int4(0, 0, 0, 0);
                const float4 v = make_float4((float)q.x * inv_s, (float)q.y * inv_s, (float)q.z * inv_s,
                                             (float)q.w * inv_s);
                const int gz = jz0 + 4 * zg;
                float* dst = J + c * N + (wrapi(jy0 + y, g.ny) * g.nx + wrapi(jx0 + x, g.nx)) * g.nz + gz;
                if (jvec && gz >= 0 && gz + 3 < g.nz) {
                    atomicAdd(reinterpret_cast<float4*>(dst), v);
                } else {
                    if ((unsigned)gz < (unsigned)g.nz && q.x) atomicAdd(dst, v.x);
                    if ((unsigned)(gz + 1) < (unsigned)g.nz && q.y) atomicAdd(dst + 1, v.y);
                    if ((unsigned)(gz + 2) < (unsigned)g.nz && q.z) atomicAdd(dst + 2, v.z);
                    if ((unsigned)(gz + 3) < (unsigned)g.nz && q.w) atomicAdd(dst + 3, v.w);
                }
            }
        }
    }
    cp_async_wait_all_p();                         // the last (empty) prefetch group
}

template <int SHAPE>
__global__ void __launch_bounds__(FUSED_T, 3) push_deposit_3d_kernel(GridP g, SpeciesP sp, const float* __restrict__ E,
                                                                     const float* __restrict__ B, float* __restrict__ J,
                                                                     int shift, int* __restrict__ defer,
                                                                     int* __restrict__ defer2) {
    extern __shared__ float4 smem4[];
    float* smem = reinterpret_cast<float*>(smem4);
    __shared__ int box[14];
    push_deposit_3d_chunks<SHAPE, true>(g, sp, E, B, J, shift, blockIdx.x, gridDim.x, smem, smem + 6 * FV3, box,
                                        defer, defer2);
}

// The chunks of defer2 (see push_deposit_3d_chunks): per particle, gather from global memory, push,
// move and deposit with global atomics (contributions that are exactly zero are not added); a
// light kernel at full occupancy.  The last CTA to finish clears the list (defer2[1] counts CTAs).
template <int SHAPE>
__global__ void __launch_bounds__(FUSED_T, 2) push_deposit_3d_particles_kernel(GridP g, SpeciesP sp,
                                                                            const float* __restrict__ E,
                                                                            const float* __restrict__ B,
                                                                            float* __restrict__ J, int shift,
                                                                            int* __restrict__ defer2) {
    const int nd = *(volatile int*)defer2;
    const long long n = *sp.count;
    for (int k = blockIdx.x; k < nd; k += gridDim.x) {
        const long long p = (long long)defer2[2 + k] * FUSED_T + threadIdx.x;
        if (p >= n) continue;
        Pos p0, p1;
        float v3;
        if (advance_one<3, SHAPE, MODE_FUSED>(g, sp, E, B, shift, p, sp.cap, p0, p1, v3)) {
            GlobalAcc acc{&g, J};
            deposit<3, SHAPE>(g, sp.qv, v3, p0, p1, acc);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(defer2 + 1, 1) == (int)gridDim.x - 1) {
            defer2[0] = 0;
            defer2[1] = 0;
            __threadfence();
        }
    }
}

constexpr int SMEM_3D_GEN = F_CAP3 + J_CAP3 + 2 * PF3 * FUSED_T;

// .x = sum Wza Wxa Wya Fa, .y = sum Wzb Wxb Wyb Fb over K^3 nodes of [y][x][z] boxes (row fzl,
// fxl rows per plane); (z, x, y) are the stencil origins in the box.
template <int K>
__device__ __forceinline__ float2 tile_interp3_pair(const float* __restrict__ Fa, int za, int xa, int ya,
                                                    const float (&Wza)[K], const float (&Wxa)[K],
                                                    const float (&Wya)[K], const float* __restrict__ Fb, int zb,
                                                    int xb, int yb, const float (&Wzb)[K], const float (&Wxb)[K],
                                                    const float (&Wyb)[K], int fzl, int fxl) {
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int c = 0; c < K; ++c) {
        float2 tc = make_float2(0.f, 0.f);
#pragma unroll
        for (int b = 0; b < K; ++b) {
            const float* ra = Fa + ((ya + c) * fxl + xa + b) * fzl + za;
            const float* rb = Fb + ((yb + c) * fxl + xb + b) * fzl + zb;
            float2 t = make_float2(0.f, 0.f);
#pragma unroll
            for (int a = 0; a < K; ++a) t = __ffma2_rn(make_float2(Wza[a], Wzb[a]), make_float2(ra[a], rb[a]), t);
            tc = __ffma2_rn(make_float2(Wxa[b], Wxb[b]), t, tc);
        }
        acc = __ffma2_rn(make_float2(Wya[c], Wyb[c]), tc, acc);
    }
    return acc;
}

// The general path for the chunks push_deposit_3d_kernel leaves (list[0 .. nlist)): boxes of any
// shape up to F_CAP3 / J_CAP3 words, runtime strides; larger boxes use global memory.
template <int SHAPE>
__device__ __forceinline__ void push_deposit_3d_general(const GridP& g, const SpeciesP& sp,
                                                        const float* __restrict__ E, const float* __restrict__ B,
                                                        float* __restrict__ J, int shift, const int* __restrict__ list,
                                                        int nlist, float* sF, float* sJ, int* box) {
    constexpr int K = Shape<SHAPE>::K;
    constexpr int KW = K + 1;
    const long long n = *sp.count;
    const long long cap = sp.cap;
    const int N = (int)g.ncell;
    const bool fvec = (g.nz & 3) == 0 && aligned16(E) && aligned16(B);
    const bool jvec = (g.nz & 3) == 0 && aligned16(J);
    float* const pfb = sJ + J_CAP3;                   // [2][PF3][FUSED_T]
    auto prefetch = [&](long long b, int buf) {
        const long long q = b + threadIdx.x;
        if (q < n) {
            float* d = pfb + buf * PF3 * FUSED_T + threadIdx.x;
            cp_async4(d, sp.cell + q);
            cp_async4(d + FUSED_T, sp.off + q);
            cp_async4(d + 2 * FUSED_T, sp.off + cap + q);
            cp_async4(d + 3 * FUSED_T, sp.off + 2 * cap + q);
            cp_async4(d + 4 * FUSED_T, sp.u + q);
            cp_async4(d + 5 * FUSED_T, sp.u + cap + q);
            cp_async4(d + 6 * FUSED_T, sp.u + 2 * cap + q);
        }
        cp_async_commit();
    };
    int buf = 0;
    const int k0 = blockIdx.x, kst = gridDim.x;
    auto chunk_base = [&](int k) { return k < nlist ? (long long)list[k] * FUSED_T : n; };
    prefetch(chunk_base(k0), 0);
    // box[0..6] and box[7..13] serve alternate chunks (see push_deposit_2d_chunks): no barrier at
    // the top of the loop or after the flush
    if (threadIdx.x < 14) {
        const int q = threadIdx.x % 7;
        box[threadIdx.x] = q == 6 ? 0 : (q & 1) ? INT_MIN : INT_MAX;
    }
    __syncthreads();
    int cur = 0;
    for (int k = k0; k < nlist; k += kst, buf ^= 1, cur ^= 7) {
        const long long base = chunk_base(k);
        int* const bc = box + cur;
        if (threadIdx.x < 7) box[(cur ^ 7) + threadIdx.x] = threadIdx.x == 6 ? 0 : (threadIdx.x & 1) ? INT_MIN : INT_MAX;
        prefetch(chunk_base(k + kst), buf ^ 1);
        cp_async_wait_prev();                      // this thread's words of this chunk
        const long long p = base + threadIdx.x;
        const float* mine = pfb + buf * PF3 * FUSED_T + threadIdx.x;
        // ---- load and decode ----
        bool ok = false;
        Pos p0;
        float u[3] = {0.f, 0.f, 0.f};
        if (p < n) {
            int cell = __float_as_int(mine[0]);
            if (cell >= 0) {
                int izg;
                decode(g, cell, izg, p0.ix, p0.iy);
                p0.iz = izg - 1 - shift;
                if (p0.iz >= 0 && p0.iz < g.nz) {
                    ok = true;
                    p0.oz = mine[FUSED_T];
                    p0.ox = mine[2 * FUSED_T];
                    p0.oy = mine[3 * FUSED_T];
                    u[0] = mine[4 * FUSED_T];
                    u[1] = mine[5 * FUSED_T];
                    u[2] = mine[6 * FUSED_T];
                } else {
                    sp.cell[p] = -1;
                }
            }
        }
        // ---- gather weights and the chunk's boxes ----
        float Wzn[K], Wzh[K], Wxn[K], Wxh[K], Wyn[K], Wyh[K];
        int bzn = 0, bzh = 0, bxn = 0, bxh = 0, byn = 0, byh = 0;
        if (ok) {
            bzn = p0.iz + Shape<SHAPE>::w(p0.oz, Wzn);
            bzh = half_weights<SHAPE>(p0.iz, p0.oz, Wzh);
            bxn = p0.ix + Shape<SHAPE>::w(p0.ox, Wxn);
            bxh = half_weights<SHAPE>(p0.ix, p0.ox, Wxh);
            byn = p0.iy + Shape<SHAPE>::w(p0.oy, Wyn);
            byh = half_weights<SHAPE>(p0.iy, p0.oy, Wyh);
        }
        box_reduce(bc, ok ? min(bzn, bzh) : INT_MAX, ok ? max(bzn, bzh) + K - 1 : INT_MIN,
                   ok ? min(bxn, bxh) : INT_MAX, ok ? max(bxn, bxh) + K - 1 : INT_MIN);
        {
            const int c = __reduce_min_sync(0xffffffffu, ok ? min(byn, byh) : INT_MAX);
            const int d = __reduce_max_sync(0xffffffffu, ok ? max(byn, byh) + K - 1 : INT_MIN);
            if ((threadIdx.x & 31) == 0 && c != INT_MAX) {
                atomicMin(bc + 4, c);
                atomicMax(bc + 5, d);
            }
        }
        __syncthreads();
        const bool any = bc[0] != INT_MAX;
        const int fz0 = any ? (bc[0] & ~3) : 0, fx0 = bc[2], fy0 = bc[4];
        const int fzl = any ? ((bc[1] + 1 - fz0 + 3) & ~3) : 0;
        const int fxl = any ? bc[3] - bc[2] + 1 : 0, fyl = any ? bc[5] - bc[4] + 1 : 0;
        const int fvol = fzl * fxl * fyl;
        const bool ftile = any && 6 * fvol <= F_CAP3 && fxl <= g.nx + 2 * K && fyl <= g.ny + 2 * K;
        const int jz0 = any ? ((bc[0] - 1) & ~3) : 0, jx0 = bc[2] - 1, jy0 = bc[4] - 1;
        const int jzl = any ? ((bc[1] + 3 - jz0 + 3) & ~3) : 0;
        const int jxl = any ? bc[3] - bc[2] + 4 : 0, jyl = any ? bc[5] - bc[4] + 4 : 0;
        const int jvol = jzl * jxl * jyl;
        const bool jtile = any && 3 * jvol <= J_CAP3 && jxl <= g.nx + 2 * KW && jyl <= g.ny + 2 * KW;
        // groups (c, y, x, z4) of the [c][y][x][z] box, copied asynchronously (all of a thread's
        // groups in flight at once); z groups start at multiples of 4, so with nz % 4 == 0 a group
        // lies wholly inside or wholly outside 0 <= z < nz
        const int ng = fzl >> 2, rows = fyl * fxl;
        const float rg = 1.f / (float)max(ng, 1), rr = 1.f / (float)max(rows, 1), rx = 1.f / (float)max(fxl, 1);
        auto staged = [&](auto&& f) {
            for (int i = threadIdx.x; i < 6 * rows * ng; i += FUSED_T) {
                const int r = box_div(i, rg), zg = i - r * ng;
                const int c = box_div(r, rr), q = r - c * rows;
                f(c, q, zg);
            }
        };
        if (ftile) {
            staged([&](int c, int q, int zg) {
                const int y = box_div(q, rx), x = q - y * fxl;
                const long long row = ((long long)wrapi(fy0 + y, g.ny) * g.nx + wrapi(fx0 + x, g.nx)) * g.nz;
                const float* f = (c < 3 ? E + c * N : B + (c - 3) * N) + row;
                float* d = sF + c * fvol + q * fzl + 4 * zg;
                const int gz = fz0 + 4 * zg;
                if (fvec) {
                    const bool in = gz >= 0 && gz < g.nz;
                    cp_async16z(d, f + (in ? gz : 0), in);
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const bool in = (unsigned)(gz + j) < (unsigned)g.nz;
                        cp_async4z(d + j, f + (in ? gz + j : 0), in);
                    }
                }
            });
        }
        cp_async_commit();
        if (jtile)
            for (int i = threadIdx.x; i < (3 * jvol) >> 2; i += FUSED_T)
                reinterpret_cast<float4*>(sJ)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        cp_async_wait_all_p();                     // the box (and the next chunk's particle words)
        // a quiet chunk (every particle at rest, every field of its footprint zero; the plasma
        // injected at the front since the last sort): only a pending window shift is applied to
        // the cells, and the rest of the chunk runs with every particle switched off.  The staged
        // groups are read back only when no particle of the chunk moves.
        const bool moving = ok && (u[0] != 0.f || u[1] != 0.f || u[2] != 0.f);
        bool live = __syncthreads_or(moving);
        if (!live && ftile) {
            unsigned fbits = 0u;
            staged([&](int c, int q, int zg) {
                const float4 v = *reinterpret_cast<const float4*>(sF + c * fvol + q * fzl + 4 * zg);
                fbits |= __float_as_uint(v.x) | __float_as_uint(v.y) | __float_as_uint(v.z) | __float_as_uint(v.w);
            });
            live = __syncthreads_or(fbits != 0u);
        }
        if (!live && ftile) {
            if (shift && ok) sp.cell[p] = encode(g, p0.iz, p0.ix, p0.iy);
            ok = false;
        }
        // ---- gather (E1 z+, E2 x+, E3 y+, B1 x+ y+, B2 z+ y+, B3 z+ x+) ----
        float eb[6];
        if (ok) {
            if (ftile) {
                const float* F = sF;
                const float2 q1 = tile_interp3_pair<K>(F, bzh - fz0, bxn - fx0, byn - fy0, Wzh, Wxn, Wyn,
                                                       F + 4 * fvol, bzh - fz0, bxn - fx0, byh - fy0, Wzh, Wxn,
                                                       Wyh, fzl, fxl);                       // E1, B2
                const float2 q2 = tile_interp3_pair<K>(F + fvol, bzn - fz0, bxh - fx0, byn - fy0, Wzn, Wxh, Wyn,
                                                       F + 3 * fvol, bzn - fz0, bxh - fx0, byh - fy0, Wzn, Wxh,
                                                       Wyh, fzl, fxl);                       // E2, B1
                const float2 q3 = tile_interp3_pair<K>(F + 2 * fvol, bzn - fz0, bxn - fx0, byh - fy0, Wzn, Wxn,
                                                       Wyh, F + 5 * fvol, bzh - fz0, bxh - fx0, byn - fy0, Wzh,
                                                       Wxh, Wyn, fzl, fxl);                  // E3, B3
                eb[0] = q1.x;
                eb[4] = q1.y;
                eb[1] = q2.x;
                eb[3] = q2.y;
                eb[2] = q3.x;
                eb[5] = q3.y;
            } else {
                gather<3, SHAPE>(g, E, B, p0, eb);
            }
        }
        // ---- push and move ----
        Pos p1 = p0;
        if (ok) {
            boris(sp.eps, eb, u);
            float gh, gl, rg;
            gamma_ff(u, gh, gl, rg);
            float dzh, dzl, dxh, dxl, dyh, dyl;
            displacement(u[0], gh, gl, rg, sp.kz[0], sp.kz[1], dzh, dzl);
            displacement(u[1], gh, gl, rg, sp.kx[0], sp.kx[1], dxh, dxl);
            displacement(u[2], gh, gl, rg, sp.ky[0], sp.ky[1], dyh, dyl);
            if (!(fabsf(dzh) < 1.f && fabsf(dxh) < 1.f && fabsf(dyh) < 1.f)) {
                ok = false;
                sp.cell[p] = -1;
            } else {
                advance_axis(p1.iz, p1.oz, dzh, dzl);
                advance_axis(p1.ix, p1.ox, dxh, dxl);
                advance_axis(p1.iy, p1.oy, dyh, dyl);
                const int wx = wrapi(p1.ix, g.nx), wy = wrapi(p1.iy, g.ny);
                sp.cell[p] = (p1.iz >= 0 && p1.iz < g.nz) ? encode(g, p1.iz, wx, wy) : -1;
                sp.off[p] = p1.oz;
                sp.off[cap + p] = p1.ox;
                sp.off[2 * cap + p] = p1.oy;
                sp.u[p] = u[0];
                sp.u[cap + p] = u[1];
                sp.u[2 * cap + p] = u[2];
            }
        }
        // ---- deposition ----
        float S0z[KW], DSz[KW], S0x[KW], DSx[KW], S0y[KW], DSy[KW];
        int bz = 0, bx = 0, by = 0;
        if (ok) {
            bz = axis_weights_from<SHAPE>(bzn, Wzn, p1.iz, p1.oz, S0z, DSz);
            bx = axis_weights_from<SHAPE>(bxn, Wxn, p1.ix, p1.ox, S0x, DSx);
            by = axis_weights_from<SHAPE>(byn, Wyn, p1.iy, p1.oy, S0y, DSy);
        } else {
#pragma unroll
            for (int k = 0; k < KW; ++k) S0z[k] = DSz[k] = S0x[k] = DSx[k] = S0y[k] = DSy[k] = 0.f;
        }
        const float f1 = -sp.qv * g.dz / g.dt, f2 = -sp.qv * g.dx / g.dt, f3 = -sp.qv * g.dy / g.dt;
        float cz[KW], cx[KW], cy[KW];
        float mb = 0.f;
        {
            float az = 0.f, ax = 0.f, ay = 0.f;
#pragma unroll
            for (int k = 0; k < KW; ++k) {
                az += DSz[k];
                ax += DSx[k];
                ay += DSy[k];
                cz[k] = az;
                cx[k] = ax;
                cy[k] = ay;
                mb = fmaxf(mb, fmaxf(fabsf(f1 * az), fmaxf(fabsf(f2 * ax), fabsf(f3 * ay))));
            }
        }
        // fixed-point scale of the chunk (see push_deposit_2d_chunks): s = 2^(22-e), max mb < 2^e
        if (jtile) {
            const unsigned wm = __reduce_max_sync(0xffffffffu, ok ? __float_as_uint(mb) : 0u);
            if ((threadIdx.x & 31) == 0 && wm) atomicMax(reinterpret_cast<unsigned*>(bc + 6), wm);
        }
        __syncthreads();
        const int mbits = bc[6];
        const int sexp = min(275 - (mbits >> 23), 253);
        const float fs = __int_as_float(sexp << 23), inv_s = __int_as_float((254 - sexp) << 23);
        int* const iJ = reinterpret_cast<int*>(sJ);
        if (any && jtile && mbits != 0) {
            float Cz[KW], Cx[KW], Cy[KW], Px[KW], Qx[KW], Py[KW], Qy[KW];
#pragma unroll
            for (int k = 0; k < KW; ++k) {
                Cz[k] = f1 * fs * cz[k];
                Cx[k] = f2 * fs * cx[k];
                Cy[k] = f3 * fs * cy[k];
                Px[k] = S0x[k] + 0.5f * DSx[k];
                Qx[k] = 0.5f * S0x[k] + (1.f / 3.f) * DSx[k];
                Py[k] = S0y[k] + 0.5f * DSy[k];
                Qy[k] = 0.5f * S0y[k] + (1.f / 3.f) * DSy[k];
            }
            // window origins are >= -2 and below 2^20 - 4 on every axis: an exact 64-bit key
            const unsigned long long key =
                ok ? (((unsigned long long)(bz + 4) << 40) | ((unsigned long long)(bx + 4) << 20) |
                      (unsigned long long)(by + 4))
                   : (0xFFFFF00000000000ull | (unsigned)threadIdx.x);
            // direct atomics when at most 4 lanes share a window (144 deposits per particle make
            // conflicts costlier than in 2D), else sums over runs of lanes first
            const int gmax = __reduce_max_sync(0xffffffffu, __popc(__match_any_sync(0xffffffffu, key)));
            int* s0 = iJ + ((by - jy0) * jxl + (bx - jx0)) * jzl + (bz - jz0);
            const float MAGIC = 12582912.f;           // 1.5 2^23
            auto terms = [&](auto&& put) {
#pragma unroll
                for (int c = 0; c < KW; ++c)
#pragma unroll
                    for (int b = 0; b < KW; ++b) {
                        const float txy = fmaf(S0x[b], Py[c], DSx[b] * Qy[c]);
#pragma unroll
                        for (int a = 0; a < KW; ++a) {
                            const int o = (c * jxl + b) * jzl + a;
                            if (a < KW - 1) put(o, fmaf(Cz[a], txy, MAGIC));
                            if (b < KW - 1) put(jvol + o, fmaf(Cx[b], fmaf(S0z[a], Py[c], DSz[a] * Qy[c]), MAGIC));
                            if (c < KW - 1)
                                put(2 * jvol + o, fmaf(Cy[c], fmaf(S0z[a], Px[b], DSz[a] * Qx[b]), MAGIC));
                        }
                    }
            };
            if (gmax <= 4) {
                if (ok) terms([&](int o, float biased) { atomicAdd(s0 + o, __float_as_int(biased) - 0x4B400000); });
            } else {
                const SegReduce seg = make_segments(key);
                terms([&](int o, float biased) {
                    const int v = seg.sum(__float_as_int(biased) - 0x4B400000);
                    if (seg.head && ok && v != 0) atomicAdd(s0 + o, v);
                });
            }
        } else if (any && !jtile && ok) {
            GlobalAcc acc{&g, J};
            deposit<3, SHAPE>(g, sp.qv, 0.f, p0, p1, acc);
        }
        __syncthreads();
        if (jtile && mbits != 0) {
            const int ng = jzl >> 2, rows = jyl * jxl;
            const float rg = 1.f / (float)ng, rr = 1.f / (float)rows, rx = 1.f / (float)jxl;
            for (int i = threadIdx.x; i < 3 * rows * ng; i += FUSED_T) {
                const int4 q = reinterpret_cast<const int4*>(iJ)[i];
                if ((q.x | q.y | q.z | q.w) == 0) continue;
                const float4 v = make_float4((float)q.x * inv_s, (float)q.y * inv_s, (float)q.z * inv_s,
                                             (float)q.w * inv_s);
                const int r = box_div(i, rg), zg = i - r * ng;
                const int c = box_div(r, rr), qq = r - c * rows;
                const int y = box_div(qq, rx), x = qq - y * jxl;
                const int gz = jz0 + 4 * zg;
                float* dst = J + c * N + (wrapi(jy0 + y, g.ny) * g.nx + wrapi(jx0 + x, g.nx)) * g.nz + gz;
                if (jvec && gz >= 0 && gz + 3 < g.nz) {
                    atomicAdd(reinterpret_cast<float4*>(dst), v);
                } else {
                    if ((unsigned)gz < (unsigned)g.nz && q.x) atomicAdd(dst, v.x);
                    if ((unsigned)(gz + 1) < (unsigned)g.nz && q.y) atomicAdd(dst + 1, v.y);
                    if ((unsigned)(gz + 2) < (unsigned)g.nz && q.z) atomicAdd(dst + 2, v.z);
                    if ((unsigned)(gz + 3) < (unsigned)g.nz && q.w) atomicAdd(dst + 3, v.w);
                }
            }
        }
    }
    cp_async_wait_all_p();                         // the last (empty) prefetch group
}

// The chunks push_deposit_3d_kernel deferred (defer[0] of them, chunk indices from defer[2]), on the
// general path.  The last CTA to finish clears the list (defer[1] counts finished CTAs).
template <int SHAPE>
__global__ void __launch_bounds__(FUSED_T, 2) push_deposit_3d_deferred_kernel(GridP g, SpeciesP sp,
                                                                              const float* __restrict__ E,
                                                                              const float* __restrict__ B,
                                                                              float* __restrict__ J, int shift,
                                                                              int* __restrict__ defer) {
    extern __shared__ float4 smem4[];
    float* smem = reinterpret_cast<float*>(smem4);
    __shared__ int box[14];
    const int nd = *(volatile int*)defer;
    push_deposit_3d_general<SHAPE>(g, sp, E, B, J, shift, defer + 2, nd, smem, smem + F_CAP3, box);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(defer + 1, 1) == (int)gridDim.x - 1) {
            defer[0] = 0;
            defer[1] = 0;
            __threadfence();
        }
    }
}

template <int SHAPE>
__global__ void __launch_bounds__(FUSED_T, 2) push_deposit_3d_batch_kernel(const PartInst* __restrict__ inst, int parity) {
    extern __shared__ float4 smem4[];
    float* smem = reinterpret_cast<float*>(smem4);
    __shared__ int box[14];
    const PartInst& q = inst[blockIdx.y];
    const GridP g = prep_device(q.g);
    push_deposit_3d_chunks<SHAPE, false>(g, q.sp, q.E[parity], q.B[parity], q.J, 0, blockIdx.x, gridDim.x, smem,
                                         smem + 6 * FV3, box, nullptr, nullptr);
}

template <int SHAPE>
__global__ void __launch_bounds__(FUSED_T, 4) push_deposit_2d_kernel(GridP g, SpeciesP sp, const float* __restrict__ E,
                                                                     const float* __restrict__ B, float* __restrict__ J,
                                                                     int shift) {
    extern __shared__ float4 smem4[];      // 16-byte aligned: the boxes are read and written as float4
    float* smem = reinterpret_cast<float*>(smem4);
    __shared__ int box[5];
    push_deposit_2d_chunks<SHAPE>(g, sp, E, B, J, shift, blockIdx.x, gridDim.x, smem, smem + F_CAP, box);
}

template <int SHAPE>
__global__ void __launch_bounds__(FUSED_T, 4) push_deposit_2d_batch_kernel(const PartInst* __restrict__ inst, int parity) {
    extern __shared__ float4 smem4[];
    float* smem = reinterpret_cast<float*>(smem4);
    __shared__ int box[5];
    const PartInst& q = inst[blockIdx.y];
    const GridP g = prep_device(q.g);
    push_deposit_2d_chunks<SHAPE>(g, q.sp, q.E[parity], q.B[parity], q.J, 0, blockIdx.x, gridDim.x, smem, smem + F_CAP,
                                  box);
}

// J = 0 for every instance (blockIdx.y) of a batch.
__global__ void zero_j_batch_kernel(const PartInst* __restrict__ inst) {
    const PartInst& q = inst[blockIdx.y];
    const long long n = 3 * q.g.ncell;
    float4* J4 = reinterpret_cast<float4*>(q.J);
    const long long n4 = ((uintptr_t)q.J & 15) ? 0 : n / 4;   // vector stores only when aligned
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x)
        J4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (long long i = 4 * n4 + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        q.J[i] = 0.f;
}

template <int NDIM, int SHAPE>
__device__ __forceinline__ void deposit_one(const GridP& g, const SpeciesP& sp, float* __restrict__ J,
                                            long long p) {
    const long long cap = sp.cap;
    int c0 = sp.prev_cell[p], c1 = sp.cell[p];
    if (c0 < 0 || c1 < 0) return;
    Pos p0, p1;
    int izg;
    decode(g, c0, izg, p0.ix, p0.iy);
    p0.iz = izg - 1;
    decode(g, c1, izg, p1.ix, p1.iy);
    p1.iz = izg - 1;
    // undo the periodic wrap of the new cell (moves are below one cell)
    if (p1.ix - p0.ix > 1) p1.ix -= g.nx;
    if (p1.ix - p0.ix < -1) p1.ix += g.nx;
    if (NDIM == 3) {
        if (p1.iy - p0.iy > 1) p1.iy -= g.ny;
        if (p1.iy - p0.iy < -1) p1.iy += g.ny;
    }
    p0.oz = sp.prev_off[p];
    p0.ox = sp.prev_off[cap + p];
    p0.oy = NDIM == 3 ? sp.prev_off[2 * cap + p] : 0.f;
    p1.oz = sp.off[p];
    p1.ox = sp.off[cap + p];
    p1.oy = NDIM == 3 ? sp.off[2 * cap + p] : 0.f;
    float u[3] = {sp.u[p], sp.u[cap + p], sp.u[2 * cap + p]};
    float gh, gl, rg;
    gamma_ff(u, gh, gl, rg);
    GlobalAcc acc{&g, J};
    deposit<NDIM, SHAPE>(g, sp.qv, u[2] * rg, p0, p1, acc);
    if (p1.iz < 0 || p1.iz >= g.nz) sp.cell[p] = -1;
}

// Unfused deposition from the positions saved by push_kernel<MODE_PUSH_ONLY>.
template <int NDIM, int SHAPE>
__global__ void __launch_bounds__(256) deposit_kernel(GridP g, SpeciesP sp, float* __restrict__ J) {
    const long long n = *sp.count;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x)
        deposit_one<NDIM, SHAPE>(g, sp, J, p);
}

// Cold plasma for the new front column.  Particle (k, j, a, b, c) (cell (nz, j, k), sub-cell
// position (a, b, c)) gets id next_id + canonical index ((k nx + j) P + (a px + b) py + c), P the
// particles per cell.  Its slot: the block starts at the old count rounded up to `align` (the gap
// filled with dead slots) and runs through patches of pxc x pyc cells (x-fastest patches, within
// a patch y, x, then the sub-cell index), clipped at the grid's edges.  In 3D, with align = 256
// and pxc pyc P <= 256, every 256 consecutive slots of the block then cover one compact patch of
// the new column, as after a sort, instead of a long row of cells.
__global__ void inject_kernel(GridP g, SpeciesP sp, int pz, int px, int py, int pxc, int pyc, int align,
                              long long nnew, long long next_id, int* status) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nnew + align - 1) return;
    const long long base0 = *sp.count;
    const long long base = (base0 + align - 1) / align * align;
    if (base + nnew > sp.cap) {
        if (t == 0) atomicOr(status, STATUS_CAPACITY);
        return;
    }
    long long s;
    if (t >= nnew) {                                   // the gap before the aligned block
        s = base0 + (t - nnew);
        if (s >= base) return;
        sp.cell[s] = -1;
        if (sp.id) sp.id[s] = -1;
        sp.off[s] = sp.off[sp.cap + s] = 0.f;
        if (g.ndim == 3) sp.off[2 * sp.cap + s] = 0.f;
        sp.u[s] = sp.u[sp.cap + s] = sp.u[2 * sp.cap + s] = 0.f;
        return;
    }
    const int P = pz * px * py, ny = g.ndim == 3 ? g.ny : 1;
    const long long band = (long long)pyc * g.nx * P;  // slots of one row of patches
    const int pb = (int)(t / band);
    long long r = t - pb * band;
    const int hb = min(pyc, ny - pb * pyc);
    const long long pw = (long long)pxc * hb * P;       // slots of a full-width patch of this row
    const int pa = (int)(r / pw);
    r -= pa * pw;
    const int wa = min(pxc, g.nx - pa * pxc);
    const int sub = (int)(r % P), cidx = (int)(r / P);
    const int j = pa * pxc + cidx % wa, k = pb * pyc + cidx / wa;
    const int c = sub % py, b = (sub / py) % px, a = sub / (py * px);
    s = base + t;
    sp.cell[s] = encode(g, g.nz, j, k);   // iz = nz: the pending shift brings it to nz - 1
    sp.off[s] = (a + 0.5f) / pz;
    sp.off[sp.cap + s] = (b + 0.5f) / px;
    if (g.ndim == 3) sp.off[2 * sp.cap + s] = (c + 0.5f) / py;
    sp.u[s] = 0.f;
    sp.u[sp.cap + s] = 0.f;
    sp.u[2 * sp.cap + s] = 0.f;
    if (sp.id) sp.id[s] = (int32_t)(next_id + ((long long)k * g.nx + j) * P + sub);
}

__global__ void add_count_kernel(int32_t* count, long long nnew, int align, long long cap) {
    const long long base = ((long long)*count + align - 1) / align * align;
    if (base + nnew <= cap) *count = (int32_t)(base + nnew);
}

// ---- counting sort by tiles of cells: 8 x 8 (z, x) in 2D, 4 x 4 x 4 in 3D ----
// (a chunk of consecutive particles then covers a compact patch, which keeps the shared-memory
// boxes of the fused kernels small; in 3D a cubic tile shrinks the chunk's field and current
// boxes by about a third against 8 x 8 x 1).  Tiles run in columns along z; the columns follow x
// then y, and the order snakes (z reversed in every other column, x in every other row of
// columns), so consecutive tiles are always neighbours: a chunk that straddles two columns stays
// compact instead of spanning the front and the back of the window.
__device__ __forceinline__ int sort_key(const GridP& g, int cell) {
    int izg, ix, iy;
    decode(g, cell, izg, ix, iy);
    if (g.ndim == 3) {          // 4 x 4 x 4-cell tiles: compact 3D chunks
        const int ntz = (g.nzg + 3) >> 2, ntx = (g.nx + 3) >> 2;
        const int ty = iy >> 2, tx = (ty & 1) ? ntx - 1 - (ix >> 2) : ix >> 2;
        const int col = ty * ntx + tx;
        const int tz = (col & 1) ? ntz - 1 - (izg >> 2) : izg >> 2;
        return (col * ntz + tz) * 64 + ((((iy & 3) << 2) + (ix & 3)) << 2) + (izg & 3);
    }
    const int ntz = (g.nzg + 7) >> 3, col = ix >> 3;
    const int tz = (col & 1) ? ntz - 1 - (izg >> 3) : izg >> 3;
    return (col * ntz + tz) * 64 + ((ix & 7) << 3) + (izg & 7);
}

// Cell-sorted particles come in runs of equal keys: the lanes of a warp with one key add their
// count with one atomic (the loop trip count is uniform across a warp).
__global__ void hist_kernel(GridP g, SpeciesP sp, int32_t* hist) {
    const long long n = *sp.count;
    const int lane = threadIdx.x & 31;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p - lane < n;
         p += (long long)gridDim.x * blockDim.x) {
        const int c = p < n ? sp.cell[p] : -1;
        const int key = c >= 0 ? sort_key(g, c) : -1;
        const unsigned grp = __match_any_sync(0xffffffffu, key);
        if (key >= 0 && lane == __ffs(grp) - 1) atomicAdd(hist + key, __popc(grp));
    }
}

constexpr int SCAN_T = 1024, SCAN_V = 4, SCAN_B = SCAN_T * SCAN_V;

__device__ int block_exclusive_scan(int v, int* sw) {
    // warp inclusive scan, then warp totals
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sw[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int t = lane < (int)(blockDim.x >> 5) ? sw[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        sw[lane] = t;   // inclusive warp-total prefix
    }
    __syncthreads();
    int before = wid > 0 ? sw[wid - 1] : 0;
    int total = sw[(blockDim.x >> 5) - 1];
    __syncthreads();
    sw[32] = total;
    return before + x - v;
}

__global__ void __launch_bounds__(SCAN_T) scan_blocks_kernel(int32_t* a, long long n, int32_t* sums) {
    __shared__ int sw[33];
    long long base = (long long)blockIdx.x * SCAN_B + (long long)threadIdx.x * SCAN_V;
    int v[SCAN_V];
    int s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_V; ++k) {
        v[k] = base + k < n ? a[base + k] : 0;
        s += v[k];
    }
    int ex = block_exclusive_scan(s, sw);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < SCAN_V; ++k) {
        if (base + k < n) a[base + k] = ex;
        ex += v[k];
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = sw[32];
}

// exclusive scan of nb block sums in one block; sums[nb] receives the grand total
__global__ void __launch_bounds__(SCAN_T) scan_sums_kernel(int32_t* sums, long long nb) {
    __shared__ int sw[33];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (long long base = 0; base < nb; base += SCAN_T) {
        long long i = base + threadIdx.x;
        int v = i < nb ? sums[i] : 0;
        int ex = block_exclusive_scan(v, sw);
        int c = carry;
        if (i < nb) sums[i] = ex + c;
        __syncthreads();
        if (threadIdx.x == 0) carry = c + sw[32];
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[nb] = carry;
}

__global__ void add_block_offsets_kernel(int32_t* a, long long n, const int32_t* sums) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] += sums[i / SCAN_B];
}

template <int NDIM>
__global__ void scatter_kernel(GridP g, SpeciesP sp, int32_t* cursor, int32_t* cell2, float* off2, float* u2,
                               int32_t* id2) {
    const long long n = *sp.count;
    const long long cap = sp.cap;
    const int lane = threadIdx.x & 31;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p - lane < n;
         p += (long long)gridDim.x * blockDim.x) {
        // one cursor atomic per key and warp; lanes keep their order within the key
        const int c = p < n ? sp.cell[p] : -1;
        const int key = c >= 0 ? sort_key(g, c) : -1;
        const unsigned grp = __match_any_sync(0xffffffffu, key);
        const int leader = __ffs(grp) - 1;
        int first = 0;
        if (key >= 0 && lane == leader) first = atomicAdd(cursor + key, __popc(grp));
        first = __shfl_sync(0xffffffffu, first, leader);
        if (key < 0) continue;
        const long long d = (long long)first + __popc(grp & ((1u << lane) - 1u));
        // every load before the first store: the source and destination arrays are distinct, and
        // the loads then overlap instead of waiting on one another's stores
        float o[NDIM], w[3];
#pragma unroll
        for (int k = 0; k < NDIM; ++k) o[k] = __ldg(sp.off + k * cap + p);
#pragma unroll
        for (int k = 0; k < 3; ++k) w[k] = __ldg(sp.u + k * cap + p);
        const int32_t idv = id2 ? __ldg(sp.id + p) : 0;
        cell2[d] = c;
#pragma unroll
        for (int k = 0; k < NDIM; ++k) off2[k * cap + d] = o[k];
#pragma unroll
        for (int k = 0; k < 3; ++k) u2[k * cap + d] = w[k];
        if (id2) id2[d] = idv;
    }
}

// copy the sorted slots [0, total) back into the caller's arrays and set the count
// (every load before the first store, as in scatter_kernel)
template <int NDIM>
__global__ void copy_back_kernel(SpeciesP sp, const int32_t* total, const int32_t* __restrict__ cell2,
                                 const float* __restrict__ off2, const float* __restrict__ u2,
                                 const int32_t* __restrict__ id2) {
    const long long n = *total;
    const long long cap = sp.cap;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const int32_t c = __ldg(cell2 + p);
        float o[NDIM], w[3];
#pragma unroll
        for (int k = 0; k < NDIM; ++k) o[k] = __ldg(off2 + k * cap + p);
#pragma unroll
        for (int k = 0; k < 3; ++k) w[k] = __ldg(u2 + k * cap + p);
        const int32_t idv = id2 ? __ldg(id2 + p) : 0;
        sp.cell[p] = c;
#pragma unroll
        for (int k = 0; k < NDIM; ++k) sp.off[k * cap + p] = o[k];
#pragma unroll
        for (int k = 0; k < 3; ++k) sp.u[k * cap + p] = w[k];
        if (id2) sp.id[p] = idv;
    }
}

__global__ void set_count_kernel(int32_t* count, const int32_t* total) { *count = *total; }

// ---- FP64 charge density at nodes ----
template <int NDIM, int SHAPE>
__device__ __forceinline__ void rho_one(const GridP& g, const SpeciesP& sp, int shift, double* rho,
                                        long long p) {
    int cell = sp.cell[p];
    if (cell < 0) return;
    int izg, ix, iy;
    decode(g, cell, izg, ix, iy);
    int iz = izg - 1 - shift;
    if (iz < 0 || iz >= g.nz) return;
    constexpr int K = Shape<SHAPE>::K;
    double wz[K], wx[K], wy[K];
    int bz = iz + Shape<SHAPE>::w((double)sp.off[p], wz);
    int bx = ix + Shape<SHAPE>::w((double)sp.off[sp.cap + p], wx);
    int by = NDIM == 3 ? iy + Shape<SHAPE>::w((double)sp.off[2 * sp.cap + p], wy) : 0;
    for (int c = 0; c < (NDIM == 3 ? K : 1); ++c)
        for (int b = 0; b < K; ++b)
            for (int a = 0; a < K; ++a) {
                int gz = bz + a;
                if (gz < 0 || gz >= g.nz) continue;
                int gx = wrapi(bx + b, g.nx);
                int gy = NDIM == 3 ? wrapi(by + c, g.ny) : 0;
                double w = wz[a] * wx[b] * (NDIM == 3 ? wy[c] : 1.0);
                atomicAdd(rho + ((long long)gy * g.nx + gx) * g.nz + gz, sp.qv64 * w);
            }
}


template <int NDIM, int SHAPE>
__global__ void rho_kernel(GridP g, SpeciesP sp, int shift, double* rho) {
    const long long n = *sp.count;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x)
        rho_one<NDIM, SHAPE>(g, sp, shift, rho, p);
}
template <typename F>
cudaError_t dispatch(int ndim, int shape, F&& f) {
    if (ndim == 2 && shape == 1) return f(std::integral_constant<int, 2>(), std::integral_constant<int, 1>());
    if (ndim == 2 && shape == 2) return f(std::integral_constant<int, 2>(), std::integral_constant<int, 2>());
    if (ndim == 3 && shape == 1) return f(std::integral_constant<int, 3>(), std::integral_constant<int, 1>());
    return f(std::integral_constant<int, 3>(), std::integral_constant<int, 2>());
}

inline unsigned nblocks(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// the particle kernels decode cells with the magic-number divisions of the grid
inline GridP prep(const GridP& g0) {
    GridP g = g0;
    g.div_nzg = make_fastdiv((uint32_t)g.nzg);
    g.div_nx = make_fastdiv((uint32_t)g.nx);
    return g;
}
// grid-stride kernels: enough CTAs for the expected extent, at most 16 per SM of a 152-SM part
inline unsigned pblocks(long long extent) {
    long long b = (extent + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

}  // namespace

cudaError_t launch_push(const GridP& g0, const SpeciesP& sp, const float* E, const float* B, float* J,
                        int shift, int mode, long long extent, int* defer, cudaStream_t s) {
    const GridP g = prep(g0);
    if (extent <= 0) return cudaSuccess;
    return dispatch(g.ndim, g.shape, [&](auto nd, auto sh) {
        constexpr int ND = decltype(nd)::value, SH = decltype(sh)::value;
        if (mode == MODE_FUSED && ND == 2) {
            auto k = push_deposit_2d_kernel<SH>;
            const size_t smem = SMEM_2D * sizeof(float);
            static bool configured = false;
            if (!configured) {
                cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e != cudaSuccess) return e;
                configured = true;
            }
            k<<<pblocks(extent), FUSED_T, smem, s>>>(g, sp, E, B, J, shift);
        } else if (mode == MODE_FUSED) {
            auto k = push_deposit_3d_kernel<SH>;
            const size_t smem = SMEM_3D * sizeof(float);
            static bool configured = false;
            if (!configured) {
                cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e != cudaSuccess) return e;
                configured = true;
            }
            // two lists of deferred chunks, each 2 + ceil(cap / FUSED_T) ints
            int* defer2 = defer + 2 + (sp.cap + FUSED_T - 1) / FUSED_T;
            k<<<pblocks(extent), FUSED_T, smem, s>>>(g, sp, E, B, J, shift, defer, defer2);
            // the deferred chunks: a fixed grid (their count is on the device)
            auto kd = push_deposit_3d_deferred_kernel<SH>;
            const size_t smem_d = SMEM_3D_GEN * sizeof(float);
            static bool configured_d = false;
            if (!configured_d) {
                cudaError_t e = cudaFuncSetAttribute(kd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_d);
                if (e != cudaSuccess) return e;
                configured_d = true;
            }
            const long long nchunk = (extent + FUSED_T - 1) / FUSED_T;
            const unsigned nb = (unsigned)(nchunk < 152 * 2 ? (nchunk < 1 ? 1 : nchunk) : 152 * 2);
            kd<<<nb, FUSED_T, smem_d, s>>>(g, sp, E, B, J, shift, defer);
            const unsigned nb2 = (unsigned)(nchunk < 152 * 4 ? (nchunk < 1 ? 1 : nchunk) : 152 * 4);
            push_deposit_3d_particles_kernel<SH><<<nb2, FUSED_T, 0, s>>>(g, sp, E, B, J, shift, defer2);
        } else {
            push_kernel<ND, SH><<<pblocks(extent), 256, 0, s>>>(g, sp, E, B, shift);
        }
        return cudaGetLastError();
    });
}

cudaError_t launch_push_batch(const PartInst* inst, int ninst, int ndim, int shape, long long max_extent, int parity,
                              cudaStream_t s) {
    if (ninst <= 0) return cudaSuccess;
    long long b = (max_extent + FUSED_T - 1) / FUSED_T;
    dim3 grid((unsigned)(b < 1 ? 1 : (b > 64 ? 64 : b)), (unsigned)ninst);
    return dispatch(ndim, shape, [&](auto nd, auto sh) {
        constexpr int ND = decltype(nd)::value, SH = decltype(sh)::value;
        if (ND == 2) {
            auto k = push_deposit_2d_batch_kernel<SH>;
            const size_t smem = SMEM_2D * sizeof(float);
            static bool configured = false;
            if (!configured) {
                cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e != cudaSuccess) return e;
                configured = true;
            }
            k<<<grid, FUSED_T, smem, s>>>(inst, parity);
            return cudaGetLastError();
        }
        auto k = push_deposit_3d_batch_kernel<SH>;
        const size_t smem = SMEM_3D * sizeof(float);
        static bool configured = false;
        if (!configured) {
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            configured = true;
        }
        k<<<grid, FUSED_T, smem, s>>>(inst, parity);
        return cudaGetLastError();
    });
}

cudaError_t launch_zero_j_batch(const PartInst* inst, int ninst, long long max_ncell, cudaStream_t s) {
    if (ninst <= 0) return cudaSuccess;
    long long b = (3 * max_ncell / 4 + 255) / 256;
    dim3 grid((unsigned)(b < 1 ? 1 : (b > 64 ? 64 : b)), (unsigned)ninst);
    zero_j_batch_kernel<<<grid, 256, 0, s>>>(inst);
    return cudaGetLastError();
}

cudaError_t launch_deposit_unfused(const GridP& g0, const SpeciesP& sp, float* J, long long extent,
                                   cudaStream_t s) {
    const GridP g = prep(g0);
    if (extent <= 0) return cudaSuccess;
    return dispatch(g.ndim, g.shape, [&](auto nd, auto sh) {
        constexpr int ND = decltype(nd)::value, SH = decltype(sh)::value;
        deposit_kernel<ND, SH><<<pblocks(extent), 256, 0, s>>>(g, sp, J);
        return cudaGetLastError();
    });
}

cudaError_t launch_inject(const GridP& g, const SpeciesP& sp, const int ppc[3], long long next_id,
                          int* status, long long* extent, cudaStream_t s) {
    int pz = ppc[0], px = ppc[1], py = g.ndim == 3 ? ppc[2] : 1;
    const long long P = (long long)pz * px * py;
    long long nnew = (long long)g.nx * (g.ndim == 3 ? g.ny : 1) * P;
    if (nnew <= 0) return cudaSuccess;
    // 2D: one patch per row, no alignment (the canonical order); 3D: the largest power-of-two
    // patch, x side >= y side, whose particles fill at most one 256-particle chunk
    int pxc = g.nx, pyc = 1, align = 1;
    if (g.ndim == 3) {
        pxc = 1;
        align = FUSED_T;
        for (;;) {
            const bool gx = 2 * pxc <= g.nx, gy = 2 * pyc <= g.ny;
            if (2 * pxc * pyc * P > FUSED_T || (!gx && !gy)) break;
            if (gx && (pxc <= pyc || !gy)) pxc *= 2;
            else pyc *= 2;
        }
    }
    inject_kernel<<<nblocks(nnew + align - 1, 256), 256, 0, s>>>(g, sp, pz, px, py, pxc, pyc, align, nnew, next_id,
                                                                 status);
    add_count_kernel<<<1, 1, 0, s>>>(sp.count, nnew, align, sp.cap);
    const long long ext = (*extent + align - 1) / align * align + nnew;
    *extent = ext < sp.cap ? ext : sp.cap;
    return cudaGetLastError();
}

long long sort_bins(const GridP& g) {
    if (g.ndim == 3) return (long long)((g.ny + 3) / 4) * ((g.nx + 3) / 4) * ((g.nzg + 3) / 4) * 64;
    return (long long)g.ny * ((g.nx + 7) / 8) * ((g.nzg + 7) / 8) * 64;
}

cudaError_t launch_sort(const GridP& g0, const SpeciesP& sp, long long extent, int32_t* hist,
                        int32_t* blocksums, int32_t* cell_alt, float* off_alt, float* u_alt,
                        int32_t* id_alt, cudaStream_t s) {
    if (extent <= 0) return cudaSuccess;
    const GridP g = prep(g0);
    const long long nb = sort_bins(g);
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(int32_t) * nb, s);
    if (e != cudaSuccess) return e;
    hist_kernel<<<pblocks(extent), 256, 0, s>>>(g, sp, hist);
    long long nblk = (nb + SCAN_B - 1) / SCAN_B;
    scan_blocks_kernel<<<(unsigned)nblk, SCAN_T, 0, s>>>(hist, nb, blocksums);
    scan_sums_kernel<<<1, SCAN_T, 0, s>>>(blocksums, nblk);
    add_block_offsets_kernel<<<nblocks(nb, 256), 256, 0, s>>>(hist, nb, blocksums);
    if (g.ndim == 2)
        scatter_kernel<2><<<pblocks(extent), 256, 0, s>>>(g, sp, hist, cell_alt, off_alt, u_alt,
                                                               sp.id ? id_alt : nullptr);
    else
        scatter_kernel<3><<<pblocks(extent), 256, 0, s>>>(g, sp, hist, cell_alt, off_alt, u_alt,
                                                               sp.id ? id_alt : nullptr);
    if (g.ndim == 2)
        copy_back_kernel<2><<<pblocks(extent), 256, 0, s>>>(sp, blocksums + nblk, cell_alt, off_alt, u_alt,
                                                             sp.id ? id_alt : nullptr);
    else
        copy_back_kernel<3><<<pblocks(extent), 256, 0, s>>>(sp, blocksums + nblk, cell_alt, off_alt, u_alt,
                                                             sp.id ? id_alt : nullptr);
    set_count_kernel<<<1, 1, 0, s>>>(sp.count, blocksums + nblk);
    return cudaGetLastError();
}

cudaError_t launch_rho(const GridP& g0, const SpeciesP& sp, int shift, double* rho, long long extent,
                       cudaStream_t s) {
    const GridP g = prep(g0);
    if (extent <= 0) return cudaSuccess;
    return dispatch(g.ndim, g.shape, [&](auto nd, auto sh) {
        constexpr int ND = decltype(nd)::value, SH = decltype(sh)::value;
        rho_kernel<ND, SH><<<pblocks(extent), 256, 0, s>>>(g, sp, shift, rho);
        return cudaGetLastError();
    });
}

}  // namespace pic
