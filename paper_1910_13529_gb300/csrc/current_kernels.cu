// Current post-processing along z, in place, between the deposit and the field advance:
//
//  * the current filter: the "5 pass filter" the paper runs with (Sec. 2.2, 2.3, Table 2) and
//    names without defining.  Four binomial passes (1/4, 1/2, 1/4) and one compensating pass
//    (-5/4, 7/2, -5/4); each pass is y_i = w1 (x_{i-1} + x_{i+1}) + w0 x_i over 0 <= i < nz with
//    x = 0 outside that range (open z ends).  A Fourier mode is multiplied by
//    cos^8(k dz/2) (1 + 5 sin^2(k dz/2)).  It acts on J1, J2 and J3.
//  * the Sec. 3 current correction J1[i] <- sum_{|m| <= hlen} h[m] J1[i - m] (J1 = 0 outside
//    0 <= i < nz), h the impulse response of 1/P, for the customised stencil.
//  * both in one launch when both are configured: J1 rows are filtered into shared memory and
//    corrected from there; J2 and J3 rows are filtered.
//
// Filter, one CTA per z row.  The CTA walks the row in segments of SEG = 8 NT cells:
//   * the segment's inputs z in [base - 8, base + SEG + 8) are staged in shared memory (16-byte
//     loads when the row allows); the 16 leftmost were read by the previous segment and are carried
//     over in registers, because the previous segment has already overwritten them in HBM;
//   * thread t produces the eight outputs z = base + 8t .. base + 8t + 7 from the 24 staged inputs
//     z = base + 8t - 8 .. base + 8t + 15 (six aligned 128-bit shared loads) and runs the five passes
//     in registers, each pass on the cells the remaining passes still need (16, 14, 12, 10, 8);
//   * cells outside 0 <= z < nz are zero after every pass, so a pass near the ends sees exactly the
//     truncated row.
// HBM traffic: one read and one write of the row (8 bytes per FP32 cell).
//
// Correction, one CTA per z row: the whole row sits in shared memory, so no other CTA reads the
// values it overwrites.  Each thread produces four consecutive outputs from the
// (2 PIC_MAX_HLEN + 4)-float window below them, read as aligned 128-bit shared loads (taps beyond
// hlen are zero).
#include <cuda_runtime.h>

#include "pic_internal.h"

namespace pic {
namespace {

// ------------------------------------------------------------------------------- filter ---

template <typename T, bool EDGE>
__device__ __forceinline__ void five_passes(T (&w)[24], int z0, int nz) {
#pragma unroll
    for (int p = 0; p < 5; ++p) {
        const T a = p < 4 ? T(0.25) : T(-1.25);
        const T c = p < 4 ? T(0.5) : T(3.5);
        // pass p is needed on window cells [4 + p, 20 - p): the final pass on the eight outputs [8, 16)
        T v[24];
#pragma unroll
        for (int k = 4 + p; k < 20 - p; ++k) {
            T y = a * (w[k - 1] + w[k + 1]) + c * w[k];
            if (EDGE) {
                const int z = z0 + k;
                y = (z >= 0 && z < nz) ? y : T(0);
            }
            v[k] = y;
        }
#pragma unroll
        for (int k = 4 + p; k < 20 - p; ++k) w[k] = v[k];
    }
}

template <typename T>
__device__ __forceinline__ void load_window(const T* s, T (&w)[24]) {
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const float4 v = reinterpret_cast<const float4*>(s)[q];
            w[4 * q] = v.x;
            w[4 * q + 1] = v.y;
            w[4 * q + 2] = v.z;
            w[4 * q + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            const double2 v = reinterpret_cast<const double2*>(s)[q];
            w[2 * q] = v.x;
            w[2 * q + 1] = v.y;
        }
    }
}

// Filters row[0, nz) into out[0, nz); out may be row itself (in place) or shared memory.
// buf: 8 NT + 16 elements, 16-byte aligned.  vec4: FP32 with nz % 4 == 0 and row, out 16-byte
// aligned.  Ends with a barrier, so out is complete for the whole CTA on return.
template <typename T, int NT>
__device__ __forceinline__ void filter_row(const T* row, T* out, int nz, bool vec4, T* __restrict__ buf) {
    constexpr int SEG = 8 * NT;
    const int t = threadIdx.x;
    T carry = T(0);
    for (int base = 0; base < nz; base += SEG) {
        // buf[b] holds z = base - 8 + b
        if (t < 16) {
            const int z = base - 8 + t;
            buf[t] = base == 0 ? ((z >= 0 && z < nz) ? row[z] : T(0)) : carry;
        }
        if constexpr (sizeof(T) == 4) {
            if (vec4) {
                for (int q = t; q < SEG / 4; q += NT) {
                    const int z = base + 8 + 4 * q;
                    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (z < nz) v = *reinterpret_cast<const float4*>(row + z);
                    reinterpret_cast<float4*>(buf + 16)[q] = v;
                }
            } else {
                for (int q = t; q < SEG; q += NT) {
                    const int z = base + 8 + q;
                    buf[16 + q] = z < nz ? row[z] : T(0);
                }
            }
        } else {
            for (int q = t; q < SEG; q += NT) {
                const int z = base + 8 + q;
                buf[16 + q] = z < nz ? row[z] : T(0);
            }
        }
        __syncthreads();
        T w[24];
        load_window(buf + 8 * t, w);
        if (t < 16) carry = buf[SEG + t];   // z = base + SEG - 8 + t: the next segment's left inputs
        const int z0 = base + 8 * t - 8;    // z of w[0]
        if (z0 >= 0 && z0 + 24 <= nz)
            five_passes<T, false>(w, z0, nz);
        else
            five_passes<T, true>(w, z0, nz);
        const int zo = base + 8 * t;        // outputs w[8 .. 15]
        if constexpr (sizeof(T) == 4) {
            if (vec4 && zo < nz) {
                // nz % 4 == 0: zo < nz implies zo + 3 < nz
                *reinterpret_cast<float4*>(out + zo) = make_float4(w[8], w[9], w[10], w[11]);
                if (zo + 4 < nz) *reinterpret_cast<float4*>(out + zo + 4) = make_float4(w[12], w[13], w[14], w[15]);
            } else if (!vec4) {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (zo + j < nz) out[zo + j] = w[8 + j];
            }
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (zo + j < nz) out[zo + j] = w[8 + j];
        }
        __syncthreads();   // every window read before the next segment refills buf
    }
}

// --------------------------------------------------------------------------- correction ---

struct CorrP {
    GridP g;
    float h[2 * PIC_MAX_HLEN + 1];
    int hlen;
    float* J1;
};

constexpr int kHL = PIC_MAX_HLEN;
constexpr int kNWIN = 2 * kHL + 4;               // window floats (a multiple of 4: kHL even)
static_assert(kNWIN % 4 == 0, "aligned windows");
static_assert(kHL % 4 == 0, "s + kHL must be 16-byte aligned for the float4 filter stores");

// floats of the correction's shared row: s[k] = J1[k - kHL] for k < nz4 + kNWIN
__host__ __device__ constexpr int corr_floats(int nz) { return ((nz + 3) & ~3) + kNWIN; }

// row[i] <- sum_k h[k] s[i + 2 kHL - k], i < nz, from the staged row s; threads tid of nt share it
__device__ __forceinline__ void correct_from(const float* s, float* row, int nz, const float* __restrict__ h, int tid,
                                             int nt) {
    for (int i = 4 * tid; i < nz; i += 4 * nt) {
        float w[kNWIN];
#pragma unroll
        for (int q = 0; q < kNWIN / 4; ++q) {
            const float4 v = *reinterpret_cast<const float4*>(s + i + 4 * q);
            w[4 * q] = v.x;
            w[4 * q + 1] = v.y;
            w[4 * q + 2] = v.z;
            w[4 * q + 3] = v.w;
        }
        // out[i + j] = sum_m h[m + kHL] J1[i + j - m] = sum_k h[k] w[j + 2 kHL - k]
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k <= 2 * kHL; ++k)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[j] = fmaf(h[k], w[j + 2 * kHL - k], acc[j]);
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (i + j < nz) row[i + j] = acc[j];
    }
}

__device__ __forceinline__ void correct_from(const float* s, float* row, int nz, const float* __restrict__ h) {
    correct_from(s, row, nz, h, threadIdx.x, blockDim.x);
}

__device__ __forceinline__ void correct_row(float* row, int nz, const float* __restrict__ h, float* s) {
    for (int k = threadIdx.x; k < corr_floats(nz); k += blockDim.x) {
        const int gz = k - kHL;
        s[k] = (gz >= 0 && gz < nz) ? row[gz] : 0.f;
    }
    __syncthreads();
    correct_from(s, row, nz, h);
}

// Several rows per CTA: rows_per_cta groups of tpr threads (tpr a multiple of 32, 4 tpr >= nz for
// one pass); vec4: rows 16-byte aligned (nz % 4 == 0), staged with 16-byte loads.
__global__ void __launch_bounds__(256) correct_j1_rows_kernel(CorrP p, long long rows, int tpr, int vec4) {
    extern __shared__ float4 s4[];
    const int nz = p.g.nz, cf = corr_floats(nz);
    const int grp = threadIdx.x / tpr, tid = threadIdx.x - grp * tpr;
    const long long r = (long long)blockIdx.x * (blockDim.x / tpr) + grp;
    float* s = reinterpret_cast<float*>(s4) + grp * cf;
    float* row = p.J1 + r * nz;
    const bool live = r < rows;
    if (live) {
        if (vec4) {
            // s[kHL + 4 q .. +3] = row[4 q .. +3]; the kHL-float margins are zero
            for (int q = tid; q < (nz >> 2); q += tpr)
                *reinterpret_cast<float4*>(s + kHL + 4 * q) = *reinterpret_cast<const float4*>(row + 4 * q);
            for (int k = tid; k < kHL; k += tpr) s[k] = 0.f;
            for (int k = kHL + nz + tid; k < cf; k += tpr) s[k] = 0.f;
        } else {
            for (int k = tid; k < cf; k += tpr) {
                const int gz = k - kHL;
                s[k] = (gz >= 0 && gz < nz) ? row[gz] : 0.f;
            }
        }
    }
    __syncthreads();
    if (live) correct_from(s, row, nz, p.h, tid, tpr);
}

// ------------------------------------------------------------------------------ kernels ---

template <typename T, int NT>
__global__ void __launch_bounds__(NT) filter_z_kernel(T* f, int nz, int vec4) {
    __shared__ __align__(16) T buf[8 * NT + 16];
    T* row = f + (long long)blockIdx.x * nz;
    filter_row<T, NT>(row, row, nz, vec4 != 0, buf);
}

// Batched: blockIdx.y = instance, blockIdx.x = row among the instance's 3 nx ny current rows.
__global__ void __launch_bounds__(128) filter_z_batch_kernel(const FiltInst* __restrict__ inst) {
    __shared__ __align__(16) float buf[8 * 128 + 16];
    const FiltInst& q = inst[blockIdx.y];
    if ((long long)blockIdx.x >= 3LL * q.g.nx * q.g.ny) return;
    float* row = q.J + (long long)blockIdx.x * q.g.nz;
    filter_row<float, 128>(row, row, q.g.nz, q.vec4 != 0, buf);
}

// Batched in-place correction: blockIdx.y = instance, blockIdx.x = z row of that instance.
__global__ void __launch_bounds__(256) correct_j1_batch_kernel(const CorrInst* __restrict__ inst) {
    extern __shared__ float4 s4[];
    const CorrInst& q = inst[blockIdx.y];
    if ((long long)blockIdx.x >= (long long)q.g.nx * q.g.ny) return;
    correct_row(q.J1 + (long long)blockIdx.x * q.g.nz, q.g.nz, q.h, reinterpret_cast<float*>(s4));
}

// Filter and correction in one launch over the 3 nx ny rows of J (p.J1 = J): a J1 row is filtered
// into the correction's shared row and corrected from there into HBM (its HBM values are read
// once and written once); J2 and J3 rows are filtered in place.
template <int NT>
__global__ void __launch_bounds__(NT) filter_correct_kernel(CorrP p, int vec4) {
    extern __shared__ float4 s4[];
    __shared__ __align__(16) float buf[8 * NT + 16];
    const int nz = p.g.nz;
    float* row = p.J1 + (long long)blockIdx.x * nz;
    if ((long long)blockIdx.x >= (long long)p.g.nx * p.g.ny) {
        filter_row<float, NT>(row, row, nz, vec4 != 0, buf);
        return;
    }
    float* s = reinterpret_cast<float*>(s4);
    for (int k = threadIdx.x; k < kHL; k += NT) s[k] = 0.f;
    for (int k = kHL + nz + threadIdx.x; k < corr_floats(nz); k += NT) s[k] = 0.f;
    filter_row<float, NT>(row, s + kHL, nz, vec4 != 0, buf);   // ends with a barrier
    correct_from(s, row, nz, p.h);
}

// smallest CTA whose filter segment covers the row (one segment per row up to nz = 2048)
inline int filter_threads(int nz) { return nz <= 256 ? 32 : nz <= 512 ? 64 : nz <= 1024 ? 128 : 256; }

template <typename T>
cudaError_t launch_rows(T* f, int nz, long long rows, int vec4, cudaStream_t s) {
    if (rows <= 0) return cudaSuccess;
    switch (filter_threads(nz)) {
        case 32: filter_z_kernel<T, 32><<<(unsigned)rows, 32, 0, s>>>(f, nz, vec4); break;
        case 64: filter_z_kernel<T, 64><<<(unsigned)rows, 64, 0, s>>>(f, nz, vec4); break;
        case 128: filter_z_kernel<T, 128><<<(unsigned)rows, 128, 0, s>>>(f, nz, vec4); break;
        default: filter_z_kernel<T, 256><<<(unsigned)rows, 256, 0, s>>>(f, nz, vec4); break;
    }
    return cudaGetLastError();
}

template <int NT>
cudaError_t launch_fc(const CorrP& p, int vec4, cudaStream_t s) {
    const size_t smem = sizeof(float) * corr_floats(p.g.nz);
    // the default limit is 48 KB for static and dynamic shared memory together
    if (smem + sizeof(float) * (8 * NT + 16) > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(filter_correct_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    filter_correct_kernel<NT><<<(unsigned)(3LL * p.g.nx * p.g.ny), NT, smem, s>>>(p, vec4);
    return cudaGetLastError();
}

CorrP corr_params(const GridP& g, const float* taps, int hlen, float* J1) {
    CorrP p;
    p.g = g;
    p.hlen = hlen;
    // taps centred on PIC_MAX_HLEN: p.h[PIC_MAX_HLEN + m] = h[m], zero for |m| > hlen
    for (int i = 0; i < 2 * PIC_MAX_HLEN + 1; ++i) {
        const int m = i - PIC_MAX_HLEN;
        p.h[i] = (m >= -hlen && m <= hlen) ? taps[m + hlen] : 0.f;
    }
    p.J1 = J1;
    return p;
}

}  // namespace

bool filter_vec4_ok(const float* J, int nz) { return nz % 4 == 0 && ((uintptr_t)J & 15) == 0; }

cudaError_t launch_filter_current(const GridP& g, float* J, cudaStream_t s) {
    return launch_rows<float>(J, g.nz, 3LL * g.nx * g.ny, filter_vec4_ok(J, g.nz) ? 1 : 0, s);
}

cudaError_t launch_filter_rho(const GridP& g, double* rho, cudaStream_t s) {
    return launch_rows<double>(rho, g.nz, (long long)g.nx * g.ny, 0, s);
}

cudaError_t launch_filter_current_batch(const FiltInst* inst, int ninst, long long max_rows3, cudaStream_t s) {
    if (ninst <= 0 || max_rows3 <= 0) return cudaSuccess;
    filter_z_batch_kernel<<<dim3((unsigned)max_rows3, (unsigned)ninst), 128, 0, s>>>(inst);
    return cudaGetLastError();
}

cudaError_t launch_correct_j1(const GridP& g, const float* taps, int hlen, float* J1, cudaStream_t s) {
    CorrP p = corr_params(g, taps, hlen, J1);
    const long long rows = (long long)g.nx * g.ny;
    // threads per row: enough for one pass of four outputs each, in whole warps, at most 256
    int tpr = (((g.nz + 3) / 4) + 31) / 32 * 32;
    tpr = tpr > 256 ? 256 : tpr;
    const int rpc = 256 / tpr;
    const size_t smem = sizeof(float) * corr_floats(g.nz) * rpc;
    static size_t opted = 48 * 1024;
    if (smem > opted) {
        cudaError_t e = cudaFuncSetAttribute(correct_j1_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        opted = smem;
    }
    const int vec4 = (g.nz % 4 == 0 && ((uintptr_t)J1 & 15) == 0) ? 1 : 0;
    correct_j1_rows_kernel<<<(unsigned)((rows + rpc - 1) / rpc), rpc * tpr, smem, s>>>(p, rows, tpr, vec4);
    return cudaGetLastError();
}

cudaError_t launch_filter_correct(const GridP& g, const float* taps, int hlen, float* J, cudaStream_t s) {
    CorrP p = corr_params(g, taps, hlen, J);
    const int vec4 = filter_vec4_ok(J, g.nz) ? 1 : 0;
    switch (filter_threads(g.nz)) {
        case 32: return launch_fc<32>(p, vec4, s);
        case 64: return launch_fc<64>(p, vec4, s);
        case 128: return launch_fc<128>(p, vec4, s);
        default: return launch_fc<256>(p, vec4, s);
    }
}

cudaError_t launch_correct_j1_batch(const CorrInst* inst, int ninst, int max_rows, int max_nz, cudaStream_t s) {
    if (ninst <= 0) return cudaSuccess;
    const size_t smem = sizeof(float) * corr_floats(max_nz);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(correct_j1_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    correct_j1_batch_kernel<<<dim3((unsigned)max_rows, (unsigned)ninst), 256, smem, s>>>(inst);
    return cudaGetLastError();
}

}  // namespace pic
