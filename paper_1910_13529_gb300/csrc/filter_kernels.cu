// Current filter along z: the "5 pass filter" the paper runs with (Sec. 2.2, 2.3, Table 2) and
// names without defining.  Four binomial passes (1/4, 1/2, 1/4) and one compensating pass
// (-5/4, 7/2, -5/4); each pass is y_i = w1 (x_{i-1} + x_{i+1}) + w0 x_i over 0 <= i < nz with x = 0
// outside that range (open z ends).  A Fourier mode is multiplied by cos^8(k dz/2) (1 + 5 sin^2(k dz/2)).
//
// In place, one CTA per z row of one array.  The CTA walks the row in segments of SEG = 8 NT cells:
//   * the segment's inputs z in [base - 8, base + SEG + 8) are staged in shared memory (16-byte
//     loads when the row allows); the 16 leftmost were read by the previous segment and are carried
//     over in registers, because the previous segment has already overwritten them in HBM;
//   * thread t produces the eight outputs z = base + 8t .. base + 8t + 7 from the 24 staged inputs
//     z = base + 8t - 8 .. base + 8t + 15 (six aligned 128-bit shared loads) and runs the five passes
//     in registers, each pass on the cells the remaining passes still need (16, 14, 12, 10, 8);
//   * cells outside 0 <= z < nz are zero after every pass, so a pass near the ends sees exactly the
//     truncated row.
// HBM traffic: one read and one write of the row (8 bytes per FP32 cell).
#include <cuda_runtime.h>

#include "pic_internal.h"

namespace pic {
namespace {

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

// buf: 8 NT + 16 elements, 16-byte aligned.  vec4: FP32 row with nz % 4 == 0 and a 16-byte aligned start.
template <typename T, int NT>
__device__ __forceinline__ void filter_row(T* __restrict__ row, int nz, bool vec4, T* __restrict__ buf) {
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
                *reinterpret_cast<float4*>(row + zo) = make_float4(w[8], w[9], w[10], w[11]);
                if (zo + 4 < nz) *reinterpret_cast<float4*>(row + zo + 4) = make_float4(w[12], w[13], w[14], w[15]);
            } else if (!vec4) {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (zo + j < nz) row[zo + j] = w[8 + j];
            }
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (zo + j < nz) row[zo + j] = w[8 + j];
        }
        __syncthreads();   // every window read before the next segment refills buf
    }
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT) filter_z_kernel(T* f, int nz, int vec4) {
    __shared__ __align__(16) T buf[8 * NT + 16];
    filter_row<T, NT>(f + (long long)blockIdx.x * nz, nz, vec4 != 0, buf);
}

// Batched: blockIdx.y = instance, blockIdx.x = row among the instance's 3 nx ny current rows.
__global__ void __launch_bounds__(128) filter_z_batch_kernel(const FiltInst* __restrict__ inst) {
    __shared__ __align__(16) float buf[8 * 128 + 16];
    const FiltInst& q = inst[blockIdx.y];
    if ((long long)blockIdx.x >= 3LL * q.g.nx * q.g.ny) return;
    filter_row<float, 128>(q.J + (long long)blockIdx.x * q.g.nz, q.g.nz, q.vec4 != 0, buf);
}

template <typename T>
cudaError_t launch_rows(T* f, int nz, long long rows, int vec4, cudaStream_t s) {
    if (rows <= 0) return cudaSuccess;
    // smallest CTA whose segment covers the row (one segment per row up to nz = 2048)
    if (nz <= 8 * 32) filter_z_kernel<T, 32><<<(unsigned)rows, 32, 0, s>>>(f, nz, vec4);
    else if (nz <= 8 * 64) filter_z_kernel<T, 64><<<(unsigned)rows, 64, 0, s>>>(f, nz, vec4);
    else if (nz <= 8 * 128) filter_z_kernel<T, 128><<<(unsigned)rows, 128, 0, s>>>(f, nz, vec4);
    else filter_z_kernel<T, 256><<<(unsigned)rows, 256, 0, s>>>(f, nz, vec4);
    return cudaGetLastError();
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

}  // namespace pic
