// Database construction kernels (environment modelling, §3; the
// geo-referenced index -> floor-plan table and its 30 cm tiles, §3.2):
// finiteness check, subspace gather, floor-plan tiles, coarse prefix slab and
// the per-row scaled BF16 / FP8-e4m3 copies with their norms.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <math.h>

#include "common.cuh"
#include "internal.h"

namespace lhr {
namespace {

__global__ void check_finite_kernel(const float* x, int64_t count, int32_t* flag) {
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        bad |= !isfinite(x[i]);
    if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

__global__ void gather_rows_kernel(const float* src, const int32_t* perm, int64_t n, int d4, float* dst) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n * d4; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / d4, c = i % d4;
        reinterpret_cast<float4*>(dst)[r * d4 + c] = reinterpret_cast<const float4*>(src)[(int64_t)perm[r] * d4 + c];
    }
}

// tx = floor(x / t), ty = floor(y / t) with IEEE double divide; flags
// non-finite coordinates and tiles outside int32.
__global__ void tiles_kernel(const double* xy, int64_t n, double t, int32_t* tile, int32_t* flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < 2 * n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = xy[i];
        const double f = floor(v / t);
        if (!isfinite(v) || !(f >= -2147483648.0 && f <= 2147483647.0)) {
            atomicOr(flag, 2);
            tile[i] = 0;
        } else {
            tile[i] = (int32_t)f;
        }
    }
}

__global__ void coarse_slab_kernel(const float* X, int64_t n, int d4, int dc4, float* Xc) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n * dc4; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / dc4, c = i % dc4;
        reinterpret_cast<float4*>(Xc)[r * dc4 + c] = reinterpret_cast<const float4*>(X)[r * d4 + c];
    }
}

// One warp per row: scale s = amax / qmax (binary32 divide), code =
// round-to-nearest-even(x / s) in the target format (FP8 saturating), and the
// FP32 norm s^2 * sum(code^2) of the quantised row.
template <bool kFp8>
__global__ void quantize_kernel(const float* X, int64_t n, int D, void* codes, float2* sn) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const float qmax = kFp8 ? 448.0f : 1.0f;
    for (int64_t r = wid; r < n; r += nw) {
        const float* x = X + r * D;
        float amax = 0.f;
        for (int j = lane; j < D; j += 32) amax = fmaxf(amax, fabsf(x[j]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(kFull, amax, o));
        const float s = amax > 0.f ? __fdiv_rn(amax, qmax) : 1.0f;
        float acc = 0.f;
        for (int j = lane; j < D; j += 32) {
            const float v = __fdiv_rn(x[j], s);
            float c;
            if (kFp8) {
                const __nv_fp8_storage_t b = __nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
                reinterpret_cast<__nv_fp8_storage_t*>(codes)[r * D + j] = b;
                const __half_raw hr = __nv_cvt_fp8_to_halfraw(b, __NV_E4M3);
                c = __half2float(__half(hr));
            } else {
                const __nv_bfloat16 b = __float2bfloat16_rn(v);
                reinterpret_cast<__nv_bfloat16*>(codes)[r * D + j] = b;
                c = __bfloat162float(b);
            }
            acc = fmaf(c, c, acc);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
        if (lane == 0) sn[r] = make_float2(s, s * s * acc);
    }
}

// One warp per row: FP32 squared norm, and the running maximum (as float
// bits, order-preserving for non-negative values).
__global__ void norms_kernel(const float* X, int64_t n, int D, float* norm, unsigned* max_bits) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned mx = 0u;
    for (int64_t r = wid; r < n; r += nw) {
        const float* x = X + r * D;
        float acc = 0.f;
        for (int j = lane; j < D; j += 32) acc = fmaf(x[j], x[j], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
        if (lane == 0) norm[r] = acc;
        mx = max(mx, __float_as_uint(acc));
    }
    if (lane == 0) atomicMax(max_bits, mx);
}

// Rows 0, stride, 2 stride, ... of a code array (row_bytes % 16 == 0) and of
// its (s, norm) pairs.
__global__ void sample_rows_kernel(const uint4* codes, const float2* sn, int64_t ns, int stride, int row_u4,
                                   uint4* codes_s, float2* sn_s) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ns * row_u4;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / row_u4, c = i % row_u4;
        codes_s[i] = codes[r * stride * row_u4 + c];
        if (c == 0) sn_s[r] = sn[r * stride];
    }
}

// FP32 rows 0, stride, 2 stride, ...
__global__ void pilot_rows_kernel(const float4* X, int64_t ns, int stride, int row_f4, float4* Xp) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ns * row_f4;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / row_f4, c = i % row_f4;
        Xp[i] = X[r * stride * row_f4 + c];
    }
}

// max |x| over count values (count % 4 == 0) into *max_bits (float bits of a
// non-negative value, so unsigned order is float order).
__global__ void absmax_kernel(const float4* X, int64_t count4, unsigned* max_bits) {
    float m = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count4; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 v = X[i];
        m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(max_bits, __float_as_uint(m));
}

// Xh = fp16(x * 2^(15 - e)), round to nearest, for max |x| = f 2^e, f in [0.5, 1).
__global__ void half_copy_kernel(const float4* X, int64_t count4, const unsigned* max_bits, __half2* Xh) {
    int ex = 0;
    frexpf(__uint_as_float(*max_bits), &ex);
    const float sc = ldexpf(1.0f, 15 - ex);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count4; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 v = X[i];
        Xh[2 * i] = __floats2half2_rn(v.x * sc, v.y * sc);
        Xh[2 * i + 1] = __floats2half2_rn(v.z * sc, v.w * sc);
    }
}

int grid_for(int64_t work, int sms) {
    const int64_t b = (work + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)sms * 8));
}

}  // namespace

cudaError_t launch_check_finite(const float* x, int64_t count, int32_t* flag, cudaStream_t stream) {
    check_finite_kernel<<<grid_for(count, 152), 256, 0, stream>>>(x, count, flag);
    return cudaGetLastError();
}

cudaError_t launch_gather_rows(const float* src, const int32_t* perm, int64_t n, int dim, float* dst,
                               cudaStream_t stream) {
    gather_rows_kernel<<<grid_for(n * (dim / 4), 152), 256, 0, stream>>>(src, perm, n, dim / 4, dst);
    return cudaGetLastError();
}

cudaError_t launch_tiles(const double* xy, int64_t n, double t, int32_t* tile, int32_t* flag, cudaStream_t stream) {
    tiles_kernel<<<grid_for(2 * n, 152), 256, 0, stream>>>(xy, n, t, tile, flag);
    return cudaGetLastError();
}

cudaError_t launch_norms(const lhr_db* db, unsigned* max_bits, cudaStream_t stream) {
    const int grid = (int)std::min<int64_t>((db->n + 7) / 8, (int64_t)db->sms * 16);
    norms_kernel<<<grid, 256, 0, stream>>>(db->X, db->n, db->dim, db->xnorm, max_bits);
    return cudaGetLastError();
}

cudaError_t launch_pilot_sample(const lhr_db* db, cudaStream_t stream) {
    if (!db->Xp) return cudaSuccess;
    const int row_f4 = db->dim / 4;
    pilot_rows_kernel<<<grid_for(db->n_pilot * row_f4, db->sms), 256, 0, stream>>>(
        reinterpret_cast<const float4*>(db->X), db->n_pilot, kSampleStride, row_f4, reinterpret_cast<float4*>(db->Xp));
    return cudaGetLastError();
}

cudaError_t launch_half_copy(const lhr_db* db, unsigned* absmax_bits, cudaStream_t stream) {
    if (!db->Xh) return cudaSuccess;
    const int64_t count4 = db->n * (int64_t)db->dim / 4;
    absmax_kernel<<<grid_for(count4, db->sms), 256, 0, stream>>>(reinterpret_cast<const float4*>(db->X), count4,
                                                                 absmax_bits);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    half_copy_kernel<<<grid_for(count4, db->sms), 256, 0, stream>>>(reinterpret_cast<const float4*>(db->X), count4,
                                                                    absmax_bits, reinterpret_cast<__half2*>(db->Xh));
    return cudaGetLastError();
}

cudaError_t launch_build_derived(lhr_db* db, cudaStream_t stream) {
    cudaError_t e;
    if (db->Xc) {
        coarse_slab_kernel<<<grid_for(db->n * (db->coarse_dim / 4), db->sms), 256, 0, stream>>>(
            db->X, db->n, db->dim / 4, db->coarse_dim / 4, db->Xc);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const int qgrid = (int)std::min<int64_t>((db->n + 7) / 8, (int64_t)db->sms * 16);
    if (db->Xb) {
        quantize_kernel<false><<<qgrid, 256, 0, stream>>>(db->X, db->n, db->dim, db->Xb, db->snb);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (db->X8) {
        quantize_kernel<true><<<qgrid, 256, 0, stream>>>(db->X, db->n, db->dim, db->X8, db->sn8);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (db->Xb_s) {
        const int row_u4 = db->dim * 2 / 16;
        sample_rows_kernel<<<grid_for(db->n_sample * row_u4, db->sms), 256, 0, stream>>>(
            reinterpret_cast<const uint4*>(db->Xb), db->snb, db->n_sample, db->sample_stride, row_u4,
            reinterpret_cast<uint4*>(db->Xb_s), db->snb_s);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (db->X8_s) {
        const int row_u4 = db->dim / 16;
        sample_rows_kernel<<<grid_for(db->n_sample * row_u4, db->sms), 256, 0, stream>>>(
            reinterpret_cast<const uint4*>(db->X8), db->sn8, db->n_sample, db->sample_stride, row_u4,
            reinterpret_cast<uint4*>(db->X8_s), db->sn8_s);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace lhr
