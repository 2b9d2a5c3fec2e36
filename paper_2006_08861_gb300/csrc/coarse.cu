// Coarse-to-fine retrieval: a prefix of the feature scored over every row,
// an S-row shortlist per frame, the full feature re-scored on the shortlist,
// top N of those. (The paper scores full features, §3.1; the prefix level is
// this library's hierarchical form. The FFT-magnitude feature of §3 puts its
// low frequencies first, which is what a prefix keeps.)
//
// Kernel 1 (coarse_kernel): one thread per row (grid-stride) computes the
//   squared prefix distance to up to 8 frames with packed FP32 FMAs, writes it
//   to scratch (frames x n floats, L2-resident at building scale) and counts
//   the distance's top 11 value bits into a per-frame 2048-bin histogram
//   (shared-memory bins, flushed once per CTA).
// Kernel 2 (shortlist_kernel): one CTA per frame. The candidate key is
//   (prefix distance bits << 32 | row); the S-th smallest key is located by a
//   radix select that starts from kernel 1's histogram and refines by further
//   11-bit digits only while the boundary bin holds more than kBinCap keys.
//   One pass then collects every key below the boundary bin plus the boundary
//   bin itself, which is sorted (bitonic, shared memory) to take exactly S.
//   The S rows are re-scored on the full feature (warp per row) and each warp
//   keeps a register top-k list; 32 lists merge into the frame's result.
#include "common.cuh"
#include "internal.h"

namespace lhr {
namespace {

constexpr int kFB = 8;           // frames per coarse CTA
constexpr int kBins = 2048;      // 11-bit digits
constexpr int kBinCap = 4096;    // boundary-bin keys sorted in shared memory
constexpr int kSelThreads = 1024;
constexpr int kMaxShortlist = 4096;

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

template <int DC4>
__global__ void __launch_bounds__(256) coarse_kernel(const float* __restrict__ Xc, int64_t n, int dc,
                                                     const float* __restrict__ Q, int qld, int nq,
                                                     float* __restrict__ dcout, unsigned* __restrict__ hist) {
    extern __shared__ __align__(16) unsigned char csm[];
    float4(*qs)[DC4] = reinterpret_cast<float4(*)[DC4]>(csm);
    unsigned(*h)[kBins] = reinterpret_cast<unsigned(*)[kBins]>(csm + sizeof(float4) * kFB * DC4);
    const int f0 = blockIdx.y * kFB;
    const int nf = min(kFB, nq - f0);
    const int d4 = dc / 4;
    for (int i = threadIdx.x; i < kFB * DC4; i += blockDim.x) {
        const int f = i / DC4, c = i % DC4;
        qs[f][c] = (f < nf && c < d4) ? reinterpret_cast<const float4*>(Q + (size_t)(f0 + f) * qld)[c]
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int i = threadIdx.x; i < kFB * kBins; i += blockDim.x) (&h[0][0])[i] = 0u;
    __syncthreads();
    const float2 neg1 = f2(-1.f, -1.f);
    for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < n;
         row += (int64_t)gridDim.x * blockDim.x) {
        float4 x[DC4];
        const float4* xr = reinterpret_cast<const float4*>(Xc + row * dc);
#pragma unroll
        for (int c = 0; c < DC4; ++c) x[c] = c < d4 ? __ldg(xr + c) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int f = 0; f < kFB; ++f) {
            if (f < nf) {
                float2 acc = f2(0.f, 0.f);
#pragma unroll
                for (int c = 0; c < DC4; ++c) {
                    const float4 qv = qs[f][c];
                    float2 a = __ffma2_rn(f2(x[c].x, x[c].y), neg1, f2(qv.x, qv.y));
                    float2 b = __ffma2_rn(f2(x[c].z, x[c].w), neg1, f2(qv.z, qv.w));
                    acc = __ffma2_rn(a, a, acc);
                    acc = __ffma2_rn(b, b, acc);
                }
                const float d = acc.x + acc.y;
                dcout[(size_t)(f0 + f) * n + row] = d;
                atomicAdd(&h[f][__float_as_uint(d) >> 20], 1u);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nf * kBins; i += blockDim.x) {
        const unsigned v = (&h[0][0])[i];
        if (v) atomicAdd(&hist[(size_t)(f0 + i / kBins) * kBins + (i % kBins)], v);
    }
}

// Block-wide exclusive scan helper: finds the bin holding the `need`-th
// smallest key. Writes (bin, keys below it, keys in it) to out[0..2].
__device__ void find_bin(const unsigned* hsm, unsigned need, unsigned* out, unsigned* tmp) {
    // 2048 bins over 1024 threads: two bins per thread.
    const int t = threadIdx.x;
    const unsigned a = hsm[2 * t], b = hsm[2 * t + 1];
    unsigned s = a + b;
    // inclusive scan of s over the block
    const int lane = t & 31, w = t >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned v = __shfl_up_sync(kFull, s, o);
        if (lane >= o) s += v;
    }
    if (lane == 31) tmp[w] = s;
    __syncthreads();
    if (w == 0) {
        unsigned v = tmp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned u = __shfl_up_sync(kFull, v, o);
            if (lane >= o) v += u;
        }
        tmp[lane] = v;
    }
    __syncthreads();
    const unsigned before = (w > 0 ? tmp[w - 1] : 0u) + s - (a + b);  // exclusive prefix of bin 2t
    if (before < need && need <= before + a) {
        out[0] = 2 * t;
        out[1] = before;
        out[2] = a;
    } else if (before + a < need && need <= before + a + b) {
        out[0] = 2 * t + 1;
        out[1] = before + a;
        out[2] = b;
    }
    __syncthreads();
}

__device__ __forceinline__ u64 coarse_key(const float* dcf, int64_t row) {
    return ((u64)__float_as_uint(dcf[row]) << 32) | (u64)row;
}

template <int CPL>
__global__ void __launch_bounds__(kSelThreads, 1)
    shortlist_kernel(const float* __restrict__ X, int D, int64_t n, const float* __restrict__ Q, int nq,
                     const float* __restrict__ dcall, const unsigned* __restrict__ hist, int S, int k,
                     int64_t* __restrict__ idx, float* __restrict__ dist) {
    extern __shared__ __align__(16) unsigned char smem[];
    u64* bin_keys = reinterpret_cast<u64*>(smem);                       // kBinCap
    int* short_rows = reinterpret_cast<int*>(bin_keys + kBinCap);       // kMaxShortlist
    unsigned* hsm = reinterpret_cast<unsigned*>(short_rows + kMaxShortlist);  // kBins
    u64* wl = reinterpret_cast<u64*>(hsm + kBins);                      // 32 warps x 32
    unsigned* ctl = reinterpret_cast<unsigned*>(wl + 32 * 32);          // control words
    unsigned* tmp = ctl + 8;                                            // 32 scan partials

    const int f = blockIdx.x;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const float* dcf = dcall + (size_t)f * n;
    const int sel = (int)((int64_t)S < n ? (int64_t)S : n);

    u64 lo = 0, hi = 0;         // boundary bin [lo, hi) of keys
    unsigned need = (unsigned)sel;
    bool take_all = (n <= S);
    if (!take_all) {
        for (int i = t; i < kBins; i += blockDim.x) hsm[i] = hist[(size_t)f * kBins + i];
        __syncthreads();
        find_bin(hsm, need, ctl, tmp);
        int shift = 52;
        lo = (u64)ctl[0] << shift;
        hi = lo + (1ull << shift);
        need -= ctl[1];
        unsigned in_bin = ctl[2];
        while (in_bin > (unsigned)kBinCap && shift > 0) {
            const int nshift = shift >= 11 ? shift - 11 : 0;
            const int dbits = shift - nshift;
            __syncthreads();
            for (int i = t; i < kBins; i += blockDim.x) hsm[i] = 0u;
            __syncthreads();
            for (int64_t r = t; r < n; r += blockDim.x) {
                const u64 key = coarse_key(dcf, r);
                if (key >= lo && key < hi)
                    atomicAdd(&hsm[(unsigned)((key >> nshift) & ((1ull << dbits) - 1))], 1u);
            }
            __syncthreads();
            find_bin(hsm, need, ctl, tmp);
            lo += (u64)ctl[0] << nshift;
            hi = lo + (1ull << nshift);
            need -= ctl[1];
            in_bin = ctl[2];
            shift = nshift;
        }
    }
    // Collection pass.
    if (t == 0) {
        ctl[4] = 0u;  // rows taken directly
        ctl[5] = 0u;  // keys in the boundary bin
    }
    __syncthreads();
    for (int64_t r = t; r < n; r += blockDim.x) {
        const u64 key = coarse_key(dcf, r);
        if (take_all || key < lo) {
            const unsigned pos = atomicAdd(&ctl[4], 1u);
            short_rows[pos] = (int)r;
        } else if (key < hi) {
            const unsigned pos = atomicAdd(&ctl[5], 1u);
            if (pos < (unsigned)kBinCap) bin_keys[pos] = key;
        }
    }
    __syncthreads();
    const unsigned direct = ctl[4];
    if (!take_all) {
        const unsigned nb = min(ctl[5], (unsigned)kBinCap);
        unsigned p2 = 1;
        while (p2 < nb) p2 <<= 1;
        for (unsigned i = nb + t; i < p2; i += blockDim.x) bin_keys[i] = kKeyEmpty;
        __syncthreads();
        // bitonic sort of bin_keys[0, p2)
        for (unsigned size = 2; size <= p2; size <<= 1) {
            for (unsigned stride = size >> 1; stride > 0; stride >>= 1) {
                for (unsigned i = t; i < p2 / 2; i += blockDim.x) {
                    const unsigned lo_i = 2 * i - (i & (stride - 1));
                    const unsigned hi_i = lo_i + stride;
                    const bool up = ((lo_i & size) == 0);
                    const u64 a = bin_keys[lo_i], b = bin_keys[hi_i];
                    if ((a > b) == up) {
                        bin_keys[lo_i] = b;
                        bin_keys[hi_i] = a;
                    }
                }
                __syncthreads();
            }
        }
        for (unsigned i = t; i < need; i += blockDim.x) short_rows[direct + i] = (int)key_row(bin_keys[i]);
        __syncthreads();
    }
    const int total = take_all ? (int)direct : (int)(direct + need);

    // Re-rank on the full feature: warp per shortlisted row.
    const int D4 = D / 4;
    float4 qv[CPL];
#pragma unroll
    for (int j = 0; j < CPL; ++j) {
        const int c = lane + 32 * j;
        qv[j] = c < D4 ? reinterpret_cast<const float4*>(Q + (size_t)f * D)[c] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const float2 neg1 = f2(-1.f, -1.f);
    u64 L = kKeyEmpty;
    u64 thr = kKeyEmpty;
    for (int i = warp; i < total; i += kSelThreads / 32) {
        const int r = short_rows[i];
        const float4* xr = reinterpret_cast<const float4*>(X + (size_t)r * D);
        float2 acc = f2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < CPL; ++j) {
            const int c = lane + 32 * j;
            if (c < D4) {
                const float4 x = __ldg(xr + c);
                float2 a = __ffma2_rn(f2(x.x, x.y), neg1, f2(qv[j].x, qv[j].y));
                float2 b = __ffma2_rn(f2(x.z, x.w), neg1, f2(qv[j].z, qv[j].w));
                acc = __ffma2_rn(a, a, acc);
                acc = __ffma2_rn(b, b, acc);
            }
        }
        float d = acc.x + acc.y;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(kFull, d, o);
        const u64 key = make_key(d, (uint32_t)r);
        if (key < thr) {
            list_insert(L, key, k, lane);
            thr = __shfl_sync(kFull, L, k - 1);
        }
    }
    wl[warp * 32 + lane] = L;
    __syncthreads();
    if (warp == 0) {
        u64 M = kKeyEmpty;
        list_merge_keys<false>(M, wl, 32 * 32, k, lane);
        if (lane < k) {
            const size_t o = (size_t)f * k + lane;
            if (M == kKeyEmpty) {
                idx[o] = -1;
                dist[o] = __int_as_float(0x7f800000);
            } else {
                idx[o] = (int64_t)key_row(M);
                dist[o] = key_dist(M);
            }
        }
    }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t shortlist_smem() {
    return kBinCap * sizeof(u64) + kMaxShortlist * sizeof(int) + kBins * sizeof(unsigned) + 32 * 32 * sizeof(u64) +
           (8 + 32) * sizeof(unsigned);
}

}  // namespace

size_t coarse_scratch_bytes(const lhr_db* db, int nq, int /*shortlist*/) {
    return align256((size_t)nq * db->n * sizeof(float)) + align256((size_t)nq * kBins * sizeof(unsigned));
}

cudaError_t launch_coarse(const lhr_db* db, const float* q, int nq, int shortlist, int k, int64_t* idx, float* dist,
                          void* scratch, cudaStream_t stream) {
    float* dcbuf = reinterpret_cast<float*>(scratch);
    unsigned* hist = reinterpret_cast<unsigned*>(reinterpret_cast<unsigned char*>(scratch) +
                                                 align256((size_t)nq * db->n * sizeof(float)));
    cudaError_t e = cudaMemsetAsync(hist, 0, (size_t)nq * kBins * sizeof(unsigned), stream);
    if (e != cudaSuccess) return e;
    const int64_t nblk = (db->n + 255) / 256;
    dim3 g1((unsigned)std::min<int64_t>(nblk, (int64_t)db->sms * 2), (nq + kFB - 1) / kFB);
    const int dc4 = db->coarse_dim / 4;
#define LHR_CK(C)                                                                                           \
    do {                                                                                                    \
        const size_t csm = sizeof(float4) * kFB * (C) + sizeof(unsigned) * kFB * kBins;                     \
        e = cudaFuncSetAttribute(coarse_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm);  \
        if (e != cudaSuccess) return e;                                                                     \
        ProfScope ps("coarse_kernel", stream);                                                              \
        coarse_kernel<C><<<g1, 256, csm, stream>>>(db->Xc, db->n, db->coarse_dim, q, db->dim, nq, dcbuf, hist); \
    } while (0)
    if (dc4 <= 8) LHR_CK(8);
    else if (dc4 <= 16) LHR_CK(16);
    else if (dc4 <= 32) LHR_CK(32);
    else return cudaErrorInvalidValue;
#undef LHR_CK
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t sm = shortlist_smem();
    const int d4 = db->dim / 4;
    const int cpl = d4 <= 32 ? 1 : (d4 <= 64 ? 2 : 4);
#define LHR_SL(C)                                                                                            \
    do {                                                                                                     \
        e = cudaFuncSetAttribute(shortlist_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
        if (e != cudaSuccess) return e;                                                                      \
        ProfScope ps("shortlist_kernel", stream);                                                            \
        shortlist_kernel<C><<<nq, kSelThreads, sm, stream>>>(db->X, db->dim, db->n, q, nq, dcbuf, hist,     \
                                                             shortlist, k, idx, dist);                       \
    } while (0)
    if (cpl == 1) LHR_SL(1);
    else if (cpl == 2) LHR_SL(2);
    else LHR_SL(4);
#undef LHR_SL
    return cudaGetLastError();
}

}  // namespace lhr
