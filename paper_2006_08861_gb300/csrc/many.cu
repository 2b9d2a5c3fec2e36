// Exhaustive per-frame top k for many query frames at once (the batched
// selection of the soft-retrieval form and the precision form's FP32 path),
// exact in FP32 like the streaming scan in scan.cu, which serves few frames.
//
// With F frames the streaming scan reduces every (row, frame) distance across
// the 32 lanes of a warp; with hundreds of frames that reduction costs as much
// as the multiply-adds. Here a CTA holds 64 frames (w * q, in shared memory)
// and streams its row chunk in 128-row tiles, K-chunked by 128 dimensions (64
// when D is not a multiple of 128; double-buffered cp.async); each thread
// owns an 8-frame x 4-row register
// tile of the expanded form
//     e(f, r) = ||x_r||_w^2 + ||q_f||_w^2 - 2 (w q_f) . x_r,
// so no cross-lane reduction is needed. A pair is a candidate when
// e <= bound_f + margin_f: bound_f is the pilot's upper bound on frame f's
// k-th exact distance (the k-th smallest of 128 bucket minima over the
// every-64th-row sample, widened 2^-12), and margin_f = 2 (gamma_{D+4} + 3u)
// (max ||x||_w + ||q_f||_w)^2 bounds |e - exact distance| (the streaming
// scan's filter margin). Candidates (orderable bits of e, row) are staged per
// frame in shared memory and appended to the frame's buffer.
// many_select_kernel, a warp per frame: with e_k the k-th smallest candidate
// e, every row of the exact top k has e <= e_k + 2 margin_f (k rows have exact
// distance <= e_k + margin_f); those rows are re-scored with the exact
// direct form sum w (q - x)^2 and the top k (distance, row) keys written. A
// frame whose buffer overflowed is scanned exhaustively by its warp.
#include <cuda_pipeline.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace lhr {
namespace {

constexpr int kMF = 64;        // frames per CTA
constexpr int kMRows = 128;    // rows per tile
constexpr int kMThreads = 256; // 8 frame groups x 32 row groups
constexpr int kMStage = 32;    // staged candidates per frame in shared memory
constexpr int kMCap = 8192;    // candidates per frame in global memory (about 64 k expected)
constexpr int kMBuckets = 128; // pilot bucket minima per frame

struct ManyParams {
    const float* X;       // n x D, internal row order
    const float* xn;      // n: ||x||_w^2 (||x||^2 without weights)
    int64_t n;
    int D;
    const float* Q;       // nq x D
    const float* w;       // D weights, nullable
    int nq, k;
    const unsigned* bmin; // nq x kMBuckets pilot bucket minima (float bits, ~0u empty)
    float margin_scale;
    float xmax;           // max ||x|| (unweighted), or
    const float* xmax_w;  // max ||x||_w^2 (weighted), nullable
    int64_t chunk_rows;
    float* thr;           // nq: bound + margin (filter threshold on e)
    float* qn;            // nq: ||q||_w^2
    float* mg;            // nq: margin
    unsigned* cnt;        // nq: candidates seen
    u64* cand;            // nq x kMCap
    const int32_t* perm;  // internal row -> caller row, nullable
    int64_t* idx;
    float* dist;
    int* err;
};

__device__ __forceinline__ u64 orderable_key(float e, uint32_t row) {
    uint32_t u = __float_as_uint(e);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ((u64)u << 32) | row;
}
__device__ __forceinline__ float orderable_value(u64 key) {
    const uint32_t u = (uint32_t)(key >> 32);
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// Per frame (one warp): ||q||_w^2, the margin, and bound + margin. The bound
// is the k-th smallest finite bucket minimum (ties by bucket), widened 2^-12;
// +inf when fewer than k buckets are filled.
__global__ void many_bound_kernel(ManyParams p) {
    const int lane = threadIdx.x & 31;
    const int f = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (f >= p.nq) return;
    float a = 0.f;
    for (int d = lane; d < p.D; d += 32) {
        const float q = p.Q[(size_t)f * p.D + d];
        const float wq = p.w ? p.w[d] * q : q;
        a = fmaf(wq, q, a);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(kFull, a, o);
    const unsigned* bm = p.bmin + (size_t)f * kMBuckets;
    unsigned v[4], rank[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = __ldcg(bm + lane + 32 * i);
    for (int src = 0; src < 32; ++src) {
#pragma unroll
        for (int i2 = 0; i2 < 4; ++i2) {
            const unsigned u = __shfl_sync(kFull, v[i2], src);
            const int ub = src + 32 * i2;
#pragma unroll
            for (int i = 0; i < 4; ++i) rank[i] += (u < v[i] || (u == v[i] && ub < lane + 32 * i)) ? 1u : 0u;
        }
    }
    unsigned b = 0xffffffffu;
#pragma unroll
    for (int i = 0; i < 4; ++i)
        if (v[i] < 0x7f800000u && rank[i] == (unsigned)p.k - 1u) b = v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) b = min(b, __shfl_xor_sync(kFull, b, o));
    if (lane == 0) {
        const float inf = __int_as_float(0x7f800000);
        const float bound = b < 0x7f800000u ? __uint_as_float(b) * (1.0f + 1.0f / 4096.0f) : inf;
        const float rad = (p.xmax_w != nullptr ? sqrtf(__ldg(p.xmax_w)) * 1.0001f : p.xmax) + sqrtf(a);
        const float margin = p.margin_scale * rad * rad;
        p.qn[f] = a;
        p.mg[f] = margin;
        p.thr[f] = bound + margin;
    }
}

// Stage one K-chunk (kMRows rows x KC dims) of rows [r0, r0 + kMRows) into xs
// (row pitch KC + 4 floats) with 16-byte cp.async copies (rows past r1 are
// zero-filled).
template <int KC>
__device__ __forceinline__ void load_chunk(const ManyParams& p, float* xs, int64_t r0, int64_t r1, int d0) {
    constexpr int kMK = KC, kXPitch = KC + 4;
    constexpr int kVec = kMRows * kMK / 4;  // float4 per chunk
    for (int i = threadIdx.x; i < kVec; i += kMThreads) {
        const int r = i / (kMK / 4), c = i % (kMK / 4);
        float* dst = xs + r * kXPitch + 4 * c;
        const int64_t row = r0 + r;
        if (row < r1) {
            __pipeline_memcpy_async(dst, p.X + (size_t)row * p.D + d0 + 4 * c, 16);
        } else {
            *reinterpret_cast<float4*>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    __pipeline_commit();
}

// Flush the staged candidates of the CTA's frames to their buffers (one
// atomic per frame).
__device__ __forceinline__ void flush_stage(const ManyParams& p, int f0, unsigned* scnt, u64* stage) {
    __syncthreads();
    for (int f = threadIdx.x; f < kMF; f += kMThreads) {
        const unsigned n = min(scnt[f], (unsigned)kMStage);
        if (n > 0 && f0 + f < p.nq) {
            const unsigned pos = atomicAdd(p.cnt + f0 + f, n);
            for (unsigned i = 0; i < n; ++i)
                if (pos + i < (unsigned)kMCap) p.cand[(size_t)(f0 + f) * kMCap + pos + i] = stage[f * kMStage + i];
        }
        scnt[f] = 0u;
    }
    __syncthreads();
}

// KC: dimensions per K-chunk (128 when D allows: half the chunk steps and
// their barriers of 64).
template <bool kWeighted, int KC>
__global__ void __launch_bounds__(kMThreads, 1) many_kernel(ManyParams p) {
    constexpr int kMK = KC, kXPitch = KC + 4;
    extern __shared__ __align__(16) float msm[];
    const int D = p.D;
    const int wpitch = D + 4;
    float* wq = msm;                                   // kMF x (D + 4): w * q
    float* xs0 = wq + kMF * wpitch;                    // kMRows x kXPitch
    float* xs1 = xs0 + kMRows * kXPitch;
    u64* stage = reinterpret_cast<u64*>(xs1 + kMRows * kXPitch);  // kMF x kMStage
    unsigned* scnt = reinterpret_cast<unsigned*>(stage + kMF * kMStage);  // kMF
    float* sthr = reinterpret_cast<float*>(scnt + kMF);                    // kMF
    float* sqn = sthr + kMF;                                                // kMF

    const int t = threadIdx.x;
    const int tf = t & 7, tr = t >> 3;  // frames tf + 8 i, rows 4 tr + j
    const int f0 = blockIdx.x * kMF;
    const int64_t row0 = (int64_t)blockIdx.y * p.chunk_rows;
    const int64_t row1 = min(p.n, row0 + p.chunk_rows);

    for (int i = t; i < kMF * D; i += kMThreads) {
        const int f = i / D, d = i % D;
        const float q = f0 + f < p.nq ? p.Q[(size_t)(f0 + f) * D + d] : 0.f;
        wq[f * wpitch + d] = kWeighted ? __ldg(p.w + d) * q : q;
    }
    for (int f = t; f < kMF; f += kMThreads) {
        scnt[f] = 0u;
        sthr[f] = f0 + f < p.nq ? p.thr[f0 + f] : -__int_as_float(0x7f800000);
        sqn[f] = f0 + f < p.nq ? p.qn[f0 + f] : 0.f;
    }
    __syncthreads();
    float thr[8], qn[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        thr[i] = sthr[tf + 8 * i];
        qn[i] = sqn[tf + 8 * i];
    }
    const int nk = D / kMK;
    const int64_t ntiles = row1 > row0 ? (row1 - row0 + kMRows - 1) / kMRows : 0;
    const int64_t nsteps = ntiles * nk;
    if (nsteps > 0) load_chunk<KC>(p, xs0, row0, row1, 0);
    float2 acc[8][4];
    for (int64_t s = 0; s < nsteps; ++s) {
        const int64_t tile = s / nk;
        const int kc = (int)(s % nk);
        const int64_t r0 = row0 + tile * kMRows;
        float* xs = (s & 1) ? xs1 : xs0;
        if (s + 1 < nsteps) {
            const int64_t tn = (s + 1) / nk;
            load_chunk<KC>(p, (s & 1) ? xs0 : xs1, row0 + tn * kMRows, row1, (int)((s + 1) % nk) * kMK);
            __pipeline_wait_prior(1);
        } else {
            __pipeline_wait_prior(0);
        }
        __syncthreads();
        if (kc == 0) {
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
        }
        const float* wqk = wq + kc * kMK;
#pragma unroll 4
        for (int d4 = 0; d4 < kMK / 4; ++d4) {
            float4 a[8], b[4];
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = *reinterpret_cast<const float4*>(wqk + (tf + 8 * i) * wpitch + 4 * d4);
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = *reinterpret_cast<const float4*>(xs + (4 * tr + j) * kXPitch + 4 * d4);
            // the (x, y) halves into every accumulator, then the (z, w) halves:
            // consecutive packed FMAs never depend on each other
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    acc[i][j] = __ffma2_rn(make_float2(a[i].x, a[i].y), make_float2(b[j].x, b[j].y), acc[i][j]);
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    acc[i][j] = __ffma2_rn(make_float2(a[i].z, a[i].w), make_float2(b[j].z, b[j].w), acc[i][j]);
        }
        if (kc == nk - 1) {
            // the tile's expanded-form values against the frames' thresholds
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int64_t row = r0 + 4 * tr + j;
                const bool rv = row < row1;
                const float xnr = rv ? __ldg(p.xn + row) : 0.f;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float e = fmaf(-2.f, acc[i][j].x + acc[i][j].y, xnr + qn[i]);
                    if (rv && e <= thr[i]) {
                        const int f = tf + 8 * i;
                        const u64 key = orderable_key(e, (uint32_t)row);
                        const unsigned slot = atomicAdd(&scnt[f], 1u);
                        if (slot < (unsigned)kMStage) {
                            stage[f * kMStage + slot] = key;
                        } else {
                            // stage full: straight to the frame's buffer
                            const unsigned pos = atomicAdd(p.cnt + f0 + f, 1u);
                            if (pos < (unsigned)kMCap) p.cand[(size_t)(f0 + f) * kMCap + pos] = key;
                        }
                    }
                }
            }
            // flush when some frame's stage is at least half full (and at the end)
            bool half = false;
            for (int f = t; f < kMF; f += kMThreads) half |= scnt[f] >= (unsigned)(kMStage / 2);
            if (__syncthreads_or(half)) flush_stage(p, f0, scnt, stage);
        }
        __syncthreads();  // the buffer just read is the next step's load target
    }
    flush_stage(p, f0, scnt, stage);
}

// Exact distance sum w (q - x)^2 of row r to frame f, by one warp (lanes split
// the dimensions; fixed butterfly order).
__device__ __forceinline__ float warp_exact(const ManyParams& p, int f, uint32_t r, int lane) {
    float a = 0.f;
    const float* x = p.X + (size_t)r * p.D;
    const float* q = p.Q + (size_t)f * p.D;
    for (int d = lane; d < p.D; d += 32) {
        const float diff = q[d] - x[d];
        a = p.w ? fmaf(p.w[d] * diff, diff, a) : fmaf(diff, diff, a);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(kFull, a, o);
    return a;
}

// Exact distance of row r (this lane's own row) to frame f, the lane alone
// (the exhaustive fallback).
__device__ __forceinline__ float lane_exact(const ManyParams& p, int f, int64_t r) {
    float a = 0.f;
    const float4* x = reinterpret_cast<const float4*>(p.X + (size_t)r * p.D);
    const float4* q = reinterpret_cast<const float4*>(p.Q + (size_t)f * p.D);
    for (int c = 0; c < p.D / 4; ++c) {
        const float4 xv = __ldg(x + c), qv = __ldg(q + c);
        const float4 wv = p.w ? __ldg(reinterpret_cast<const float4*>(p.w) + c) : make_float4(1.f, 1.f, 1.f, 1.f);
        const float d0 = qv.x - xv.x, d1 = qv.y - xv.y, d2 = qv.z - xv.z, d3 = qv.w - xv.w;
        a = fmaf(wv.x * d0, d0, a);
        a = fmaf(wv.y * d1, d1, a);
        a = fmaf(wv.z * d2, d2, a);
        a = fmaf(wv.w * d3, d3, a);
    }
    return a;
}

// Per frame (one warp): e_k = the k-th smallest candidate e (a running 64
// smallest keys in registers), then the exact top k of the candidates with
// e <= e_k + 2 margin; an overflowed buffer falls back to an exhaustive exact
// pass over the frame (one row per lane).
__global__ void many_select_kernel(ManyParams p) {
    const int lane = threadIdx.x & 31;
    const int f = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (f >= p.nq) return;
    const unsigned c = __ldcg(p.cnt + f);
    u64 L = kKeyEmpty;  // exact (distance, row) top k, lane i = i-th
    if (c > (unsigned)kMCap) {
        for (int64_t base = 0; base < p.n; base += 32) {
            const int64_t r = base + lane;
            const u64 key = r < p.n ? make_key(lane_exact(p, f, r), (uint32_t)r) : kKeyEmpty;
            unsigned m = __ballot_sync(kFull, key < __shfl_sync(kFull, L, p.k - 1));
            while (m) {
                const int j = __ffs(m) - 1;
                m &= m - 1;
                list_insert(L, __shfl_sync(kFull, key, j), p.k, lane);
            }
        }
    } else {
        const u64* cf = p.cand + (size_t)f * kMCap;
        u64 best[2] = {kKeyEmpty, kKeyEmpty};
        for (unsigned base = 0; base < c; base += 64) {
            u64 cur[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const unsigned i = base + e * 32 + lane;
                cur[e] = i < c ? __ldcg(cf + i) : kKeyEmpty;
            }
            warp_sort64(cur, lane);
            warp_merge64(best, cur, lane);
        }
        // element k - 1 of the sorted 64 (layout e * 32 + lane)
        const u64 ek = __shfl_sync(kFull, best[(p.k - 1) / 32], (p.k - 1) % 32);
        const float lim = (c >= (unsigned)p.k && ek != kKeyEmpty) ? orderable_value(ek) + 2.f * p.mg[f]
                                                                  : __int_as_float(0x7f800000);
        for (unsigned base = 0; base < c; base += 32) {
            const unsigned i = base + lane;
            const u64 v = i < c ? __ldcg(cf + i) : kKeyEmpty;
            unsigned m = __ballot_sync(kFull, i < c && orderable_value(v) <= lim);
            while (m) {
                const int j = __ffs(m) - 1;
                m &= m - 1;
                const uint32_t r = (uint32_t)__shfl_sync(kFull, v, j);
                const float d = warp_exact(p, f, r, lane);
                const u64 key = make_key(d, r);
                if (key < __shfl_sync(kFull, L, p.k - 1)) list_insert(L, key, p.k, lane);
            }
        }
    }
    if (lane < p.k) {
        const size_t o = (size_t)f * p.k + lane;
        if (L == kKeyEmpty) {
            p.idx[o] = -1;
            p.dist[o] = __int_as_float(0x7f800000);
        } else {
            const uint32_t r = key_row(L);
            p.idx[o] = p.perm ? (int64_t)p.perm[r] : (int64_t)r;
            p.dist[o] = key_dist(L);
        }
    }
}

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t many_smem(int D, int kc) {
    return (size_t)kMF * (D + 4) * sizeof(float) + 2 * (size_t)kMRows * (kc + 4) * sizeof(float) +
           (size_t)kMF * kMStage * sizeof(u64) + 3 * (size_t)kMF * sizeof(float);
}

}  // namespace

// Many frames over a database of up to 1M rows: there the streaming scan's
// CTAs get short row chunks (n / SMs rows per 8 frames) and their fixed costs
// dominate (measured: 200,000 x 1,280 frames, 7.97 ms streaming vs 6.40 ms
// here); over 2,000,000 rows x 1,024 frames the streaming scan is faster
// (39 ms vs 52 ms).
bool many_eligible(const lhr_db* db, int nq, int k) {
    return db->n_sub == 1 && db->Xp != nullptr && nq >= kMF && k >= 1 && k <= 32 && db->dim % 64 == 0 &&
           db->dim <= 256 && db->n < 1000000;
}

size_t many_scratch_bytes(int nq) {
    return 3 * a256((size_t)nq * sizeof(float)) + a256((size_t)nq * sizeof(unsigned)) +
           a256((size_t)nq * kMCap * sizeof(u64));
}

cudaError_t launch_many(const lhr_db* db, const float* q, int nq, int k, const float* w, const float* xn,
                        const float* xmax_w, const unsigned* bmin, float margin_scale, int64_t* idx, float* dist,
                        void* scratch, cudaStream_t stream) {
    ManyParams p{};
    p.X = db->X;
    p.xn = xn;
    p.n = db->n;
    p.D = db->dim;
    p.Q = q;
    p.w = w;
    p.nq = nq;
    p.k = k;
    p.bmin = bmin;
    p.margin_scale = margin_scale;
    p.xmax = (float)(sqrt((double)db->xnorm_max) * 1.0001);
    p.xmax_w = xmax_w;
    unsigned char* base = reinterpret_cast<unsigned char*>(scratch);
    p.thr = reinterpret_cast<float*>(base);
    p.qn = reinterpret_cast<float*>(base + a256((size_t)nq * sizeof(float)));
    p.mg = reinterpret_cast<float*>(base + 2 * a256((size_t)nq * sizeof(float)));
    p.cnt = reinterpret_cast<unsigned*>(base + 3 * a256((size_t)nq * sizeof(float)));
    p.cand = reinterpret_cast<u64*>(base + 3 * a256((size_t)nq * sizeof(float)) + a256((size_t)nq * sizeof(unsigned)));
    p.perm = db->perm;
    p.idx = idx;
    p.dist = dist;
    p.err = db->err;
    const int nfb = (nq + kMF - 1) / kMF;
    // about one CTA per SM over frame blocks x row chunks; chunks are whole tiles
    const int chunks = std::max(1, (db->sms + nfb - 1) / nfb);
    int64_t cr = (db->n + chunks - 1) / chunks;
    cr = (cr + kMRows - 1) / kMRows * kMRows;
    p.chunk_rows = cr;
    const int nchunks = (int)((db->n + cr - 1) / cr);
    if (nchunks > 65535) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(p.cnt, 0, (size_t)nq * sizeof(unsigned), stream);
    if (e != cudaSuccess) return e;
    {
        ProfScope ps("many_bound_kernel", stream);
        many_bound_kernel<<<(nq + 7) / 8, 256, 0, stream>>>(p);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const int kc = db->dim % 128 == 0 ? 128 : 64;
    const size_t sm = many_smem(db->dim, kc);
    {
        auto kern = kc == 128 ? (w ? many_kernel<true, 128> : many_kernel<false, 128>)
                              : (w ? many_kernel<true, 64> : many_kernel<false, 64>);
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) != cudaSuccess)
            return e;
        ProfScope ps("many_kernel", stream);
        kern<<<dim3(nfb, nchunks), kMThreads, sm, stream>>>(p);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    {
        ProfScope ps("many_select_kernel", stream);
        many_select_kernel<<<(nq + 7) / 8, 256, 0, stream>>>(p);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace lhr
