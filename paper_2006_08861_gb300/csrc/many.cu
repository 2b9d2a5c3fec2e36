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
//
// Where D is a multiple of 32 the filter runs on the tensor cores instead
// (tf32_many_kernel: tcgen05.mma kind::tf32, 128 rows x 128 frames per MMA,
// operands staged by TMA, accumulators in TMEM) with the margin widened for
// TF32 operands; the candidates and their exact re-score are the same.
#include <cuda_pipeline.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "tc.cuh"

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
    // Tensor-core form: the bucket minima are TF32 scores (each within the margin
    // of its row's exact distance), so the bound adds one margin; fT (nullable)
    // receives thr - qn + slack, the threshold on ||x||_w^2 - 2 (w q) . x.
    bool bmin_scored;
    float* fT;
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
        const float xnmax = p.xmax_w != nullptr ? __ldg(p.xmax_w) : p.xmax * p.xmax;
        const float rad = (p.xmax_w != nullptr ? sqrtf(xnmax) * 1.0001f : p.xmax) + sqrtf(a);
        const float margin = p.margin_scale * rad * rad;
        float bound = b < 0x7f800000u ? __uint_as_float(b) * (1.0f + 1.0f / 4096.0f) : inf;
        if (p.bmin_scored) bound += margin;
        const float thr = bound + margin;
        p.qn[f] = a;
        p.mg[f] = margin;
        p.thr[f] = thr;
        if (p.fT != nullptr) {
            // the pass tests u = fl(||x||_w^2 - 2 (w q) . x) <= fT and keys e = fl(u + qn): a pair
            // with e <= thr has u <= thr - qn up to three roundings of magnitude at most
            // |thr| + |qn| + max ||x||_w^2 each; the slack is four units in the last place of that
            const float slack = 4.0f * 5.9604645e-08f * (fabsf(thr) + a + xnmax);
            p.fT[f] = (thr - a) + slack;
        }
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

// ------------------------------------------------------------------ TF32 tensor-core pass
// The filter of many_kernel on the tensor cores: u(f, r) = ||x_r||_w^2 - 2 (w q_f) . x_r
// with the dot by tcgen05.mma kind::tf32 (operands truncated to TF32, FP32
// accumulation) over 128-row x 128-frame tiles, one CTA per (128-frame block,
// row chunk): database rows stream through a TMA ring, the block's w q rows stay
// in shared memory, accumulators rotate through TMEM. The epilogue thread of a
// row tests its 64 frames exactly, u <= fT_f (fT_f = thr_f - ||q_f||_w^2 +
// slack, held in registers), with a three-input minimum over the 64 differences
// deciding whether any passes; the passing pairs are keyed (orderable e = u +
// ||q_f||_w^2, row) into a per-frame stage in shared memory and appended to the
// frames' buffers at the end, one atomic per frame.
//
// kPilot: the same pipeline over every kTfPilotStride-th row (a strided tensor
// map, no copy) writes bucket minima instead: per warp (32 sample rows) and
// frame the smallest e (column_min32), clamped at 0, into bucket
// (sample row / 32) mod 128 by atomic minimum. Minima of distinct buckets are
// distinct rows, each within the margin of its exact distance, so the k-th
// smallest plus one margin bounds the frame's k-th exact distance.
using namespace tc;
constexpr int kFT = 128;                 // frames per CTA (UMMA N)
constexpr int kFAcc = 4;                 // 128-column FP32 accumulators (all of TMEM)
constexpr int kFEpiWarps = 8;            // two per TMEM lane quadrant, 64 columns each
constexpr int kFEpiThreads = 32 * kFEpiWarps;
constexpr int kFThreads = 64 + kFEpiThreads;
constexpr int kFMaxStages = 8;
constexpr int kFStage = 32;              // staged candidates per frame of the CTA
constexpr int kFSlice = kFT * kTcSliceBytes;  // 16 KB: one 128-byte K slice of 128 rows
constexpr int kTfPilotStride = 8;        // pilot sample: every 8th row

struct TfParams {
    int64_t n;            // rows of this pass (sample rows for the pilot)
    int slices, stages;
    int64_t chunk_rows;
    int64_t xn_stride;    // pass row r has norm xn[r * xn_stride]
    const float* xn;      // ||x||_w^2 per database row
    const float* fT;      // per frame: threshold on u (main pass)
    const float* qn;      // per frame: ||q||_w^2
    unsigned* cnt;        // per frame: candidates seen
    u64* cand;            // per frame: kMCap candidate keys (orderable e, row)
    unsigned* bmin;       // pilot: per frame kMBuckets bucket minima (float bits)
    int nq;
    int* err;
};

// Appends key to frame column col's stage (the frame's buffer when the stage is full).
__device__ __forceinline__ void tf_emit(const TfParams& p, unsigned* scnt, u64* stage, int col, int f, u64 key) {
    const unsigned slot = atomicAdd(&scnt[col], 1u);
    if (slot < (unsigned)kFStage) {
        stage[col * kFStage + slot] = key;
    } else {
        const unsigned pos = atomicAdd(p.cnt + f, 1u);
        if (pos < (unsigned)kMCap) p.cand[(size_t)f * kMCap + pos] = key;
    }
}

// Exact test of one row against a group of 32 frames (columns col0 + j), the
// passing pairs keyed. Called only when some difference u - fT is <= 0.
__device__ __forceinline__ void tf_pass32(const TfParams& p, const uint32_t (&v)[32], const float (&T)[32], float xn,
                                          uint32_t row, int col0, int fbase, const float* sqn, unsigned* scnt,
                                          u64* stage) {
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        const float u = fmaf(-2.f, __uint_as_float(v[j]), xn);
        if (u <= T[j]) tf_emit(p, scnt, stage, col0 + j, fbase + col0 + j, orderable_key(u + sqn[col0 + j], row));
    }
}

// min over j of (fl(xn - 2 v_j) - T_j): <= 0 exactly when some u_j <= T_j.
__device__ __forceinline__ float tf_min_diff(const uint32_t (&v)[32], const float (&T)[32], float xn) {
    float m = fmaf(-2.f, __uint_as_float(v[0]), xn) - T[0];
#pragma unroll
    for (int j = 1; j < 31; j += 2)
        m = fmin3(m, fmaf(-2.f, __uint_as_float(v[j]), xn) - T[j], fmaf(-2.f, __uint_as_float(v[j + 1]), xn) - T[j + 1]);
    return fminf(m, fmaf(-2.f, __uint_as_float(v[31]), xn) - T[31]);
}

// Pilot: column minima of e over the warp's 32 rows into the frames' bucket.
__device__ __forceinline__ void tf_pilot32(const TfParams& p, const uint32_t (&v)[32], float xn, bool rowvalid,
                                           int col, int f, const float* sqn, int bucket, int lane) {
    float c[32];
    const float inf = __int_as_float(0x7f800000);
#pragma unroll
    for (int j = 0; j < 32; ++j) c[j] = rowvalid ? fmaf(-2.f, __uint_as_float(v[j]), xn) : inf;
    const float mn = column_min32(c, lane);
    if (f < p.nq && mn < inf) {
        const float e = fmaxf(mn + sqn[col], 0.f);
        atomicMin(p.bmin + (size_t)f * kMBuckets + bucket, __float_as_uint(e));
    }
}

template <bool kPilot>
__global__ void __launch_bounds__(kFThreads, 1)
    tf32_many_kernel(const __grid_constant__ CUtensorMap tmQ, const __grid_constant__ CUtensorMap tmX, const TfParams p) {
    extern __shared__ unsigned char smem_raw[];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int chunk = blockIdx.x, fblock = blockIdx.y;
    unsigned char* smem =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int stages = p.stages;
    unsigned char* sQ = smem;                                    // slices x 16 KB: the block's frames (w q)
    unsigned char* sX = sQ + (size_t)p.slices * kFSlice;         // stages x 16 KB: database slices
    float* sqn = reinterpret_cast<float*>(sX + (size_t)stages * kFSlice);  // kFT: ||q||_w^2 per column
    unsigned* scnt = reinterpret_cast<unsigned*>(sqn + kFT);               // kFT: staged keys per column
    u64* full = reinterpret_cast<u64*>(scnt + kFT);
    u64* empty = full + kFMaxStages;
    u64* q_full = empty + kFMaxStages;
    u64* acc_full = q_full + 1;
    u64* acc_empty = acc_full + kFAcc;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(acc_empty + kFAcc);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
    u64* stage = reinterpret_cast<u64*>(tmem_holder + 4);       // main pass: kFT x kFStage keys

    const int64_t row0 = (int64_t)chunk * p.chunk_rows;
    const int64_t row1 = min(p.n, row0 + p.chunk_rows);
    const int ntiles = row1 > row0 ? (int)((row1 - row0 + kTcM - 1) / kTcM) : 0;
    const int fbase = fblock * kFT;
    constexpr int kElemPerSlice = kTcSliceBytes / 4;  // 32 floats
    constexpr int kMmaK = 8;                          // TF32 elements per MMA (32 bytes)
    constexpr int kMmaPerSlice = kElemPerSlice / kMmaK;
    constexpr uint32_t kIdesc = tc_idesc(kTcTF32, kFT);

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(q_full, 1);
        for (int i = 0; i < kFAcc; ++i) {
            mbar_init(&acc_full[i], 1);
            mbar_init(&acc_empty[i], kFEpiWarps);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    for (int c = threadIdx.x; c < kFT; c += kFThreads) {
        sqn[c] = fbase + c < p.nq ? __ldg(p.qn + fbase + c) : 0.f;
        scnt[c] = 0u;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(kFAcc * kFT)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    if (warp == 0) {
        if (lane == 0) {
            mbar_arrive_expect_tx(q_full, (uint32_t)p.slices * kFSlice);
            for (int s = 0; s < p.slices; ++s)
                tma_load_2d(sQ + (size_t)s * kFSlice, &tmQ, s * kElemPerSlice, fbase, q_full);
            int b_issued = 0, st = 0;
            uint32_t ph = 0;
            for (int t = 0; t < ntiles && !*abort_flag; ++t) {
                const int r = (int)(row0 + (int64_t)t * kTcM);
                for (int s = 0; s < p.slices; ++s) {
                    if (!mbar_wait(&empty[st], ph ^ 1u, abort_flag)) {
                        *abort_flag = 1;
                        record_error(p.err, kErrTimeout);
                        break;
                    }
                    mbar_arrive_expect_tx(&full[st], kFSlice);
                    tma_load_2d(sX + (size_t)st * kFSlice, &tmX, s * kElemPerSlice, r, &full[st]);
                    ++b_issued;
                    if (++st == stages) {
                        st = 0;
                        ph ^= 1u;
                    }
                }
            }
            if (*abort_flag) {
                // let this thread's copies still in flight land before the CTA exits (bounded waits)
                mbar_wait(q_full, 0u, nullptr);
                for (int it = b_issued > stages ? b_issued - stages : 0; it < b_issued; ++it)
                    mbar_wait(&full[it % stages], (uint32_t)((it / stages) & 1), nullptr);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            bool ok = mbar_wait(q_full, 0u, abort_flag);
            int st = 0;
            uint32_t ph = 0;
            for (int t = 0; ok && t < ntiles; ++t) {
                const int a = t % kFAcc;
                if (!mbar_wait(&acc_empty[a], (uint32_t)((t / kFAcc) & 1) ^ 1u, abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(a * kFT);
                for (int s = 0; s < p.slices; ++s) {
                    if (!mbar_wait(&full[st], ph, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t x_base = smem_u32(sX + (size_t)st * kFSlice);
                    const uint32_t q_base = smem_u32(sQ + (size_t)s * kFSlice);
#pragma unroll
                    for (int kk = 0; kk < kMmaPerSlice; ++kk) {
                        const uint32_t off = (uint32_t)(kk * kMmaK * 4);
                        tc::tc_mma<kTcTF32>(d_tmem, sw128_desc(x_base + off), sw128_desc(q_base + off), kIdesc,
                                            (s | kk) != 0 ? 1u : 0u);
                    }
                    tc_commit(&empty[st]);
                    if (++st == stages) {
                        st = 0;
                        ph ^= 1u;
                    }
                }
                if (!ok) break;
                tc_commit(&acc_full[a]);
            }
            if (!ok) {
                *abort_flag = 1;
                record_error(p.err, kErrTimeout);
            }
        }
    } else {
        // ------------------------------------------------ epilogue: thread = database row
        const int ew = warp - 2;
        const int quad = warp & 3;                            // TMEM lanes 32 quad .. 32 quad + 31
        const int rl = quad * 32 + lane;
        const int cb = (ew / 4) * 64;                         // first column (frame) of this warp's half
        const float ninf = -__int_as_float(0x7f800000);
        float T0[32], T1[32];                                 // per column: the frame's threshold on u
        if (!kPilot) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int f0 = fbase + cb + j, f1 = f0 + 32;
                T0[j] = f0 < p.nq ? __ldg(p.fT + f0) : ninf;
                T1[j] = f1 < p.nq ? __ldg(p.fT + f1) : ninf;
            }
        }
        for (int t = 0; t < ntiles; ++t) {
            const int a = t % kFAcc;
            const int64_t row = row0 + (int64_t)t * kTcM + rl;
            const bool rowvalid = row < row1;
            const float xn = rowvalid ? __ldg(p.xn + row * p.xn_stride) : 0.f;
            if (!mbar_wait(&acc_full[a], (uint32_t)((t / kFAcc) & 1), abort_flag)) {
                if (lane == 0) {
                    *abort_flag = 1;
                    record_error(p.err, kErrTimeout);
                }
                break;
            }
            tc_fence_after();
            const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(a * kFT + cb);
            uint32_t va[32], vb[32];
            tmem_ld32_issue(tbase, va);
            tmem_ld32_issue(tbase + 32u, vb);
            tmem_ld_wait(va);  // waits for both loads; the second wait only names vb's registers
            tmem_ld_wait(vb);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[a]);
            if (kPilot) {
                const int bucket = (int)(((row0 + (int64_t)t * kTcM + quad * 32) >> 5) & (kMBuckets - 1));
                tf_pilot32(p, va, xn, rowvalid, cb + lane, fbase + cb + lane, sqn, bucket, lane);
                tf_pilot32(p, vb, xn, rowvalid, cb + 32 + lane, fbase + cb + 32 + lane, sqn, bucket, lane);
            } else if (rowvalid) {
                if (tf_min_diff(va, T0, xn) <= 0.f) tf_pass32(p, va, T0, xn, (uint32_t)row, cb, fbase, sqn, scnt, stage);
                if (tf_min_diff(vb, T1, xn) <= 0.f)
                    tf_pass32(p, vb, T1, xn, (uint32_t)row, cb + 32, fbase, sqn, scnt, stage);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kFAcc * kFT) : "memory");
    if (!kPilot) {
        // the stages to the frames' buffers: one atomic per frame
        for (int c = threadIdx.x; c < kFT; c += kFThreads) {
            const int f = fbase + c;
            const unsigned n = min(scnt[c], (unsigned)kFStage);
            if (f < p.nq && n > 0) {
                const unsigned pos = atomicAdd(p.cnt + f, n);
                for (unsigned i = 0; i < n; ++i)
                    if (pos + i < (unsigned)kMCap) p.cand[(size_t)f * kMCap + pos + i] = stage[c * kFStage + i];
            }
        }
    }
}

// Per frame (one warp): the B operand row w q and ||q||_w^2 (summed as many_bound_kernel does).
__global__ void tf32_prep_kernel(const float* Q, const float* w, int nq, int D, float* wq, float* qn) {
    const int lane = threadIdx.x & 31;
    const int f = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (f >= nq) return;
    float a = 0.f;
    for (int d = lane; d < D; d += 32) {
        const float q = Q[(size_t)f * D + d];
        const float v = w ? w[d] * q : q;
        wq[(size_t)f * D + d] = v;
        a = fmaf(v, q, a);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(kFull, a, o);
    if (lane == 0) qn[f] = a;
}

size_t tf32_smem(int slices, int stages, bool pilot) {
    return 1024 + (size_t)(slices + stages) * kFSlice + 2 * kFT * sizeof(float) +
           (2 * kFMaxStages + 1 + 2 * kFAcc) * sizeof(u64) + 16 + (pilot ? 0 : (size_t)kFT * kFStage * sizeof(u64));
}

int tf32_stages(int slices, bool pilot) {
    const size_t fixed = tf32_smem(slices, 0, pilot);
    const size_t lim = 227 * 1024;
    const int fit = fixed < lim ? (int)((lim - fixed) / kFSlice) : 0;
    return std::min(kFMaxStages, fit);
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

// The TF32 pass serves whole 32-float K slices of at most 256 dimensions and row
// indices that fit the candidate keys.
// The tensor-core form serves whole 32-float K slices of at most 256
// dimensions and row indices that fit the candidate keys.
bool many_tf32(const lhr_db* db) { return db->dim % 32 == 0 && db->dim <= 256 && db->n < (int64_t)1 << 31; }

namespace {

struct TfLayout {
    size_t thr, qn, mg, cnt, cand, fT, wq, bmin, total;
};

TfLayout many_layout(const lhr_db* db, int nq) {
    TfLayout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t r = off;
        off += a256(bytes);
        return r;
    };
    L.thr = take((size_t)nq * sizeof(float));
    L.qn = take((size_t)nq * sizeof(float));
    L.mg = take((size_t)nq * sizeof(float));
    L.cnt = take((size_t)nq * sizeof(unsigned));
    L.cand = take((size_t)nq * kMCap * sizeof(u64));
    if (many_tf32(db)) {
        L.fT = take((size_t)nq * sizeof(float));
        L.wq = take((size_t)nq * db->dim * sizeof(float));
        L.bmin = take((size_t)nq * kMBuckets * sizeof(unsigned));
    }
    L.total = off;
    return L;
}

// Row chunks per frame block so that the CTAs fill whole waves of the SMs as
// far as possible (waves x tiles per CTA, plus a per-CTA fixed cost of about
// two tiles: the frames' operand and the pipeline's fill).
int tf32_chunks(int nfb, int sms, int64_t n) {
    const int64_t tiles = (n + kTcM - 1) / kTcM;
    int best = 1;
    double best_cost = 1e300;
    for (int c = 1; c <= 4 * sms && c <= tiles; ++c) {
        const int64_t per = (tiles + c - 1) / c;
        const int64_t waves = ((int64_t)c * nfb + sms - 1) / sms;
        const double cost = (double)waves * (double)(per + 2);
        if (cost < best_cost) {
            best_cost = cost;
            best = c;
        }
    }
    return best;
}

// One TF32 pass (pilot over every kTfPilotStride-th row, or the main pass)
// over the frames' w q rows.
template <bool kPilot>
cudaError_t tf32_pass(const lhr_db* db, const float* wq, int nq, TfParams t, cudaStream_t stream) {
    const int D = db->dim;
    const int64_t stride = kPilot ? kTfPilotStride : 1;
    t.n = (db->n + stride - 1) / stride;
    t.xn_stride = stride;
    CUtensorMap tmQ, tmX;
    if (!make_map(&tmQ, wq, nq, D, kTcTF32, kFT) || !make_map(&tmX, db->X, t.n, D, kTcTF32, kTcM, stride * D))
        return cudaErrorInvalidValue;
    t.slices = D / 32;
    t.stages = tf32_stages(t.slices, kPilot);
    if (t.stages < 2) return cudaErrorInvalidValue;
    const int nfb = (nq + kFT - 1) / kFT;
    if (nfb > 65535) return cudaErrorInvalidValue;
    const int nchunks = tf32_chunks(nfb, db->sms, t.n);
    const int64_t cr = (t.n + nchunks - 1) / nchunks;
    t.chunk_rows = (cr + kTcM - 1) / kTcM * kTcM;
    const int grid_x = (int)((t.n + t.chunk_rows - 1) / t.chunk_rows);
    const size_t sm = tf32_smem(t.slices, t.stages, kPilot);
    cudaError_t e =
        cudaFuncSetAttribute(tf32_many_kernel<kPilot>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    ProfScope ps(kPilot ? "tf32_pilot_kernel" : "tf32_many_kernel", stream);
    tf32_many_kernel<kPilot><<<dim3(grid_x, nfb), kFThreads, sm, stream>>>(tmQ, tmX, t);
    return cudaGetLastError();
}

}  // namespace

size_t many_scratch_bytes(const lhr_db* db, int nq) { return many_layout(db, nq).total; }

// bmin: the pilot's bucket minima for the FP32 register-tiled form; the
// tensor-core form (many_tf32) runs its own pilot and takes nullptr.
cudaError_t launch_many(const lhr_db* db, const float* q, int nq, int k, const float* w, const float* xn,
                        const float* xmax_w, const unsigned* bmin, float margin_scale, int64_t* idx, float* dist,
                        void* scratch, cudaStream_t stream) {
    const bool tf32 = many_tf32(db);
    if (!tf32 && bmin == nullptr) return cudaErrorInvalidValue;
    const TfLayout L = many_layout(db, nq);
    unsigned char* base = reinterpret_cast<unsigned char*>(scratch);
    ManyParams p{};
    p.X = db->X;
    p.xn = xn;
    p.n = db->n;
    p.D = db->dim;
    p.Q = q;
    p.w = w;
    p.nq = nq;
    p.k = k;
    p.bmin = tf32 ? reinterpret_cast<unsigned*>(base + L.bmin) : bmin;
    // TF32 operands (10 stored mantissa bits, truncated or rounded): each product
    // w q_d x_d is off by less than (2^-9 + 2^-20) of its magnitude, so 2 |dot
    // error| <= (2^-9 + 2^-20) 2 ||q||_w ||x||_w <= (2^-10 + 2^-21) rad^2; the FP32
    // accumulation term is doubled for the tensor core's own summation order.
    p.margin_scale = tf32 ? 2.f * margin_scale + 1.0f / 1024.f * 1.001f : margin_scale;
    p.xmax = (float)(sqrt((double)db->xnorm_max) * 1.0001);
    p.xmax_w = xmax_w;
    p.thr = reinterpret_cast<float*>(base + L.thr);
    p.qn = reinterpret_cast<float*>(base + L.qn);
    p.mg = reinterpret_cast<float*>(base + L.mg);
    p.cnt = reinterpret_cast<unsigned*>(base + L.cnt);
    p.cand = reinterpret_cast<u64*>(base + L.cand);
    p.bmin_scored = tf32;
    p.fT = tf32 ? reinterpret_cast<float*>(base + L.fT) : nullptr;
    p.perm = db->perm;
    p.idx = idx;
    p.dist = dist;
    p.err = db->err;
    cudaError_t e = cudaMemsetAsync(p.cnt, 0, (size_t)nq * sizeof(unsigned), stream);
    if (e != cudaSuccess) return e;
    TfParams t{};
    float* wq = tf32 ? reinterpret_cast<float*>(base + L.wq) : nullptr;
    if (tf32) {
        // the frames' w q rows and norms, then the pilot's bucket minima
        unsigned* bm = reinterpret_cast<unsigned*>(base + L.bmin);
        if ((e = cudaMemsetAsync(bm, 0xff, (size_t)nq * kMBuckets * sizeof(unsigned), stream)) != cudaSuccess)
            return e;
        {
            ProfScope ps("tf32_prep_kernel", stream);
            tf32_prep_kernel<<<(nq + 7) / 8, 256, 0, stream>>>(q, w, nq, db->dim, wq, p.qn);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        t.xn = xn;
        t.fT = p.fT;
        t.qn = p.qn;
        t.cnt = p.cnt;
        t.cand = p.cand;
        t.bmin = bm;
        t.nq = nq;
        t.err = db->err;
        if ((e = tf32_pass<true>(db, wq, nq, t, stream)) != cudaSuccess) return e;
    }
    {
        ProfScope ps("many_bound_kernel", stream);
        many_bound_kernel<<<(nq + 7) / 8, 256, 0, stream>>>(p);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (tf32) {
        if ((e = tf32_pass<false>(db, wq, nq, t, stream)) != cudaSuccess) return e;
    } else {
        const int nfb = (nq + kMF - 1) / kMF;
        // about one CTA per SM over frame blocks x row chunks; chunks are whole tiles
        const int chunks = std::max(1, (db->sms + nfb - 1) / nfb);
        int64_t cr = (db->n + chunks - 1) / chunks;
        cr = (cr + kMRows - 1) / kMRows * kMRows;
        p.chunk_rows = cr;
        const int nchunks = (int)((db->n + cr - 1) / cr);
        if (nchunks > 65535) return cudaErrorInvalidValue;
        const int kc = db->dim % 128 == 0 ? 128 : 64;
        const size_t sm = many_smem(db->dim, kc);
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
