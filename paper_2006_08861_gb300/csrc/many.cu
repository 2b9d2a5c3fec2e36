// Exhaustive per-frame top k for many query frames at once (the batched
// selection of the soft-retrieval form and the precision form's FP32 path),
// exact in FP32 like the streaming scan in scan.cu, which serves few frames.
//
// With F frames the streaming scan reduces every (row, frame) distance across
// the 32 lanes of a warp; with hundreds of frames the work is a dense
// contraction, so here it runs on the tensor cores in the expanded form
//     e(f, r) = ||x_r||_w^2 + ||q_f||_w^2 - 2 (w q_f) . x_r
// over the database's FP16 copy (f16_many_kernel: tcgen05.mma kind::f16, the
// frames' w q resident in tensor memory, database rows streamed by TMA). The
// filter keeps a pair when e <= thr_f = bound_f + margin_f, where margin_f
// bounds |e - exact distance| for FP16 operands and FP32 accumulation, and
// bound_f is an upper bound on frame f's k-th exact distance taken by the same
// kernel over every 8th row (the k-th smallest of 128 bucket minima, plus one
// margin). Candidates (orderable bits of e, row) are appended to the frame's
// buffer. many_select_kernel, a warp per frame: with e_k the k-th smallest
// candidate e, every row of the exact top k has e <= e_k + 2 margin_f (k rows
// have exact distance <= e_k + margin_f); those rows are re-scored with the
// exact direct form sum w (q - x)^2 and the top k (distance, row) keys
// written. A frame whose buffer overflowed is scanned exhaustively by its warp.
#include <cuda_fp16.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "tc.cuh"

namespace lhr {
namespace {

constexpr int kManyMinFrames = 64;    // fewer frames take the streaming scan
constexpr int kManyMaxFrames = 8192;  // candidate buffers: kMCap keys per frame
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
    const float* mabs;    // nq: absolute margin term added to margin_scale rad^2
    float* thr;           // nq: bound + margin (filter threshold on e)
    float* qn;            // nq: ||q||_w^2
    float* mg;            // nq: margin
    unsigned* cnt;        // nq: candidates seen
    u64* cand;            // nq x kMCap
    float* fT;            // nq: thr - qn + slack, the threshold on u = ||x||_w^2 - 2 (w q) . x
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
        const float margin = p.margin_scale * rad * rad + __ldg(p.mabs + f);
        // each bucket minimum is a filter score, within one margin of its row's exact
        // distance: k distinct rows lie at most bound away
        const float bound = b < 0x7f800000u ? __uint_as_float(b) * (1.0f + 1.0f / 4096.0f) + margin : inf;
        const float thr = bound + margin;
        p.qn[f] = a;
        p.mg[f] = margin;
        p.thr[f] = thr;
        // the pass tests u = fl(||x||_w^2 - 2 (w q) . x) <= fT and keys e = fl(u + qn): a pair
        // with e <= thr has u <= thr - qn up to three roundings of magnitude at most
        // |thr| + |qn| + max ||x||_w^2 each; the slack is four units in the last place of that
        const float slack = 4.0f * 5.9604645e-08f * (fabsf(thr) + a + xnmax);
        p.fT[f] = (thr - a) + slack;
    }
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

// Per frame, one block of kSelWarps warps: e_k = the k-th smallest candidate e
// (each warp keeps the 64 smallest of its share of the 64-key chunks in
// registers, warp 0 merges them), then the exact top k of the candidates with
// e <= e_k + 2 margin (the warps split the candidates; rows re-scored four at a
// time, each warp keeping its own top k, merged at the end); an overflowed
// buffer falls back to an exhaustive exact pass over the frame (the warps split
// the rows, one row per lane).
constexpr int kSelWarps = 4;

__global__ void __launch_bounds__(kSelWarps * 32, 10) many_select_kernel(ManyParams p) {
    __shared__ u64 sh[kSelWarps * 64];
    __shared__ float s_lim;
    const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
    const int f = blockIdx.x;
    if (f >= p.nq) return;
    const unsigned c = __ldcg(p.cnt + f);
    u64 L = kKeyEmpty;  // this warp's exact (distance, row) top k, lane i = i-th
    if (c > (unsigned)kMCap) {
        for (int64_t base = (int64_t)warp * 32; base < p.n; base += kSelWarps * 32) {
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
        for (unsigned base = warp * 64u; base < c; base += kSelWarps * 64u) {
            u64 cur[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const unsigned i = base + e * 32 + lane;
                cur[e] = i < c ? __ldcg(cf + i) : kKeyEmpty;
            }
            const u64 worst = __shfl_sync(kFull, best[1], 31);
            if (!__any_sync(kFull, cur[0] < worst || cur[1] < worst)) continue;
            warp_sort64(cur, lane);
            warp_merge64(best, cur, lane);
        }
#pragma unroll
        for (int e = 0; e < 2; ++e) sh[warp * 64 + e * 32 + lane] = best[e];
        __syncthreads();
        if (warp == 0) {
            for (int w = 1; w < kSelWarps; ++w) {
                const u64 cur[2] = {sh[w * 64 + lane], sh[w * 64 + 32 + lane]};
                warp_merge64(best, cur, lane);
            }
            // element k - 1 of the sorted 64 (layout e * 32 + lane)
            const u64 ek = __shfl_sync(kFull, best[(p.k - 1) / 32], (p.k - 1) % 32);
            if (lane == 0)
                s_lim = (c >= (unsigned)p.k && ek != kKeyEmpty) ? orderable_value(ek) + 2.f * p.mg[f]
                                                               : __int_as_float(0x7f800000);
        }
        __syncthreads();
        const float lim = s_lim;
        // the frame's q and w in registers (D <= 256: at most 8 values per lane)
        constexpr int kMaxPer = 8, kRows = 4;
        const int per = p.D / 32;
        float qv[kMaxPer], wv[kMaxPer];
#pragma unroll
        for (int t = 0; t < kMaxPer; ++t) {
            const int d = lane + 32 * t;
            qv[t] = t < per ? p.Q[(size_t)f * p.D + d] : 0.f;
            wv[t] = t < per ? (p.w ? p.w[d] : 1.f) : 0.f;
        }
        for (unsigned base = warp * 32u; base < c; base += kSelWarps * 32u) {
            const unsigned i = base + lane;
            const u64 v = i < c ? __ldcg(cf + i) : kKeyEmpty;
            unsigned m = __ballot_sync(kFull, i < c && orderable_value(v) <= lim);
            while (m) {
                // up to four rows at a time: their loads in flight together, each summed in
                // the same order (the lane's dimensions in turn, then the butterfly)
                uint32_t r[kRows];
                int nr = 0;
#pragma unroll
                for (int t = 0; t < kRows; ++t) {
                    r[t] = 0u;
                    if (m) {
                        const int j = __ffs(m) - 1;
                        m &= m - 1;
                        r[t] = (uint32_t)__shfl_sync(kFull, v, j);
                        nr = t + 1;
                    }
                }
                float a[kRows];
#pragma unroll
                for (int t = 0; t < kRows; ++t) a[t] = 0.f;
#pragma unroll
                for (int u = 0; u < kMaxPer; ++u) {
                    if (u < per) {
                        float x[kRows];
#pragma unroll
                        for (int t = 0; t < kRows; ++t)
                            x[t] = t < nr ? __ldg(p.X + (size_t)r[t] * p.D + lane + 32 * u) : 0.f;
#pragma unroll
                        for (int t = 0; t < kRows; ++t) {
                            const float diff = qv[u] - x[t];
                            a[t] = p.w ? fmaf(wv[u] * diff, diff, a[t]) : fmaf(diff, diff, a[t]);
                        }
                    }
                }
#pragma unroll
                for (int t = 0; t < kRows; ++t) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) a[t] += __shfl_xor_sync(kFull, a[t], o);
                }
                for (int t = 0; t < nr; ++t) {
                    const u64 key = make_key(a[t], r[t]);
                    if (key < __shfl_sync(kFull, L, p.k - 1)) list_insert(L, key, p.k, lane);
                }
            }
        }
    }
    // the warps' top-k lists merged: 4 x 32 keys, the smallest k
    __syncthreads();
    sh[warp * 32 + lane] = lane < p.k ? L : kKeyEmpty;
    __syncthreads();
    if (warp == 0) {
        // each list is sorted (lane i = i-th), so {list, empty} is a sorted 64-key list and the
        // lists merge pairwise without sorting
        u64 a2[2] = {sh[lane], kKeyEmpty};
        for (int w = 1; w < kSelWarps; ++w) {
            const u64 b2[2] = {sh[w * 32 + lane], kKeyEmpty};
            warp_merge64(a2, b2, lane);
        }
        if (lane < p.k) {
            const u64 Lk = a2[0];
            const size_t o = (size_t)f * p.k + lane;
            if (Lk == kKeyEmpty) {
                p.idx[o] = -1;
                p.dist[o] = __int_as_float(0x7f800000);
            } else {
                const uint32_t r = key_row(Lk);
                p.idx[o] = p.perm ? (int64_t)p.perm[r] : (int64_t)r;
                p.dist[o] = key_dist(Lk);
            }
        }
    }
}

// ------------------------------------------------------------------ FP16 tensor-core pass
// The filter on the tensor cores: u(f, r) = ||x_r||_w^2 - 2 (w q_f) . x_r with
// the dot by tcgen05.mma kind::f16 over FP16 operands (the database copy Xh and
// each frame's w q, both scaled by powers of two; FP32 accumulation), one CTA
// per (128-frame block, row chunk). The block's w q rows are the A operand,
// resident in tensor memory (a frame per TMEM lane, two dimensions per
// column), so shared memory holds only the deep TMA ring that
// streams the database rows (the B operand, 128 rows per tile); the 128 x 128
// accumulators alternate in the rest of TMEM. The epilogue thread of TMEM lane m
// owns frame m over 64 of the tile's rows: per 32 rows the smallest u (three-
// input minima) against the frame's threshold fT_f = thr_f - ||q_f||_w^2 +
// slack decides whether any row passes; the frames with a passing row are
// then taken one at a time by the whole warp (their 32 dots through a small
// shared buffer, lane j testing row j), and the passing pairs keyed (orderable
// e = u + ||q_f||_w^2, row) into the frame's stage in shared memory, appended
// to the frame's buffer at the end with one atomic.
//
// kPilot: the same pipeline over every kF16PilotStride-th row (a strided tensor
// map, no copy) writes bucket minima instead: per frame and 32 sample rows the
// smallest e, clamped at 0, into bucket (sample row / 32) mod 128 by atomic
// minimum. Minima of distinct buckets are distinct rows, each within the margin
// of its exact distance, so the k-th smallest plus one margin bounds the
// frame's k-th exact distance.
using namespace tc;
constexpr int kFT = 128;                 // frames per CTA (UMMA M, TMEM lanes)
constexpr int kFN = 128;                 // database rows per tile (UMMA N)
constexpr int kFMaxAcc = 3;              // 128-column accumulators beside the resident frames
constexpr int kFEpiWarps = 8;            // two per TMEM lane quadrant, 64 rows each
constexpr int kFThreads = 64 + 32 * kFEpiWarps;
constexpr int kFMaxStages = 14;
constexpr int kFStage = 16;              // staged candidates per (frame, epilogue half) of the CTA
constexpr int kFSlice = kFN * kTcSliceBytes;  // 16 KB: one 128-byte K slice of 128 rows
constexpr int kF16PilotStride = 8;        // pilot sample: every 8th row

struct F16Params {
    int64_t n;            // rows of this pass (sample rows for the pilot)
    int slices, stages;   // D / 64; TMA ring depth
    int nacc;             // accumulators (TMEM columns 0, 128, ...)
    int a_col;            // first TMEM column of the frames' operand
    int64_t chunk_rows;
    int64_t xn_stride;    // pass row r has norm xn[r * xn_stride]
    const float* xn;      // ||x||_w^2 per database row
    const uint32_t* wqh;  // nq x D / 2: per frame FP16 pairs of w q s_f (s_f a power of 2)
    const float* fc;      // per frame: -2 / (s_x s_f), the scale of the accumulated dot in u
    const float* fT;      // per frame: threshold on u (main pass)
    const float* qn;      // per frame: ||q||_w^2
    unsigned* cnt;        // per frame: candidates seen
    u64* cand;            // per frame: kMCap candidate keys (orderable e, row)
    unsigned* bmin;       // pilot: per frame kMBuckets bucket minima (float bits)
    int nq;
    int* err;
};

// Smallest u = fl(xn_j + c v_j) over a group's 32 rows (xn from shared memory).
__device__ __forceinline__ float f16_min_u(const uint32_t (&v)[32], float c, const float* sxn) {
    // packed pairs: each half is the same correctly rounded fma as fmaf(c, v_j, xn_j)
    const float4* x4 = reinterpret_cast<const float4*>(sxn);
    const float2 cc = make_float2(c, c);
    float mn = __int_as_float(0x7f800000);
#pragma unroll
    for (int j4 = 0; j4 < 8; ++j4) {
        const float4 x = x4[j4];
        const float2 u01 = __ffma2_rn(cc, make_float2(__uint_as_float(v[4 * j4]), __uint_as_float(v[4 * j4 + 1])),
                                      make_float2(x.x, x.y));
        const float2 u23 = __ffma2_rn(cc, make_float2(__uint_as_float(v[4 * j4 + 2]), __uint_as_float(v[4 * j4 + 3])),
                                      make_float2(x.z, x.w));
        mn = fmin3(mn, u01.x, u01.y);
        mn = fmin3(mn, u23.x, u23.y);
    }
    return mn;
}

// Main pass, one group of 32 rows (the warp's lanes own frames m0 .. m0 + 31):
// the frames with a passing row, one at a time, through the warp.
__device__ __forceinline__ void f16_group(const F16Params& p, const uint32_t (&v)[32], const float* sxn, float* tb,
                                         float c_own, float T_own, float qn_own, unsigned& cnt_own, u64* stage_h,
                                         int m0, int fbase, int64_t row_g0, int lane) {
    unsigned ev = __ballot_sync(kFull, f16_min_u(v, c_own, sxn) <= T_own);
    const unsigned lt = (1u << lane) - 1u;
    while (ev) {
        const int L = __ffs(ev) - 1;
        ev &= ev - 1;
        if (lane == L) {
            float4* d = reinterpret_cast<float4*>(tb);
#pragma unroll
            for (int j = 0; j < 8; ++j)
                d[j] = make_float4(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]),
                                   __uint_as_float(v[4 * j + 2]), __uint_as_float(v[4 * j + 3]));
        }
        __syncwarp();
        const float u = fmaf(__shfl_sync(kFull, c_own, L), tb[lane], sxn[lane]);  // frame L, row row_g0 + lane
        const float TL = __shfl_sync(kFull, T_own, L);
        const float qL = __shfl_sync(kFull, qn_own, L);
        const unsigned cL = __shfl_sync(kFull, cnt_own, L);
        const bool ps = u <= TL;
        const unsigned pm = __ballot_sync(kFull, ps);
        if (ps) {
            const unsigned pos = cL + __popc(pm & lt);
            const u64 key = orderable_key(u + qL, (uint32_t)(row_g0 + lane));
            if (pos < (unsigned)kFStage) {
                stage_h[(m0 + L) * kFStage + pos] = key;
            } else {
                const int f = fbase + m0 + L;
                const unsigned g = atomicAdd(p.cnt + f, 1u);
                if (g < (unsigned)kMCap) p.cand[(size_t)f * kMCap + g] = key;
            }
        }
        if (lane == L) cnt_own += __popc(pm);
        __syncwarp();
    }
}

template <bool kPilot>
__global__ void __launch_bounds__(kFThreads, 1) f16_many_kernel(const __grid_constant__ CUtensorMap tmX, const F16Params p) {
    extern __shared__ unsigned char smem_raw[];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int chunk = blockIdx.x, fblock = blockIdx.y;
    unsigned char* smem =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int stages = p.stages;
    unsigned char* sX = smem;                                                // stages x 16 KB: database slices
    u64* stage = reinterpret_cast<u64*>(sX + (size_t)stages * kFSlice);      // main: 2 x kFT x kFStage keys
    float* sxn_all = reinterpret_cast<float*>(stage + (kPilot ? 0 : 2 * kFT * kFStage));  // 64 per epilogue warp
    float* tb_all = sxn_all + kFEpiWarps * 64;                               // 32 per epilogue warp
    u64* full = reinterpret_cast<u64*>(tb_all + kFEpiWarps * 32);
    u64* empty = full + kFMaxStages;
    u64* a_full = empty + kFMaxStages;
    u64* acc_full = a_full + 1;
    u64* acc_empty = acc_full + kFMaxAcc;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(acc_empty + kFMaxAcc);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

    const int64_t row0 = (int64_t)chunk * p.chunk_rows;
    const int64_t row1 = min(p.n, row0 + p.chunk_rows);
    const int ntiles = row1 > row0 ? (int)((row1 - row0 + kFN - 1) / kFN) : 0;
    const int fbase = fblock * kFT;
    const int nacc = p.nacc;
    constexpr int kElemPerSlice = kTcSliceBytes / 2;  // 64 FP16 values
    constexpr int kColPerSlice = kElemPerSlice / 2;   // TMEM columns of A per slice (two values each)
    constexpr int kMmaK = 16;                         // FP16 values per MMA (32 bytes, 8 TMEM columns)
    constexpr int kMmaPerSlice = kElemPerSlice / kMmaK;
    constexpr uint32_t kIdesc = tc_idesc(kTcF16, kFN);

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(a_full, kFEpiWarps);
        for (int i = 0; i < kFMaxAcc; ++i) {
            mbar_init(&acc_full[i], 1);
            mbar_init(&acc_empty[i], kFEpiWarps);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    if (warp == 0) {
        if (lane == 0) {
            int b_issued = 0, st = 0;
            uint32_t ph = 0;
            for (int t = 0; t < ntiles && !*abort_flag; ++t) {
                const int r = (int)(row0 + (int64_t)t * kFN);
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
                for (int it = b_issued > stages ? b_issued - stages : 0; it < b_issued; ++it)
                    mbar_wait(&full[it % stages], (uint32_t)((it / stages) & 1), nullptr);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            bool ok = mbar_wait(a_full, 0u, abort_flag);
            tc_fence_after();
            int st = 0;
            uint32_t ph = 0;
            for (int t = 0; ok && t < ntiles; ++t) {
                const int a = t % nacc;
                if (!mbar_wait(&acc_empty[a], (uint32_t)((t / nacc) & 1) ^ 1u, abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(a * kFN);
                for (int s = 0; s < p.slices; ++s) {
                    if (!mbar_wait(&full[st], ph, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t x_base = smem_u32(sX + (size_t)st * kFSlice);
                    const uint32_t a_tmem = tmem + (uint32_t)(p.a_col + s * kColPerSlice);
#pragma unroll
                    for (int kk = 0; kk < kMmaPerSlice; ++kk)
                        tc_mma_tmem_a<kTcF16>(d_tmem, a_tmem + (uint32_t)(kk * kMmaK / 2),
                                              sw128_desc(x_base + kk * kMmaK * 2), kIdesc, (s | kk) != 0 ? 1u : 0u);
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
        // ------------------------------------------------ epilogue: thread = frame (TMEM lane)
        const int ew = warp - 2;
        const int quad = warp & 3;                 // TMEM lanes 32 quad .. 32 quad + 31
        const int h = ew / 4;                      // rows 64 h .. 64 h + 63 of each tile
        const int m0 = quad * 32, m = m0 + lane;
        const int f = fbase + m;
        const uint32_t lane_base = tmem + ((uint32_t)m0 << 16);
        // the frame's FP16 pairs into TMEM columns a_col + d / 2 (slices alternate between the two halves)
        for (int s = h; s < p.slices; s += 2) {
            uint32_t r[32];
            const uint4* src = reinterpret_cast<const uint4*>(p.wqh + ((size_t)f * p.slices + s) * kColPerSlice);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const uint4 x = f < p.nq ? __ldg(src + j) : make_uint4(0u, 0u, 0u, 0u);
                r[4 * j] = x.x;
                r[4 * j + 1] = x.y;
                r[4 * j + 2] = x.z;
                r[4 * j + 3] = x.w;
            }
            tmem_st32(lane_base + (uint32_t)(p.a_col + s * kColPerSlice), r);
        }
        tmem_st_wait();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(a_full);

        const float inf = __int_as_float(0x7f800000);
        const float T_own = !kPilot && f < p.nq ? __ldg(p.fT + f) : -inf;
        const float qn_own = f < p.nq ? __ldg(p.qn + f) : 0.f;
        const float c_own = f < p.nq ? __ldg(p.fc + f) : 0.f;
        float* sxn = sxn_all + ew * 64;
        float* tb = tb_all + ew * 32;
        u64* stage_h = stage + (size_t)h * kFT * kFStage;
        unsigned cnt_own = 0;
        // the tile's row norms one tile ahead (+inf past the chunk: no pair passes there)
        auto xn_of = [&](int tt, int c) {
            const int64_t r = row0 + (int64_t)tt * kFN + h * 64 + c;
            return tt < ntiles && r < row1 ? __ldg(p.xn + r * p.xn_stride) : inf;
        };
        float xa_n = xn_of(0, lane), xb_n = xn_of(0, 32 + lane);
        for (int t = 0; t < ntiles; ++t) {
            const int a = t % nacc;
            const int64_t rg = row0 + (int64_t)t * kFN + h * 64;  // first row of this warp's 64
            __syncwarp();
            sxn[lane] = xa_n;
            sxn[32 + lane] = xb_n;
            xa_n = xn_of(t + 1, lane);
            xb_n = xn_of(t + 1, 32 + lane);
            if (!mbar_wait(&acc_full[a], (uint32_t)((t / nacc) & 1), abort_flag)) {
                if (lane == 0) {
                    *abort_flag = 1;
                    record_error(p.err, kErrTimeout);
                }
                break;
            }
            tc_fence_after();
            const uint32_t tbase = lane_base + (uint32_t)(a * kFN + h * 64);
            uint32_t va[32], vb[32];
            tmem_ld32_issue(tbase, va);
            tmem_ld32_issue(tbase + 32u, vb);
            tmem_ld_wait(va);  // waits for both loads; the second wait only names vb's registers
            tmem_ld_wait(vb);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[a]);
            if (kPilot) {
                const int bucket = (int)((rg >> 5) & (kMBuckets - 1));
                const float mna = f16_min_u(va, c_own, sxn), mnb = f16_min_u(vb, c_own, sxn + 32);
                if (f < p.nq) {
                    if (mna < inf) atomicMin(p.bmin + (size_t)f * kMBuckets + bucket, __float_as_uint(fmaxf(mna + qn_own, 0.f)));
                    if (mnb < inf)
                        atomicMin(p.bmin + (size_t)f * kMBuckets + ((bucket + 1) & (kMBuckets - 1)),
                                  __float_as_uint(fmaxf(mnb + qn_own, 0.f)));
                }
            } else {
                f16_group(p, va, sxn, tb, c_own, T_own, qn_own, cnt_own, stage_h, m0, fbase, rg, lane);
                f16_group(p, vb, sxn + 32, tb, c_own, T_own, qn_own, cnt_own, stage_h, m0, fbase, rg + 32, lane);
            }
        }
        if (!kPilot) {
            // this frame's stage (written by the warp's lanes) to its buffer: one atomic
            __syncwarp();
            const unsigned n = min(cnt_own, (unsigned)kFStage);
            if (f < p.nq && n > 0) {
                const unsigned pos = atomicAdd(p.cnt + f, n);
                for (unsigned i = 0; i < n; ++i)
                    if (pos + i < (unsigned)kMCap) p.cand[(size_t)f * kMCap + pos + i] = stage_h[m * kFStage + i];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

// Per frame (one warp): w q scaled by s_f = 2^(15 - e) (max |w q| = g 2^e, g in
// [0.5, 1)) as FP16 pairs, the A operand row; ||q||_w^2 (summed as
// many_bound_kernel does); fc = -2 / (s_x s_f), the scale of the accumulated dot
// in u; and mabs, the absolute part of the filter margin: a value in FP16's
// subnormal range is off by at most 2^-25 after scaling, which over D products
// moves the dot by less than D max|w q| 2^-23 / s_x, and e by twice that.
__global__ void f16_prep_kernel(const float* Q, const float* w, int nq, int D, float sx, __half2* wqh, float* qn,
                                float* fc, float* mabs) {
    const int lane = threadIdx.x & 31;
    const int f = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (f >= nq) return;
    const float* q = Q + (size_t)f * D;
    float a = 0.f, mx = 0.f;
    for (int d = lane; d < D; d += 32) {
        const float v = w ? w[d] * q[d] : q[d];
        a = fmaf(v, q[d], a);
        mx = fmaxf(mx, fabsf(v));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(kFull, a, o);
        mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
    }
    int ex = 0;
    frexpf(mx, &ex);
    const float sf = ldexpf(1.0f, 15 - ex);
    for (int d2 = lane; d2 < D / 2; d2 += 32) {
        const float v0 = w ? w[2 * d2] * q[2 * d2] : q[2 * d2];
        const float v1 = w ? w[2 * d2 + 1] * q[2 * d2 + 1] : q[2 * d2 + 1];
        wqh[(size_t)f * (D / 2) + d2] = __floats2half2_rn(v0 * sf, v1 * sf);
    }
    if (lane == 0) {
        qn[f] = a;
        fc[f] = -2.0f / sx / sf;
        mabs[f] = (float)D * mx * ldexpf(1.0f, -21) / sx;
    }
}

size_t f16_smem(int stages, bool pilot) {
    return 1024 + (size_t)stages * kFSlice + (pilot ? 0 : (size_t)2 * kFT * kFStage * sizeof(u64)) +
           (size_t)kFEpiWarps * 96 * sizeof(float) + (2 * kFMaxStages + 1 + 2 * kFMaxAcc) * sizeof(u64) + 16;
}

int f16_stages(bool pilot) {
    const size_t fixed = f16_smem(0, pilot);
    const size_t lim = 227 * 1024;
    const int fit = fixed < lim ? (int)((lim - fixed) / kFSlice) : 0;
    return std::min(kFMaxStages, fit);
}

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

// Many frames at once: the tensor-core filter over the FP16 copy. Fewer
// frames (or a batch beyond the candidate buffers) take the streaming scan.
bool many_eligible(const lhr_db* db, int nq, int k) {
    return db->Xh != nullptr && db->n_sub == 1 && nq >= kManyMinFrames && nq <= kManyMaxFrames && k >= 1 && k <= 32;
}

namespace {

struct ManyLayout {
    size_t thr, qn, mg, cnt, cand, fT, wqh, fc, mabs, bmin, total;
};

ManyLayout many_layout(const lhr_db* db, int nq) {
    ManyLayout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t r = off;
        off += a256(bytes);
        return r;
    };
    const size_t f4 = (size_t)nq * sizeof(float);
    L.thr = take(f4);
    L.qn = take(f4);
    L.mg = take(f4);
    L.cnt = take((size_t)nq * sizeof(unsigned));
    L.cand = take((size_t)nq * kMCap * sizeof(u64));
    L.fT = take(f4);
    L.wqh = take((size_t)nq * db->dim * 2);
    L.fc = take(f4);
    L.mabs = take(f4);
    L.bmin = take((size_t)nq * kMBuckets * sizeof(unsigned));
    L.total = off;
    return L;
}

// Row chunks per frame block so that the CTAs fill whole waves of the SMs as
// far as possible (waves x tiles per CTA, plus a per-CTA fixed cost of about
// two tiles: the frames' operand and the pipeline's fill).
int f16_chunks(int nfb, int sms, int64_t n) {
    const int64_t tiles = (n + kFN - 1) / kFN;
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

// One pass of f16_many_kernel (the pilot over every kF16PilotStride-th row, or
// the main pass).
template <bool kPilot>
cudaError_t f16_pass(const lhr_db* db, int nq, F16Params t, cudaStream_t stream) {
    const int D = db->dim;
    const int64_t stride = kPilot ? kF16PilotStride : 1;
    t.n = (db->n + stride - 1) / stride;
    t.xn_stride = stride;
    CUtensorMap tmX;
    if (!make_map(&tmX, db->Xh, t.n, D, kTcF16, kFN, stride * D)) return cudaErrorInvalidValue;
    t.slices = D / 64;
    // TMEM: three accumulators at columns 0, 128, 256, the frames' D / 2 columns from 384
    t.nacc = 3;
    t.a_col = 384;
    t.stages = f16_stages(kPilot);
    if (t.stages < 2) return cudaErrorInvalidValue;
    const int nfb = (nq + kFT - 1) / kFT;
    if (nfb > 65535) return cudaErrorInvalidValue;
    const int nchunks = f16_chunks(nfb, db->sms, t.n);
    const int64_t cr = (t.n + nchunks - 1) / nchunks;
    t.chunk_rows = (cr + kFN - 1) / kFN * kFN;
    const int grid_x = (int)((t.n + t.chunk_rows - 1) / t.chunk_rows);
    const size_t sm = f16_smem(t.stages, kPilot);
    cudaError_t e = cudaFuncSetAttribute(f16_many_kernel<kPilot>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    ProfScope ps(kPilot ? "f16_pilot_kernel" : "f16_many_kernel", stream);
    f16_many_kernel<kPilot><<<dim3(grid_x, nfb), kFThreads, sm, stream>>>(tmX, t);
    return cudaGetLastError();
}

}  // namespace

size_t many_scratch_bytes(const lhr_db* db, int nq) { return many_layout(db, nq).total; }

cudaError_t launch_many(const lhr_db* db, const float* q, int nq, int k, const float* w, const float* xn,
                        const float* xmax_w, float margin_scale, int64_t* idx, float* dist, void* scratch,
                        cudaStream_t stream) {
    if (!many_eligible(db, nq, k)) return cudaErrorInvalidValue;
    const ManyLayout L = many_layout(db, nq);
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
    unsigned* bmin = reinterpret_cast<unsigned*>(base + L.bmin);
    p.bmin = bmin;
    // FP16 operands (11-bit significands, rounded to nearest): each product
    // w q_d x_d is off by at most (2^-10 + 2^-22) of its magnitude, so 2 |dot
    // error| <= (2^-10 + 2^-22) 2 ||q||_w ||x||_w <= (2^-11 + 2^-23) rad^2 (plus the
    // subnormal term mabs); the FP32 term is doubled for the tensor core's own
    // summation order.
    p.margin_scale = 2.f * margin_scale + 1.0f / 2048.f * 1.01f;
    p.xmax = (float)(sqrt((double)db->xnorm_max) * 1.0001);
    p.xmax_w = xmax_w;
    p.thr = reinterpret_cast<float*>(base + L.thr);
    p.qn = reinterpret_cast<float*>(base + L.qn);
    p.mg = reinterpret_cast<float*>(base + L.mg);
    p.cnt = reinterpret_cast<unsigned*>(base + L.cnt);
    p.cand = reinterpret_cast<u64*>(base + L.cand);
    p.fT = reinterpret_cast<float*>(base + L.fT);
    p.mabs = reinterpret_cast<const float*>(base + L.mabs);
    p.perm = db->perm;
    p.idx = idx;
    p.dist = dist;
    p.err = db->err;
    float* fc = reinterpret_cast<float*>(base + L.fc);
    float* mabs = reinterpret_cast<float*>(base + L.mabs);
    __half2* wqh = reinterpret_cast<__half2*>(base + L.wqh);
    cudaError_t e = cudaMemsetAsync(p.cnt, 0, (size_t)nq * sizeof(unsigned), stream);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(bmin, 0xff, (size_t)nq * kMBuckets * sizeof(unsigned), stream)) != cudaSuccess) return e;
    {
        ProfScope ps("f16_prep_kernel", stream);
        f16_prep_kernel<<<(nq + 7) / 8, 256, 0, stream>>>(q, w, nq, db->dim, db->xh_scale, wqh, p.qn, fc, mabs);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    F16Params t{};
    t.xn = xn;
    t.wqh = reinterpret_cast<const uint32_t*>(wqh);
    t.fc = fc;
    t.fT = p.fT;
    t.qn = p.qn;
    t.cnt = p.cnt;
    t.cand = p.cand;
    t.bmin = bmin;
    t.nq = nq;
    t.err = db->err;
    // the pilot's bucket minima, the bound and thresholds, the full pass, the exact re-score
    if ((e = f16_pass<true>(db, nq, t, stream)) != cudaSuccess) return e;
    {
        ProfScope ps("many_bound_kernel", stream);
        many_bound_kernel<<<(nq + 7) / 8, 256, 0, stream>>>(p);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = f16_pass<false>(db, nq, t, stream)) != cudaSuccess) return e;
    {
        ProfScope ps("many_select_kernel", stream);
        many_select_kernel<<<nq, kSelWarps * 32, 0, stream>>>(p);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace lhr
