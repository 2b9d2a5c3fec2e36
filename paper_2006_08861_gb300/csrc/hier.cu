// Fused coarse-to-fine retrieval and Algorithm 2 for a small request: up to
// 8 query frames (one window of M frames, §3.1) in a single cooperative
// launch of one CTA per SM. The steps are those of coarse.cu and aggregate.cu
// (same keys, same tie rules, same tests); only the scheduling differs: a
// building-scale request is a few microseconds of work, so instead of four
// kernels with mostly idle SMs the whole GPU walks through four phases:
//   A  every CTA scores its slice of rows on the coarse prefix for every frame
//      (packed FP32 FMAs), writes the distances to scratch and counts them in
//      per-frame histograms of a 1/32-octave digit of the distance;
//   -- grid barrier
//   B  every CTA locates, per frame, the bin holding the S-th key (one warp per
//      frame), takes its rows below that bin (direct) and inside it
//      (boundary), re-scores each on the full feature (one warp per row) and
//      appends the keys with one global atomic per (frame, list) and chunk;
//   -- grid barrier
//   C  CTA f cuts frame f's boundary list at its need-th coarse key (radix
//      select: exactly S rows in all) and selects the top k of the
//      shortlist's full keys (radix select, then one warp sorts the k); a
//      frame whose boundary bin overflowed is refined and ranked by CTA f
//      alone, over the frame's distances; CTAs with no frame leave;
//   -- a done counter (only the window CTAs wait for it)
//   D  CTA w runs Algorithm 2 on window w's candidates (one warp).
// The grid barrier is a global arrival counter; every wait gives up after
// kWaitLimitNs and records LHR_ERR_TIMEOUT. The words that must be zero at the
// start (histograms, per-frame counters, grid words) sit in a control block
// that the launch leaves zeroed (hier_leave), so a stream that keeps its block
// issues no memset before the next launch.
#include "aggregate.cuh"
#include "common.cuh"
#include "internal.h"
#include "select.cuh"

namespace lhr {
namespace {

using namespace sel;

constexpr int kHT = 512;  // threads per CTA
constexpr int kHW = kHT / 32;
constexpr int kHBinCap = 4096;
constexpr int kHMaxShort = 4096;
constexpr int kHStage = 8 * kBins * 4 + 256;  // phase A: offset of the warps' staging buffers in the region
constexpr int kHRegion = kHStage + kHW * 2 * 32 * 8 * 16;  // shared region reused by every phase
constexpr int kHCtl = 8;             // control words per frame
enum { cDirect = 0, cInBin = 1, cRefine = 2, cNeed = 3 };
static_assert((2 * kHBinCap + kHMaxShort + 32) * 8 + kBins * 4 <= kHRegion, "phase C's arrays fit the region");
static_assert(kHStage >= 8 * kBins * 4 + 16 * 4 && kHStage % 16 == 0, "staging follows the histograms");

// Coarse digit of a distance d >= 0: 8 exponent bits and the top 5 mantissa
// bits, i.e. 1/32-octave bins, over 2^-32 .. 2^32; smaller and larger values
// share the end bins. It is a monotone function of the key's top bits
// (key >> 50), so each bin is one key range (bin_range).
constexpr unsigned kDigitBase = (127u - 32u) << 5;
__device__ __forceinline__ unsigned coarse_digit(float d) {
    const unsigned v = __float_as_uint(d) >> 18;
    return v <= kDigitBase ? 0u : min(v - kDigitBase, (unsigned)kBins - 1u);
}
__device__ __forceinline__ void bin_range(unsigned b, u64& lo, u64& hi) {  // keys of bin b: [lo, hi]
    lo = b == 0 ? 0ull : (u64)(kDigitBase + b) << 50;
    hi = b == (unsigned)kBins - 1u ? ~0ull : ((u64)(kDigitBase + b + 1u) << 50) - 1ull;
}

struct HierParams {
    const float* Xc;
    int dc;
    const float* X;
    int D;
    int64_t n;
    const float* Q;
    int nf;
    int S, k;
    float* dcbuf;     // nf x n coarse distances
    unsigned* hist;   // nf x kBins    } zero when the launch starts,
    unsigned* ctl;    // nf x kHCtl    } and zero again when it ends
    unsigned* bar;    // barrier arrivals, abort flag, frames done, CTAs gone }
    u64* bins;        // nf x kHBinCap coarse keys of the boundary rows
    u64* fkb;         // nf x kHBinCap their full keys (same slots)
    u64* fkd;         // nf x kHMaxShort full keys of the direct rows
    int64_t* idx;     // nf x k
    float* dist;
    u64* ctk;         // nf x k tile keys of the results (Algorithm 2 reads them)
    agg::AggParams ap;  // windows over the frames (per_frame = k), ap.a.nw of them; nw = 0: none
    int* err;
};

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// 16-byte asynchronous global -> shared copy (zero-filled when bytes = 0) and
// its group bookkeeping.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, unsigned bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Bounded grid-wide barrier (all CTAs are co-resident: cooperative launch).
// bar[0] counts arrivals over the whole launch (zero when it starts); the j-th
// barrier completes when it reaches j * gridDim.x, so the last arrival has
// nothing more to do.
__device__ bool grid_sync(unsigned* bar, unsigned& epoch, volatile int* abort_sm, int* err) {
    __syncthreads();
    epoch += gridDim.x;
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned arrived = atomicAdd(&bar[0], 1u) + 1u;
        if (arrived < epoch) {
            volatile unsigned* cnt = bar;
            const u64 t0 = globaltimer();
            while (*cnt < epoch) {
                if (globaltimer() - t0 > kWaitLimitNs) {
                    *abort_sm = 1;
                    record_error(err, kErrTimeout);
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *abort_sm == 0;
}

// Full-feature squared distance of row r to frame q, by one warp.
template <int CPL>
__device__ __forceinline__ float warp_dist(const float* X, int D, const float* q, uint32_t r, int lane) {
    const int D4 = D / 4;
    const float4* xr = reinterpret_cast<const float4*>(X + (size_t)r * D);
    const float4* qr = reinterpret_cast<const float4*>(q);
    float2 acc = f2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < CPL; ++j) {
        const int c = lane + 32 * j;
        if (c < D4) {
            const float4 x = __ldg(xr + c), qv = __ldg(qr + c);
            const float2 a = __ffma2_rn(f2(x.x, x.y), f2(-1.f, -1.f), f2(qv.x, qv.y));
            const float2 b = __ffma2_rn(f2(x.z, x.w), f2(-1.f, -1.f), f2(qv.z, qv.w));
            acc = __ffma2_rn(a, a, acc);
            acc = __ffma2_rn(b, b, acc);
        }
    }
    float d = acc.x + acc.y;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(kFull, d, o);
    return d;
}

// Full-feature distances of up to 4 (row, frame) pairs by one warp, all loads
// issued before any reduction (the rows usually come from HBM). Entries with
// row < 0 are skipped (their result is unspecified).
template <int CPL>
__device__ __forceinline__ void warp_dist4(const float* X, int D, const float* Q, const int* rows, const int* frames,
                                           float* out, int lane) {
    const int D4 = D / 4;
    float4 x[4][CPL];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float4* xr = reinterpret_cast<const float4*>(X + (size_t)max(rows[i], 0) * D);
#pragma unroll
        for (int j = 0; j < CPL; ++j) {
            const int c = lane + 32 * j;
            x[i][j] = (rows[i] >= 0 && c < D4) ? __ldg(xr + c) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float4* qr = reinterpret_cast<const float4*>(Q + (size_t)frames[i] * D);
        float2 acc = f2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < CPL; ++j) {
            const int c = lane + 32 * j;
            if (rows[i] >= 0 && c < D4) {
                const float4 qv = __ldg(qr + c);
                const float2 a = __ffma2_rn(f2(x[i][j].x, x[i][j].y), f2(-1.f, -1.f), f2(qv.x, qv.y));
                const float2 b = __ffma2_rn(f2(x[i][j].z, x[i][j].w), f2(-1.f, -1.f), f2(qv.z, qv.w));
                acc = __ffma2_rn(a, a, acc);
                acc = __ffma2_rn(b, b, acc);
            }
        }
        out[i] = acc.x + acc.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int i = 0; i < 4; ++i) out[i] += __shfl_xor_sync(kFull, out[i], o);
    }
}

// Full-feature key of a row whose phase-B queue was full, by its own thread
// (rare: the queue holds 8 rows per thread).
__device__ __forceinline__ void rescore_alone(const float* X, const float* q, int D, int64_t row, u64* out) {
    const float4* xr = reinterpret_cast<const float4*>(X + (size_t)row * D);
    const float4* qr = reinterpret_cast<const float4*>(q);
    float a = 0.f;
    for (int c = 0; c < D / 4; ++c) {
        const float4 xv = __ldg(xr + c), qv = __ldg(qr + c);
        a = fmaf(qv.x - xv.x, qv.x - xv.x, a);
        a = fmaf(qv.y - xv.y, qv.y - xv.y, a);
        a = fmaf(qv.z - xv.z, qv.z - xv.z, a);
        a = fmaf(qv.w - xv.w, qv.w - xv.w, a);
    }
    *out = make_key(a, (uint32_t)row);
}

// Writes frame f's final top k: the keys of fk[0, total) that are <= kth
// (at most 32 of them, distinct) are gathered, sorted by warp 0 and written.
__device__ void write_topk(const HierParams& p, int f, const u64* fk, unsigned total, u64 kth, u64* outk,
                           unsigned* res) {
    const int t = threadIdx.x, lane = t % 32;
    if (t == 0) res[3] = 0u;
    __syncthreads();
    for (unsigned i = t; i < total; i += kHT) {
        const u64 key = fk[i];
        if (key <= kth) {
            const unsigned pos = atomicAdd(&res[3], 1u);
            if (pos < 32u) outk[pos] = key;
        }
    }
    __syncthreads();
    if (t < 32) {
        const unsigned cnt = min(res[3], 32u);
        u64 v = (unsigned)lane < cnt ? outk[lane] : kKeyEmpty;
#pragma unroll
        for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                const u64 o = __shfl_xor_sync(kFull, v, stride);
                const bool keep_min = ((lane & stride) == 0) == ((lane & size) == 0);
                v = keep_min ? (o < v ? o : v) : (o > v ? o : v);
            }
        }
        if (lane < p.k) {
            const size_t o = (size_t)f * p.k + lane;
            if (v == kKeyEmpty) {
                p.idx[o] = -1;
                p.dist[o] = __int_as_float(0x7f800000);
            } else {
                const uint32_t r = key_row(v);
                p.idx[o] = (int64_t)r;
                p.dist[o] = key_dist(v);
                if (p.ctk != nullptr) p.ctk[o] = agg::tile_key(__ldg(p.ap.tile + 2 * r), __ldg(p.ap.tile + 2 * r + 1));
            }
        }
    }
    __syncthreads();
}

// Top k (k <= 32) of at most kHT distinct keys, by warps: each warp sorts
// its 32 keys (one per lane, a bitonic network), then four levels of
// pairwise merges keep the 32 smallest -- warp w takes its list and warp w +
// h's reversed, the elementwise minima (a bitonic sequence holding the 32
// smallest) sorted by a half-cleaner cascade -- and warp 0 writes the first k.
// `lists` holds kHW x 32 keys.
__device__ void select_topk_small(const HierParams& p, int f, const u64* fk, unsigned total, u64* lists,
                                  unsigned* res) {
    const int t = threadIdx.x, warp = t / 32, lane = t % 32;
    u64 v = (unsigned)t < total ? fk[t] : kKeyEmpty;
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const u64 o = __shfl_xor_sync(kFull, v, stride);
            const bool keep_min = ((lane & stride) == 0) == ((lane & size) == 0);
            v = keep_min ? (o < v ? o : v) : (o > v ? o : v);
        }
    }
    lists[warp * 32 + lane] = v;
    __syncthreads();
#pragma unroll
    for (int h = kHW / 2; h >= 1; h >>= 1) {
        if (warp < h) {
            const u64 a = lists[warp * 32 + lane], b = lists[(warp + h) * 32 + (31 - lane)];
            u64 m = a < b ? a : b;
#pragma unroll
            for (int stride = 16; stride > 0; stride >>= 1) {
                const u64 o = __shfl_xor_sync(kFull, m, stride);
                m = (lane & stride) == 0 ? (o < m ? o : m) : (o > m ? o : m);
            }
            lists[warp * 32 + lane] = m;  // warp w's own slot: no other warp reads it at this level
        }
        __syncthreads();
    }
    if (warp == 0 && lane < p.k) {
        const u64 r0 = lists[lane];
        const size_t o = (size_t)f * p.k + lane;
        if (r0 == kKeyEmpty) {
            p.idx[o] = -1;
            p.dist[o] = __int_as_float(0x7f800000);
        } else {
            const uint32_t r = key_row(r0);
            p.idx[o] = (int64_t)r;
            p.dist[o] = key_dist(r0);
            if (p.ctk != nullptr) p.ctk[o] = agg::tile_key(__ldg(p.ap.tile + 2 * r), __ldg(p.ap.tile + 2 * r + 1));
        }
    }
    __syncthreads();
}

// Top k of fk[0, total) (distinct keys) written as frame f's result.
__device__ void select_topk(const HierParams& p, int f, const u64* fk, unsigned total, unsigned* hs, u64* outk,
                            unsigned* res, unsigned* tmp) {
    static_assert(kHW * 32 * sizeof(u64) <= kBins * sizeof(unsigned), "the warp lists fit the histogram space");
    if (total <= (unsigned)kHT && p.k <= 32) {
        select_topk_small(p, f, fk, total, reinterpret_cast<u64*>(hs), res);
        return;
    }
    u64 kth = ~0ull;
    if (total > (unsigned)p.k) {
        // the keys' range first, so the radix passes split it from the start
        u64* mm = reinterpret_cast<u64*>(hs);  // [kHW] minima, [kHW] maxima
        u64 lo = ~0ull, hi = 0ull;
        for (unsigned i = threadIdx.x; i < total; i += kHT) {
            const u64 v = fk[i];
            lo = v < lo ? v : lo;
            hi = v > hi ? v : hi;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const u64 a = __shfl_xor_sync(kFull, lo, o), b = __shfl_xor_sync(kFull, hi, o);
            lo = a < lo ? a : lo;
            hi = b > hi ? b : hi;
        }
        if ((threadIdx.x & 31) == 0) {
            mm[threadIdx.x / 32] = lo;
            mm[kHW + threadIdx.x / 32] = hi;
        }
        __syncthreads();
        lo = ~0ull;
        hi = 0ull;
        for (int w = 0; w < kHW; ++w) {
            lo = mm[w] < lo ? mm[w] : lo;
            hi = mm[kHW + w] > hi ? mm[kHW + w] : hi;
        }
        __syncthreads();
        kth = block_kth_key<kHT>(fk, total, (unsigned)p.k, lo, hi, hs, res, tmp);
    }
    write_topk(p, f, fk, total, kth, outk, res);
}

// Frame f whose boundary bin overflowed: refine the radix select over the
// frame's coarse distances, collect the S rows, re-score and rank them (this
// CTA alone).
template <int CPL>
__device__ void refine_frame(const HierParams& p, int f, unsigned char* region, unsigned* res, unsigned* tmp) {
    const int t = threadIdx.x, warp = t / 32, lane = t % 32;
    unsigned* hsm = reinterpret_cast<unsigned*>(region);               // kBins
    u64* bin_keys = reinterpret_cast<u64*>(hsm + kBins);                // kHBinCap
    u64* fk = bin_keys + kHBinCap;                                      // kHMaxShort: rows, then full keys
    u64* outk = fk + kHMaxShort;                                        // 32
    const float* dcf = p.dcbuf + (size_t)f * p.n;
    unsigned need = (unsigned)p.S;
    for (int i = t; i < kBins; i += kHT) hsm[i] = __ldcg(p.hist + (size_t)f * kBins + i);
    __syncthreads();
    find_bin<kHT>(hsm, need, res, tmp);
    u64 lo, hi;
    bin_range(res[0], lo, hi);
    need -= res[1];
    unsigned in_bin = res[2];
    while (in_bin > (unsigned)kHBinCap && hi > lo) {
        const u64 span = hi - lo;
        const int bits = 64 - __clzll((long long)span);
        const int shift = bits > 11 ? bits - 11 : 0;
        __syncthreads();
        for (int i = t; i < kBins; i += kHT) hsm[i] = 0u;
        __syncthreads();
        for (int64_t r = t; r < p.n; r += kHT) {
            const u64 key = coarse_key(dcf, r);
            if (key >= lo && key <= hi) atomicAdd(&hsm[(unsigned)((key - lo) >> shift)], 1u);
        }
        __syncthreads();
        find_bin<kHT>(hsm, need, res, tmp);
        const u64 nlo = lo + ((u64)res[0] << shift);
        const u64 room = hi - nlo, width = (1ull << shift) - 1ull;
        hi = nlo + (room < width ? room : width);
        lo = nlo;
        need -= res[1];
        in_bin = res[2];
    }
    __syncthreads();
    if (t == 0) {
        res[0] = 0u;
        res[1] = 0u;
    }
    __syncthreads();
    for (int64_t r = t; r < p.n; r += kHT) {
        const u64 key = coarse_key(dcf, r);
        if (key < lo) {
            const unsigned pos = atomicAdd(&res[0], 1u);
            if (pos < (unsigned)kHMaxShort) fk[pos] = (u64)r;
        } else if (key <= hi) {
            const unsigned pos = atomicAdd(&res[1], 1u);
            if (pos < (unsigned)kHBinCap) bin_keys[pos] = key;
        }
    }
    __syncthreads();
    const unsigned direct = min(res[0], (unsigned)kHMaxShort);
    const unsigned nb = min(res[1], (unsigned)kHBinCap);
    need = min(need, nb);
    if (need > 0) {
        const u64 cstar = block_kth_key<kHT>(bin_keys, nb, need, lo, hi, hsm, res, tmp);
        if (t == 0) res[0] = direct;
        __syncthreads();
        for (unsigned i = t; i < nb; i += kHT) {
            const u64 key = bin_keys[i];
            if (key <= cstar) {
                const unsigned pos = atomicAdd(&res[0], 1u);
                if (pos < (unsigned)kHMaxShort) fk[pos] = (u64)key_row(key);
            }
        }
        __syncthreads();
    }
    const unsigned total = min(direct + need, (unsigned)kHMaxShort);
    const float* q = p.Q + (size_t)f * p.D;
    for (unsigned i = warp; i < total; i += kHW) {
        const uint32_t r = (uint32_t)fk[i];
        const float d = warp_dist<CPL>(p.X, p.D, q, r, lane);
        __syncwarp();
        if (lane == 0) fk[i] = make_key(d, r);
    }
    __syncthreads();
    select_topk(p, f, fk, total, hsm, outk, res, tmp);
}

template <int DC4, int CPL>
__device__ __forceinline__ void hier_phases(const HierParams& p) {
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char* region = smem;                                           // kHRegion
    float4* qsc = reinterpret_cast<float4*>(smem + kHRegion);               // 8 frames x DC4
    unsigned* fr = reinterpret_cast<unsigned*>(qsc + 8 * DC4);              // per frame: lo(2) hi(2) flags
    unsigned* res = fr + 8 * 8;                                             // 4
    unsigned* tmp = res + 4;                                                // kHW
    volatile int* abort_sm = reinterpret_cast<volatile int*>(tmp + kHW);
    int* woff = reinterpret_cast<int*>(tmp + kHW + 1);  // window blockIdx.x's frame offsets (phase D)

    const int t = threadIdx.x, warp = t / 32, lane = t % 32;
    const int nf = p.nf;
    const int64_t per = (p.n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = min(p.n, (int64_t)blockIdx.x * per), r1 = min(p.n, r0 + per);
    // Phase A's loads go out first, so that their latency overlaps the set-up.
    // Warp w scores the 32-row blocks r0 + 32 w + i kHT (lane l: row + l),
    // each in DC4 / 8 units of 8 16-byte chunks per row. A unit is copied
    // into one of the warp's two staging buffers with coalesced 16-byte
    // copies (four rows per instruction), chunk c of row r at slot c ^ (r & 7),
    // so that both the copies and the reads of one row per lane hit distinct
    // banks; unit u + 2 is in flight while unit u is scored.
    constexpr int kUnits = DC4 / 8;
    const int dc4 = p.dc / 4;
    float4* stg = reinterpret_cast<float4*>(region + kHStage) + warp * 512;
    const int64_t wrows = r1 - r0 - 32 * warp;
    const int nunits = wrows > 0 ? (int)((wrows + kHT - 1) / kHT) * kUnits : 0;
    auto issue = [&](int u) {
        const int64_t wb = r0 + 32 * warp + (int64_t)(u / kUnits) * kHT;
        const int blk = (u % kUnits) * 8;
        float4* buf = stg + (u & 1) * 256;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int rr = 4 * i + lane / 8, c = blk + (lane & 7);
            const bool ok = wb + rr < r1 && c < dc4;
            const float* src = ok ? p.Xc + (wb + rr) * p.dc + 4 * c : p.Xc;
            cp_async16(buf + rr * 8 + ((lane & 7) ^ (rr & 7)), src, ok ? 16u : 0u);
        }
        cp_async_commit();
    };
    if (nunits > 0) issue(0);
    if (nunits > 1) issue(1);
    if (t == 0) *abort_sm = 0;
    if (t == 0 && (int)blockIdx.x < p.ap.a.nw) {  // read now: phase D starts on them
        woff[0] = __ldg(p.ap.a.offsets + blockIdx.x);
        woff[1] = __ldg(p.ap.a.offsets + blockIdx.x + 1);
    }
    unsigned epoch = 0;  // barrier target (same in every thread)

    // ------------------------------------------------ A: coarse distances + histograms
    // Thread t scores rows r0 + t + i kHT; with at most two such rows each
    // (in_regs) the distances also stay in registers for phase B.
    const bool in_regs = r1 - r0 <= 2 * kHT;
    float dreg[2][8];
    unsigned* hsm = reinterpret_cast<unsigned*>(region);  // nf x kBins
    unsigned* drange = hsm + 8 * kBins;                    // per frame: lowest, highest digit seen
    for (int i = t; i < nf * kBins; i += kHT) hsm[i] = 0u;
    if (t < 8) {
        drange[2 * t] = kBins;
        drange[2 * t + 1] = 0u;
    }
    for (int i = t; i < 8 * DC4; i += kHT) {
        const int f = i / DC4, c = i % DC4;
        qsc[i] = (f < nf && c < dc4) ? reinterpret_cast<const float4*>(p.Q + (size_t)f * p.D)[c]
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    {
        unsigned dlo[8], dhi[8];
#pragma unroll
        for (int f = 0; f < 8; ++f) {
            dlo[f] = kBins;
            dhi[f] = 0u;
        }
        float2 acc[8];
        for (int u = 0; u < nunits; ++u) {
            const int blk = (u % kUnits) * 8;
            if (blk == 0) {
#pragma unroll
                for (int f = 0; f < 8; ++f) acc[f] = f2(0.f, 0.f);
            }
            if (u + 1 < nunits) cp_async_wait<1>();
            else cp_async_wait<0>();
            __syncwarp();
            const float4* buf = stg + (u & 1) * 256;
            float4 x[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) x[c] = buf[lane * 8 + (c ^ (lane & 7))];
            __syncwarp();
            if (u + 2 < nunits) issue(u + 2);
#pragma unroll
            for (int f = 0; f < 8; ++f) {
                if (f >= nf) break;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const float4 qv = qsc[f * DC4 + blk + c];
                    const float2 a = __ffma2_rn(f2(x[c].x, x[c].y), f2(-1.f, -1.f), f2(qv.x, qv.y));
                    const float2 b = __ffma2_rn(f2(x[c].z, x[c].w), f2(-1.f, -1.f), f2(qv.z, qv.w));
                    acc[f] = __ffma2_rn(a, a, acc[f]);
                    acc[f] = __ffma2_rn(b, b, acc[f]);
                }
            }
            if (blk + 8 < DC4) continue;  // the row's prefix continues in the next unit
            const int slot = u / kUnits;
            const int64_t row = r0 + 32 * warp + (int64_t)slot * kHT + lane;
            if (row >= r1) continue;
#pragma unroll
            for (int f = 0; f < 8; ++f) {
                if (f >= nf) break;
                const float d = acc[f].x + acc[f].y;
                p.dcbuf[(size_t)f * p.n + row] = d;
                if (slot == 0) dreg[0][f] = d;
                else if (slot == 1) dreg[1][f] = d;
                const unsigned g = coarse_digit(d);
                dlo[f] = min(dlo[f], g);
                dhi[f] = max(dhi[f], g);
                atomicAdd(&hsm[f * kBins + g], 1u);
            }
        }
#pragma unroll
        for (int f = 0; f < 8; ++f) {
            if (f >= nf) break;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                dlo[f] = min(dlo[f], __shfl_xor_sync(kFull, dlo[f], o));
                dhi[f] = max(dhi[f], __shfl_xor_sync(kFull, dhi[f], o));
            }
            if (lane == 0 && dlo[f] <= dhi[f]) {
                atomicMin(&drange[2 * f], dlo[f]);
                atomicMax(&drange[2 * f + 1], dhi[f]);
            }
        }
    }
    __syncthreads();
    // only the digits this CTA met are flushed
    for (int f = 0; f < nf; ++f) {
        const unsigned lo = drange[2 * f], hi = drange[2 * f + 1];
        for (unsigned g = lo + t; g <= hi; g += kHT) {
            const unsigned v = hsm[f * kBins + g];
            if (v) atomicAdd(&p.hist[(size_t)f * kBins + g], v);
        }
    }
    if (!grid_sync(p.bar, epoch, abort_sm, p.err)) return;

    // ------------------------------------------------ B: boundary bin per frame, collect, re-score
    const bool take_all = p.n <= p.S;
    if (warp < nf) {
        const int f = warp;
        if (take_all) {
            if (lane == 0) {
                *reinterpret_cast<u64*>(&fr[f * 8 + 0]) = ~0ull;
                *reinterpret_cast<u64*>(&fr[f * 8 + 2]) = ~0ull;
                fr[f * 8 + 4] = 0u;
            }
        } else {
            const uint3 b = warp_find_bin(p.hist + (size_t)f * kBins, (unsigned)p.S, lane);
            if (lane == 0) {
                u64 lo, hi;
                bin_range(b.x, lo, hi);
                *reinterpret_cast<u64*>(&fr[f * 8 + 0]) = lo;
                *reinterpret_cast<u64*>(&fr[f * 8 + 2]) = hi;
                fr[f * 8 + 4] = b.z > (unsigned)kHBinCap ? 1u : 0u;
                if (blockIdx.x == 0) {
                    p.ctl[f * kHCtl + cRefine] = fr[f * 8 + 4];
                    p.ctl[f * kHCtl + cNeed] = (unsigned)p.S - b.y;
                }
            }
        }
    }
    __syncthreads();
    {
        // Rows are taken two per thread (rows base + t and base + t + kHT) per
        // round; appends are counted per warp, placed with one global atomic
        // per (frame, list) and round, and queued in shared memory; the CTA's
        // warps re-score the queue (4 rows per warp at a time) when the next
        // round might not fit, and at the end. A row that finds the queue full
        // is re-scored by its own thread.
        constexpr unsigned kQCap = kHT * 8;
        unsigned* wcnt = reinterpret_cast<unsigned*>(region);  // [16][kHW] per-warp counts, then offsets
        unsigned* gbase = wcnt + 16 * kHW;                      // [16] global slot of the CTA's first append
        unsigned* ibase = gbase + 16;                           // [16] queue offsets per (frame, list); [16] fill
        int* q_row = reinterpret_cast<int*>(ibase + 32);        // queue: row
        unsigned* q_meta = reinterpret_cast<unsigned*>(q_row + kQCap);  // queue: slot << 4 | frame << 1 | list
        const unsigned below = (1u << lane) - 1u;
        auto drain = [&](unsigned nitems) {
            for (unsigned i0 = 4 * warp; i0 < nitems; i0 += 4 * kHW) {
                int rows[4], frames[4];
                unsigned meta[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const unsigned i = i0 + u;
                    rows[u] = i < nitems ? q_row[i] : -1;
                    meta[u] = i < nitems ? q_meta[i] : 0u;
                    frames[u] = (int)((meta[u] >> 1) & 7u);
                }
                float d[4];
                warp_dist4<CPL>(p.X, p.D, p.Q, rows, frames, d, lane);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (lane == u && rows[u] >= 0) {
                        const unsigned slot = meta[u] >> 4;
                        const u64 key = make_key(d[u], (uint32_t)rows[u]);
                        if (meta[u] & 1u) p.fkb[(size_t)frames[u] * kHBinCap + slot] = key;
                        else p.fkd[(size_t)frames[u] * kHMaxShort + slot] = key;
                    }
                }
            }
        };
        unsigned qfill = 0;  // same value in every thread
        for (int64_t base = r0; base < r1; base += 2 * kHT) {
            if (qfill + (unsigned)(2 * kHT * nf) > kQCap && qfill > 0) {
                drain(qfill);
                qfill = 0;
                __syncthreads();
            }
            // code[i][f]: 0xffff = row i takes no part in frame f's lists, else
            // list << 15 | rank of the row among the warp's appends to that list
            unsigned code[2][8];
            float dv[2][8];  // coarse distances of the two rows
            // membership first, without warp votes: bit 8 i + f of dm (direct) / bm (boundary)
            unsigned dm = 0u, bm = 0u;
#pragma unroll
            for (int f = 0; f < 8; ++f) {
                if (f >= nf) break;
                const bool refine = fr[f * 8 + 4] != 0u;
                const u64 lo = *reinterpret_cast<const u64*>(&fr[f * 8 + 0]);
                const u64 hi = *reinterpret_cast<const u64*>(&fr[f * 8 + 2]);
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int64_t row = base + t + i * kHT;
                    dv[i][f] = 0.f;
                    if (!refine && row < r1) {
                        dv[i][f] = in_regs ? dreg[i][f] : __ldcg(p.dcbuf + (size_t)f * p.n + row);
                        const u64 key = ((u64)__float_as_uint(dv[i][f]) << 32) | (u64)row;
                        const bool d = take_all || key < lo;
                        const bool b = !d && key <= hi;
                        dm |= (d ? 1u : 0u) << (8 * i + f);
                        bm |= (b ? 1u : 0u) << (8 * i + f);
                    }
                }
            }
            // most warps hold no shortlist row at all: then no per-list votes
            const bool any = __ballot_sync(kFull, (dm | bm) != 0u) != 0u;
#pragma unroll
            for (int f = 0; f < 8; ++f) {
                if (f >= nf) break;
                unsigned mdv[2] = {0u, 0u}, mbv[2] = {0u, 0u};
                if (any) {
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        mdv[i] = __ballot_sync(kFull, (dm >> (8 * i + f)) & 1u);
                        mbv[i] = __ballot_sync(kFull, (bm >> (8 * i + f)) & 1u);
                    }
                }
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const bool d = (dm >> (8 * i + f)) & 1u, b = (bm >> (8 * i + f)) & 1u;
                    const unsigned pre_d = i ? __popc(mdv[0]) : 0u, pre_b = i ? __popc(mbv[0]) : 0u;
                    code[i][f] = d ? pre_d + __popc(mdv[i] & below)
                                   : (b ? 0x8000u | (pre_b + __popc(mbv[i] & below)) : 0xffffu);
                }
                if (lane == 0) {
                    wcnt[(2 * f) * kHW + warp] = __popc(mdv[0]) + __popc(mdv[1]);
                    wcnt[(2 * f + 1) * kHW + warp] = __popc(mbv[0]) + __popc(mbv[1]);
                }
            }
            __syncthreads();
            if (t < 32) {
                // lane j < 2 nf owns list j = 2 f + kind: CTA total, one global atomic, per-warp offsets
                unsigned tot = 0;
                if (t < 2 * nf)
                    for (int w = 0; w < kHW; ++w) tot += wcnt[t * kHW + w];
                const unsigned at =
                    (t < 2 * nf && tot) ? atomicAdd(&p.ctl[(t / 2) * kHCtl + ((t & 1) ? cInBin : cDirect)], tot) : 0u;
                unsigned incl = tot;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned v = __shfl_up_sync(kFull, incl, o);
                    if (t >= o) incl += v;
                }
                if (t < 2 * nf) {
                    gbase[t] = at;
                    ibase[t] = qfill + incl - tot;
                    unsigned run = 0;
                    for (int w = 0; w < kHW; ++w) {
                        const unsigned c = wcnt[t * kHW + w];
                        wcnt[t * kHW + w] = run;
                        run += c;
                    }
                }
                if (t == 31) ibase[16] = incl;  // items this round (lanes >= 2 nf add 0)
            }
            __syncthreads();
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int64_t row = base + t + i * kHT;
#pragma unroll
                for (int f = 0; f < 8; ++f) {
                    if (f >= nf) break;
                    {
                        if (code[i][f] == 0xffffu) continue;
                        const int kind = (int)(code[i][f] >> 15);
                        const unsigned rk = code[i][f] & 0x7fffu;
                        const int j = 2 * f + kind;
                        const unsigned local = wcnt[j * kHW + warp] + rk;
                        const unsigned slot = gbase[j] + local;
                        const unsigned cap = kind ? (unsigned)kHBinCap : (unsigned)kHMaxShort;
                        const bool kept = slot < cap;  // else a boundary overflow: the frame is refined in phase C
                        if (kept && kind)
                            p.bins[(size_t)f * kHBinCap + slot] = ((u64)__float_as_uint(dv[i][f]) << 32) | (u64)row;
                        const unsigned qi = ibase[j] + local;
                        if (qi < kQCap) {
                            q_row[qi] = kept ? (int)row : -1;
                            q_meta[qi] = (slot << 4) | ((unsigned)f << 1) | (unsigned)kind;
                        } else if (kept) {
                            rescore_alone(p.X, p.Q + (size_t)f * p.D, p.D, row,
                                          kind ? p.fkb + (size_t)f * kHBinCap + slot : p.fkd + (size_t)f * kHMaxShort + slot);
                        }
                    }
                }
            }
            // entries of this round that did not fit were handled in place
            qfill = min(qfill + ibase[16], kQCap);
            __syncthreads();
        }
        drain(qfill);
    }
    if (!grid_sync(p.bar, epoch, abort_sm, p.err)) return;

    // ------------------------------------------------ C: per frame, exact S-cut and top k
    if ((int)blockIdx.x < nf) {
        const int f = blockIdx.x;
        if (__ldcg(&p.ctl[f * kHCtl + cRefine]) != 0u) {
            refine_frame<CPL>(p, f, region, res, tmp);
        } else {
            const unsigned cd = min(__ldcg(&p.ctl[f * kHCtl + cDirect]), (unsigned)kHMaxShort);
            const unsigned nb = min(__ldcg(&p.ctl[f * kHCtl + cInBin]), (unsigned)kHBinCap);
            const unsigned need = take_all ? 0u : min(__ldcg(&p.ctl[f * kHCtl + cNeed]), nb);
            u64* sk = reinterpret_cast<u64*>(region);                   // kHBinCap coarse keys
            u64* fk = sk + kHBinCap;                                    // kHMaxShort full keys
            unsigned* hs = reinterpret_cast<unsigned*>(fk + kHMaxShort); // kBins
            u64* outk = reinterpret_cast<u64*>(hs + kBins);             // 32
            u64* skf = outk + 32;                                       // kHBinCap full keys of sk's rows
            for (unsigned i = t; i < nb; i += kHT) {
                sk[i] = __ldcg(p.bins + (size_t)f * kHBinCap + i);
                skf[i] = __ldcg(p.fkb + (size_t)f * kHBinCap + i);
            }
            for (unsigned i = t; i < cd; i += kHT) fk[i] = __ldcg(p.fkd + (size_t)f * kHMaxShort + i);
            __syncthreads();
            unsigned total = cd;
            if (need > 0) {
                // last boundary key inside the shortlist; exactly `need` keys are <= it
                const u64 cstar = block_kth_key<kHT>(sk, nb, need, *reinterpret_cast<const u64*>(&fr[f * 8 + 0]),
                                                     *reinterpret_cast<const u64*>(&fr[f * 8 + 2]), hs, res, tmp);
                if (t == 0) res[3] = cd;
                __syncthreads();
                for (unsigned i = t; i < nb; i += kHT)
                    if (sk[i] <= cstar) {
                        const unsigned pos = atomicAdd(&res[3], 1u);
                        if (pos < (unsigned)kHMaxShort) fk[pos] = skf[i];
                    }
                __syncthreads();
                total = min(res[3], (unsigned)kHMaxShort);
                __syncthreads();
            }
            select_topk(p, f, fk, total, hs, outk, res, tmp);
        }
        // the frame's histogram and counters are not read again: zeroed for the next launch
        for (int i = t; i < kBins; i += kHT) p.hist[(size_t)f * kBins + i] = 0u;
        if (t < kHCtl) p.ctl[f * kHCtl + t] = 0u;
        __threadfence();  // this frame's idx / dist before the count
        __syncthreads();
        if (t == 0) atomicAdd(&p.bar[2], 1u);  // frame f done
    }
    if (p.ap.a.nw == 0 || (int)blockIdx.x >= p.ap.a.nw) return;

    // ------------------------------------------------ D: Algorithm 2 per window
    if (t == 0) {
        volatile unsigned* done = p.bar + 2;
        const u64 t0 = globaltimer();
        while (*done < (unsigned)nf) {
            if (globaltimer() - t0 > kWaitLimitNs) {
                *abort_sm = 1;
                record_error(p.err, kErrTimeout);
                break;
            }
        }
        __threadfence();
    }
    __syncthreads();
    if (*abort_sm) return;
    if (warp == 0) {
        const AggArgs& a = p.ap.a;
        const int w = blockIdx.x;
        const long long b0 = (long long)woff[0] * a.per_frame, b1 = (long long)woff[1] * a.per_frame;
        const long long total = b1 - b0;
        if (total <= 0 || total > agg::kWarpCand || b0 < 0 || b1 > a.limit) {
            if (lane == 0) agg::write_invalid(a, w);
        } else if (total <= 128 && a.mode != 2) {
            u64* tab = reinterpret_cast<u64*>(region);                       // 256
            unsigned* tcnt = reinterpret_cast<unsigned*>(tab + 256);         // 256
            int* rows = reinterpret_cast<int*>(tcnt + 256);                  // 128
            agg::aggregate_warp_small(p.ap, w, b0, total, tab, tcnt, rows);
        } else {
            u64* keys = reinterpret_cast<u64*>(region);                      // kWarpCand
            int* rows = reinterpret_cast<int*>(keys + agg::kWarpCand);       // kWarpCand
            float* dd = reinterpret_cast<float*>(rows + agg::kWarpCand);     // kWarpCand
            int* cnt = reinterpret_cast<int*>(dd + agg::kWarpCand);          // kWarpCand + 1
            agg::aggregate_warp(p.ap, w, b0, total, keys, rows, dd, cnt);
        }
    }
}

// Every CTA leaves through here. The last one to leave re-zeroes the grid
// words (barrier arrivals, abort flag, frames done, departures); each frame's
// histogram and counters were re-zeroed by its CTA in phase C, and are zeroed
// here again after an abort (a CTA may have left before that step). So the
// control block is all zero when the next launch on it starts.
__device__ __forceinline__ void hier_leave(const HierParams& p, volatile int* abort_sm, volatile unsigned* flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        if (*abort_sm) atomicOr(&p.bar[1], 1u);
        __threadfence();
        const unsigned gone = atomicAdd(&p.bar[3], 1u) + 1u;
        unsigned f = 0u;
        if (gone == gridDim.x) {
            __threadfence();
            f = 1u | (atomicOr(&p.bar[1], 0u) ? 2u : 0u);
        }
        *flag = f;
    }
    __syncthreads();
    const unsigned f = *flag;
    if (!(f & 1u)) return;
    if (f & 2u) {
        for (int i = threadIdx.x; i < p.nf * kBins; i += kHT) p.hist[i] = 0u;
        for (int i = threadIdx.x; i < p.nf * kHCtl; i += kHT) p.ctl[i] = 0u;
    }
    if (threadIdx.x == 0) {
        p.bar[0] = 0u;
        p.bar[1] = 0u;
        p.bar[2] = 0u;
        p.bar[3] = 0u;
    }
}

template <int DC4, int CPL>
__global__ void __launch_bounds__(kHT, 1) hier_fused_kernel(const HierParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    // the tail words after fr, res and tmp: abort flag, window offsets (2), leave flag
    unsigned* tail = reinterpret_cast<unsigned*>(smem + kHRegion + 8 * DC4 * sizeof(float4)) + 8 * 8 + 4 + kHW;
    hier_phases<DC4, CPL>(p);
    hier_leave(p, reinterpret_cast<volatile int*>(tail), tail + 3);
}

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct HierLayout {
    size_t dcbuf, hist, ctl, bar, zero_end, bins, fkd, fkb, ctk, total;
};

HierLayout hlayout(const lhr_db* db, int nf) {
    HierLayout L{};
    L.dcbuf = 0;
    L.hist = a256((size_t)nf * db->n * sizeof(float));
    L.ctl = L.hist + (size_t)nf * kBins * sizeof(unsigned);
    L.bar = L.ctl + (size_t)nf * kHCtl * sizeof(unsigned);
    L.zero_end = L.bar + 4 * sizeof(unsigned);
    L.bins = a256(L.zero_end);
    L.fkd = a256(L.bins + (size_t)nf * kHBinCap * sizeof(u64));
    L.fkb = a256(L.fkd + (size_t)nf * kHMaxShort * sizeof(u64));
    L.ctk = a256(L.fkb + (size_t)nf * kHBinCap * sizeof(u64));
    L.total = a256(L.ctk + (size_t)nf * 32 * sizeof(u64));
    return L;
}

size_t hier_smem(int dc4) {
    // region, frames' prefixes, then fr (64 words), res (4), tmp (kHW), abort flag (1), window offsets (2)
    return kHRegion + (size_t)8 * dc4 * sizeof(float4) + (8 * 8 + 4 + kHW + 4) * sizeof(unsigned);
}

template <int DC4, int CPL>
cudaError_t launch_h(const HierParams& hp, int grid, cudaStream_t stream) {
    auto kern = hier_fused_kernel<DC4, CPL>;
    const size_t sm = hier_smem(DC4);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kHT);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    ProfScope ps("hier_fused_kernel", stream);
    return cudaLaunchKernelEx(&cfg, kern, hp);
}

}  // namespace

bool hier_fused_eligible(const lhr_db* db, int nq, int shortlist) {
    return nq >= 1 && nq <= 8 && db->Xc != nullptr && db->n_sub == 1 && shortlist <= kHMaxShort &&
           db->coarse_dim <= 128;
}

size_t hier_scratch_bytes(const lhr_db* db, int nq) { return hlayout(db, nq).total; }

// A control block: histograms (8 frames), counters (8 frames), grid words.
size_t hier_ws_block_bytes() { return a256((size_t)8 * kBins * 4 + (size_t)8 * kHCtl * 4 + 4 * 4); }

// The control block of `stream`: the one it holds, else a free one (taken for
// the handle's lifetime), else nullptr.
static unsigned char* hier_ws_block(const lhr_db* db, cudaStream_t stream) {
    if (db->hws == nullptr || db->hws_map == nullptr) return nullptr;
    HierWsMap& m = *db->hws_map;
    std::lock_guard<std::mutex> lk(m.mu);
    int slot = -1;
    for (int i = 0; i < kHierWsBlocks && slot < 0; ++i)
        if (m.used[i] && m.owner[i] == stream) slot = i;
    for (int i = 0; i < kHierWsBlocks && slot < 0; ++i)
        if (!m.used[i]) {
            m.used[i] = true;
            m.owner[i] = stream;
            slot = i;
        }
    return slot < 0 ? nullptr : db->hws + (size_t)slot * hier_ws_block_bytes();
}

cudaError_t launch_hier_fused(const lhr_db* db, const float* q, int nq, int shortlist, int k, int64_t* idx,
                              float* dist, const AggArgs* agg_args, void* scratch, cudaStream_t stream) {
    const HierLayout L = hlayout(db, nq);
    unsigned char* base = reinterpret_cast<unsigned char*>(scratch);
    // the words that must be zero at the start: the stream's control block
    // (left zeroed by the previous launch on it), else scratch and a memset
    unsigned char* zb = hier_ws_block(db, stream);
    unsigned *hist, *ctl, *bar;
    if (zb != nullptr) {
        hist = reinterpret_cast<unsigned*>(zb);
        ctl = hist + 8 * kBins;
        bar = ctl + 8 * kHCtl;
    } else {
        cudaError_t e = cudaMemsetAsync(base + L.hist, 0, L.zero_end - L.hist, stream);
        if (e != cudaSuccess) return e;
        hist = reinterpret_cast<unsigned*>(base + L.hist);
        ctl = reinterpret_cast<unsigned*>(base + L.ctl);
        bar = reinterpret_cast<unsigned*>(base + L.bar);
    }
    HierParams hp{};
    hp.Xc = db->Xc;
    hp.dc = db->coarse_dim;
    hp.X = db->X;
    hp.D = db->dim;
    hp.n = db->n;
    hp.Q = q;
    hp.nf = nq;
    hp.S = shortlist;
    hp.k = k;
    hp.dcbuf = reinterpret_cast<float*>(base + L.dcbuf);
    hp.hist = hist;
    hp.ctl = ctl;
    hp.bar = bar;
    hp.bins = reinterpret_cast<u64*>(base + L.bins);
    hp.fkd = reinterpret_cast<u64*>(base + L.fkd);
    hp.fkb = reinterpret_cast<u64*>(base + L.fkb);
    hp.ctk = agg_args ? reinterpret_cast<u64*>(base + L.ctk) : nullptr;  // tile keys only feed Algorithm 2
    hp.idx = idx;
    hp.dist = dist;
    hp.err = db->err;
    if (agg_args) {
        hp.ap.a = *agg_args;
        hp.ap.tile = db->tile;
        hp.ap.xy = db->xy;
        hp.ap.n = db->n;
        hp.ap.rlim = (long long)floor(sqrt((double)agg_args->r2max)) + 1;
        hp.ap.err = db->err;
        hp.ap.tile_keys = hp.ctk;  // written with the results, in the same slots as idx
    } else {
        hp.ap.a.nw = 0;
    }
    const int dc4 = db->coarse_dim / 4;
    const int d4 = db->dim / 4;
    const int cpl = d4 <= 32 ? 1 : (d4 <= 64 ? 2 : 4);
    const int grid = db->sms;
    if (dc4 <= 8) {
        if (cpl == 1) return launch_h<8, 1>(hp, grid, stream);
        if (cpl == 2) return launch_h<8, 2>(hp, grid, stream);
        return launch_h<8, 4>(hp, grid, stream);
    }
    if (dc4 <= 16) {
        if (cpl == 1) return launch_h<16, 1>(hp, grid, stream);
        if (cpl == 2) return launch_h<16, 2>(hp, grid, stream);
        return launch_h<16, 4>(hp, grid, stream);
    }
    if (cpl == 1) return launch_h<32, 1>(hp, grid, stream);
    if (cpl == 2) return launch_h<32, 2>(hp, grid, stream);
    return launch_h<32, 4>(hp, grid, stream);
}

}  // namespace lhr
