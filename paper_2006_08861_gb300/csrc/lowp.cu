// Low-precision form: tensor-core scores over a BF16 / FP8-e4m3 copy of the
// database with per-row scales, a per-query top-W shortlist by score, and an
// FP32 re-rank of the shortlist on the FP32 rows (the paper scores FP
// features directly, §3.1; this form trades a widened shortlist for
// tensor-core throughput when many query frames are batched).
//
// score(q, x_j) = fma(m s_j, q^ . x^_j, n_j)       (||q||^2 dropped: constant per query)
//   x^_j, s_j : database codes and per-row scale, n_j = s_j^2 ||x^_j||^2
//               (built with the database);
//   q^, s_Q   : query codes and the batch's shared power-of-two scale (the
//               smallest 2^e >= max |q| / QMAX), m = -2 s_Q, so m s_j is exact.
// Keys are (orderable score bits << 32 | row); the shortlist is the W
// smallest keys, exactly.
//
// Per batch of queries:
//   query_amax_kernel + quantize_queries_kernel  the batch's power-of-two scale and the codes
//   tc_main_kernel<kPilot = true>   pilot over every 64th database row (a copy built with the
//                                   database): per query, the 8 smallest 32-row bucket minima
//   tau_kernel                      tau_q = the 8th smallest of them (at least 8 sample rows score
//                                   at most tau_q; about 8 x 64 database rows in expectation)
//   sort_queries_kernel             queries in ascending tau order: sorted codes, the query at each
//                                   position, and per 32 positions the largest tau (group bound)
//   tc_main_kernel<kPilot = false>  main pass: every key <= tau_q into query q's candidate buffer
//   tc_kernel (full)                fallback: exact per-chunk top W of a 128-query block whose
//                                   candidate count fell outside [W, kCap]; exits at once otherwise
//   merge_rerank_kernel             the W smallest candidates, re-scored in FP32 (direct form), top k
//
// tc_main_kernel: warp-specialised, 18 warps, one CTA per (256-query block, database chunk), one
// CTA per SM:
//   warp 0  producer: TMA (cp.async.bulk.tensor.2d, 128-byte swizzle) of the block's 256 query
//           codes once, then the chunk's 128-row tiles, one 128-byte K slice per stage, through a
//           mbarrier ring as deep as shared memory allows.
//   warp 1  TMEM allocator and MMA issuer: tcgen05.mma M = 128 rows (A, the database tile) x
//           N = 256 queries (B, resident) x K = 32 FP8 / 16 BF16 into two 256-column FP32
//           accumulators (all of TMEM), in turn per tile; tcgen05.commit frees ring stages and
//           publishes accumulators.
//   warps 2-17 epilogue: four warps per TMEM lane quadrant, a thread = a database row and one
//           64-column quarter of the queries, read as two 32-column groups. A group's smallest
//           score for the row is fma(m s_j, max dot, n_j) (m s_j <= 0; fma is monotone), compared
//           with the group's bound. Rows that pass go through the warp's shared-memory transpose
//           buffer so that lane l checks column l -- the query it owns -- exactly, and stages a
//           qualifying key; a full stage goes to the query's candidate buffer with one atomic.
//           In pilot mode the epilogue instead takes, per group and 32-row bucket, the column
//           minima (a butterfly over the warp) and keeps each query's 8 smallest.
// tc_kernel (fallback pass): 10 warps, one CTA per (128-query block, database chunk); the query
//   block is the A operand, a thread is a query and reads each column's (s_j, n_j) from shared
//   memory (a 1-D bulk copy per tile) and keeps its query's exact top W of the chunk in local
//   memory, filled through a 16-entry shared-memory survivor buffer. It is the only pass for
//   databases too small to sample.
// merge_rerank_kernel, one block of four warps per query: the shortlist is the
//   W smallest keys of the query's candidate buffer (for W <= 64 each warp keeps
//   a running 64 smallest in registers over its share of the 64-key chunks and
//   warp 0 merges the four; else, and after the full pass, warp 0 sorts the
//   candidates or the per-chunk lists cut at the smallest chunk's W-th key);
//   the four warps re-score its rows with the exact FP32 direct form (eight
//   rows in flight each) and the sorted exact keys give the top k.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "tc.cuh"

namespace lhr {
namespace {

constexpr int kTile = 128;        // queries per CTA (UMMA M) and rows per tile (UMMA N)
constexpr int kSliceBytes = 128;  // K bytes per smem row (one 128-byte swizzle atom)
constexpr int kSliceTile = kTile * kSliceBytes;  // 16 KB per tile slice
constexpr int kMaxStages = 8;     // operand ring depth: as many 16 KB slices as shared memory leaves room for
constexpr int kAcc = 4;           // FP32 accumulators in TMEM (4 x 128 columns = all 512)
constexpr int kSnSlots = 8;       // (s_j, n_j) tiles in flight: deeper than the operand ring, so never its limit
constexpr int kBuf = 16;          // survivor buffer entries per epilogue thread
constexpr int kHalves = 2;        // epilogue warps per TMEM lane quadrant (each takes a column range)
constexpr int kEpiWarps = 4 * kHalves;
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kThreads = 64 + kEpiThreads;  // producer, MMA issuer, epilogue
constexpr int kQTile = 256;       // queries per CTA of the main pass (UMMA N)
constexpr int kMainAcc = 2;       // main pass: 2 x 256 FP32 accumulator columns = all of TMEM

// ------------------------------------------------------------------ PTX (tc.cuh)
using namespace tc;

template <bool kFp8>
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, u64 adesc, u64 bdesc, uint32_t idesc, uint32_t accum) {
    tc::tc_mma<kFp8 ? kTcFP8 : kTcBF16>(d_tmem, adesc, bdesc, idesc, accum);
}
__host__ __device__ constexpr uint32_t tc_idesc(bool fp8, int n = kTile) { return tc::tc_idesc(fp8 ? kTcFP8 : kTcBF16, n); }

// Orderable key of a (possibly negative) FP32 score and a row.
__device__ __forceinline__ u64 score_key(float t, uint32_t row) {
    uint32_t u = __float_as_uint(t);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ((u64)u << 32) | row;
}


enum { kModeFull = 2 };
constexpr int kPilotR = 8;        // sample keys kept per query by the pilot pass
constexpr int kCap = 2048;        // candidate keys kept per query by the main pass
constexpr int kMergeWarps = 4;

struct TcParams {
    int64_t n;
    int slices;          // D * elem / 128
    int stages;          // operand ring depth, <= kMaxStages
    int chunk_rows;      // multiple of kTile
    int nchunks;
    const float2* sn;    // per row (s_j, n_j), padded
    const float* qs;     // [0] = s_Q, [1] = m = -2 s_Q
    int nq;
    int W;
    u64* partial;        // full: [query][chunk][W]; pilot: [query][chunk][kPilotR]
    const unsigned* cnt; // full: keys the main pass saw per query; nullptr = always run
    int* err;
};

struct MainParams {
    int64_t n;
    int slices, stages, chunk_rows, nchunks;
    const float2* sn;     // per row (s_j, n_j), kSnPad rows of zero padding
    const float* qs;      // [0] = s_Q, [1] = m = -2 s_Q
    const float* tau_s;   // per padded query: threshold score (-inf for padding queries)
    const u64* tau_key;   // per padded query: threshold key
    const int* perm;      // per sorted position: the query there (caller's order), -1 = padding
    const float* tgrp;    // per 32 sorted positions: the largest threshold among them (-inf if none)
    u64* cand;            // [query][kCap]
    unsigned* cnt;        // keys <= tau seen per query
    int nq;
    int cs;               // CTAs per cluster along the query blocks (1, 2 or 4): they share each database tile
    u64* pilot_out;       // pilot mode: [query][lists][kPilotR] keys of 32-row bucket minima
    int pilot_lists;      // pilot mode: lists per query (chunks x 4 lane quadrants)
    int* err;
};

__device__ __forceinline__ float key_score(u64 key) {
    const uint32_t u = (uint32_t)(key >> 32);
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// Sorted register network of kPilotR keys (static indices only).
__device__ __forceinline__ void net_insert(u64 (&net)[kPilotR], u64 key) {
    if (key >= net[kPilotR - 1]) return;
#pragma unroll
    for (int i = kPilotR - 1; i > 0; --i) {
        const u64 prev = net[i - 1];
        net[i] = key < prev ? prev : (key < net[i] ? key : net[i]);
    }
    net[0] = key < net[0] ? key : net[0];
}

template <int WMAX>
__device__ __noinline__ void flush_buffer(u64* list, const u64* buf, int stride, int nb, int W) {
    u64 tmp[kBuf];
    for (int i = 0; i < nb; ++i) {
        const u64 v = buf[i * stride];
        int j = i;
        while (j > 0 && tmp[j - 1] > v) {
            tmp[j] = tmp[j - 1];
            --j;
        }
        tmp[j] = v;
    }
    u64 out[WMAX];
    int a = 0, b = 0;
    for (int o = 0; o < W; ++o) {
        const u64 x = list[a];
        const u64 y = b < nb ? tmp[b] : kKeyEmpty;
        if (y < x) {
            out[o] = y;
            ++b;
        } else {
            out[o] = x;
            ++a;
        }
    }
    for (int o = 0; o < W; ++o) list[o] = out[o];
}

template <bool kFp8, int MODE, int WMAX>
__global__ void __launch_bounds__(kThreads, 1)
    tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const TcParams p) {
    extern __shared__ unsigned char smem_raw[];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int chunk = blockIdx.x, qblock = blockIdx.y;
    if (p.cnt != nullptr) {
        // fallback after a main pass: run only if a query of this block needs it
        bool need = false;
        if (threadIdx.x < kTile) {
            const int64_t qi = (int64_t)qblock * kTile + threadIdx.x;
            if (qi < p.nq) {
                const unsigned c = p.cnt[qi];
                need = c < (unsigned)p.W || c > (unsigned)kCap;
            }
        }
        if (!__syncthreads_or(need)) return;
    }
    // 1024-byte alignment for the 128-byte swizzle pattern
    unsigned char* smem =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char* sA = smem;                                   // slices x 16 KB
    unsigned char* sB = sA + (size_t)p.slices * kSliceTile;     // p.stages x 16 KB
    const int stages = p.stages;
    float2* sSN = reinterpret_cast<float2*>(sB + (size_t)stages * kSliceTile);  // kSnSlots x 128
    u64* sBuf = reinterpret_cast<u64*>(sSN + kSnSlots * kTile);  // full: kBuf x kEpiThreads (slot-major)
    u64* bars = sBuf + kBuf * kEpiThreads;
    u64* full = bars;
    u64* empty = full + kMaxStages;
    u64* a_full = empty + kMaxStages;
    u64* acc_full = a_full + 1;
    u64* acc_empty = acc_full + kAcc;
    u64* sn_full = acc_empty + kAcc;
    u64* sn_empty = sn_full + kSnSlots;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(sn_empty + kSnSlots);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

    const int64_t row0 = (int64_t)chunk * p.chunk_rows;
    const int64_t row1 = min(p.n, row0 + p.chunk_rows);
    const int ntiles = row1 > row0 ? (int)((row1 - row0 + kTile - 1) / kTile) : 0;
    constexpr int kElemPerSlice = kFp8 ? 128 : 64;
    constexpr int kMmaK = kFp8 ? 32 : 16;                       // elements per MMA
    constexpr int kMmaPerSlice = kElemPerSlice / kMmaK;         // 4
    constexpr uint32_t kIdesc = tc_idesc(kFp8);

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(a_full, 1);
        for (int i = 0; i < kAcc; ++i) {
            mbar_init(&acc_full[i], 1);
            mbar_init(&acc_empty[i], kEpiWarps);
        }
        for (int i = 0; i < kSnSlots; ++i) {
            mbar_init(&sn_full[i], 1);
            mbar_init(&sn_empty[i], kEpiWarps);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(kAcc * kTile)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    if (warp == 0) {
        if (lane == 0) {
            // queries of this block, all K slices, once
            mbar_arrive_expect_tx(a_full, (uint32_t)p.slices * kSliceTile);
            for (int s = 0; s < p.slices; ++s)
                tma_load_2d(sA + (size_t)s * kSliceTile, &tmA, s * kElemPerSlice, qblock * kTile, a_full);
            int sn_issued = 0, b_issued = 0;
            int st = 0;
            uint32_t ph = 0;  // ring slot and its wrap parity
            for (int t = 0; t < ntiles && !*abort_flag; ++t) {
                const int64_t r = row0 + (int64_t)t * kTile;
                const int slot = t % kSnSlots;
                if (!mbar_wait(&sn_empty[slot], (uint32_t)((t / kSnSlots) & 1) ^ 1u, abort_flag)) {
                    *abort_flag = 1;
                    record_error(p.err, kErrTimeout);
                    break;
                }
                const int nr = (int)((row1 - r) < kTile ? (row1 - r) : kTile);
                const uint32_t snb = (uint32_t)((nr + 1) / 2) * 16u;
                mbar_arrive_expect_tx(&sn_full[slot], snb);
                bulk_g2s(sSN + slot * kTile, p.sn + r, snb, &sn_full[slot]);
                ++sn_issued;
                for (int s = 0; s < p.slices; ++s) {
                    if (!mbar_wait(&empty[st], ph ^ 1u, abort_flag)) {
                        *abort_flag = 1;
                        record_error(p.err, kErrTimeout);
                        break;
                    }
                    mbar_arrive_expect_tx(&full[st], kSliceTile);
                    tma_load_2d(sB + (size_t)st * kSliceTile, &tmB, s * kElemPerSlice, (int)r, &full[st]);
                    ++b_issued;
                    if (++st == stages) {
                        st = 0;
                        ph ^= 1u;
                    }
                }
            }
            if (*abort_flag) {
                // let this thread's copies still in flight land before the CTA exits (bounded waits)
                mbar_wait(a_full, 0u, nullptr);
                for (int t = sn_issued > kSnSlots ? sn_issued - kSnSlots : 0; t < sn_issued; ++t)
                    mbar_wait(&sn_full[t % kSnSlots], (uint32_t)((t / kSnSlots) & 1), nullptr);
                for (int it = b_issued > stages ? b_issued - stages : 0; it < b_issued; ++it)
                    mbar_wait(&full[it % stages], (uint32_t)((it / stages) & 1), nullptr);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            bool ok = mbar_wait(a_full, 0u, abort_flag);
            int st = 0;
            uint32_t ph = 0;
            for (int t = 0; ok && t < ntiles; ++t) {
                const int a = t % kAcc;
                if (!mbar_wait(&acc_empty[a], (uint32_t)((t / kAcc) & 1) ^ 1u, abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(a * kTile);
                for (int s = 0; s < p.slices; ++s) {
                    if (!mbar_wait(&full[st], ph, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a_base = smem_u32(sA + (size_t)s * kSliceTile);
                    const uint32_t b_base = smem_u32(sB + (size_t)st * kSliceTile);
#pragma unroll
                    for (int kk = 0; kk < kMmaPerSlice; ++kk) {
                        const uint32_t off = (uint32_t)(kk * kMmaK * (kFp8 ? 1 : 2));
                        tc_mma<kFp8>(d_tmem, sw128_desc(a_base + off), sw128_desc(b_base + off), kIdesc,
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
        // ------------------------------------------------ epilogue
        const int quad = warp & 3;                 // TMEM lane quadrant this warp may access
        const int qrow = quad * 32 + lane;         // query row within the block
        const int ew = warp - 2;                   // epilogue warp 0 .. kEpiWarps-1
        const int half = ew / 4;                   // column half of every tile this warp scores
        const int lchunk = chunk * kHalves + half; // this thread's list slot among the chunk lists
        const int64_t qi = (int64_t)qblock * kTile + qrow;
        const bool qvalid = qi < p.nq;
        const float m = qvalid ? __ldg(p.qs + 1) : 0.f;
        // exact top W of the chunk
        u64 list[WMAX];
        for (int i = 0; i < WMAX; ++i) list[i] = kKeyEmpty;
        u64 thr = kKeyEmpty;
        int nb = 0;
        u64* buf = sBuf + ew * 32 + lane;
        for (int t = 0; t < ntiles; ++t) {
            const int a = t % kAcc;
            const uint32_t par = (uint32_t)((t / kAcc) & 1);
            const int sl = t % kSnSlots;
            if (!mbar_wait(&acc_full[a], par, abort_flag) ||
                !mbar_wait(&sn_full[sl], (uint32_t)((t / kSnSlots) & 1), abort_flag)) {
                if (lane == 0) {
                    *abort_flag = 1;
                    record_error(p.err, kErrTimeout);
                }
                break;
            }
            tc_fence_after();
            const int64_t r = row0 + (int64_t)t * kTile;
            const int nr = (int)((row1 - r) < kTile ? (row1 - r) : kTile);
            const float2* snt = sSN + sl * kTile;
            // 32 columns at a time; the second load is in flight while the first is scored
            auto score32 = [&](const uint32_t(&v)[32], const int c0) {
                if (qvalid) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int col = c0 + j;
                        const float2 sn = snt[col];
                        const float score = fmaf(m * sn.x, __uint_as_float(v[j]), sn.y);
                        const u64 key = score_key(score, (uint32_t)(r + col));
                        if (col < nr && key < thr) {
                            buf[nb * kEpiThreads] = key;
                            if (++nb == kBuf) {
                                flush_buffer<WMAX>(list, buf, kEpiThreads, nb, p.W);
                                nb = 0;
                                thr = list[p.W - 1];
                            }
                        }
                    }
                }
            };
            static_assert(kTile / kHalves == 64, "two 32-column loads per warp and tile");
            const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(a * kTile);
            const int cb = half * (kTile / kHalves);
            uint32_t va[32], vb[32];
            tmem_ld32_issue(tbase + (uint32_t)cb, va);
            tmem_ld32_issue(tbase + (uint32_t)(cb + 32), vb);
            tmem_ld_wait(va);  // waits for both loads; the second wait only names vb's registers
            tmem_ld_wait(vb);
            // the accumulator is in registers: hand it back to the MMA issuer before scoring
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[a]);
            score32(va, cb);
            score32(vb, cb + 32);
            __syncwarp();
            if (lane == 0) mbar_arrive(&sn_empty[sl]);
        }
        if (nb) flush_buffer<WMAX>(list, buf, kEpiThreads, nb, p.W);
        if (qvalid) {
            u64* dst = p.partial + ((size_t)qi * p.nchunks * kHalves + lchunk) * p.W;
            for (int i = 0; i < p.W; ++i) dst[i] = list[i];
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kAcc * kTile) : "memory");
}

// Main pass layout: 2 + kMainEpiWarps warps. Epilogue warp w reads TMEM lane
// quadrant w % 4 (its 32 database rows) and column quarter (w - 2) / 4 of each
// 256-query tile: kMGroups 32-query groups.
constexpr int kMainEpiWarps = 16;
constexpr int kMainEpiThreads = 32 * kMainEpiWarps;
constexpr int kMainThreads = 64 + kMainEpiThreads;
constexpr int kMGroups = kQTile / (kMainEpiWarps / 4) / 32;  // 2
constexpr int kOwnSlots = 4;       // staged keys per owned query
constexpr int kTRows = 8;          // rows a warp moves through its transpose buffer at a time
constexpr int kTStride = 36;       // floats per buffered row: 32 values, then (A, B, row, -); 144 B apart

// Staged keys of one owned query (slot i at slot[i * kMainEpiThreads]) to its
// candidate buffer: one atomic for the lot.
__device__ __forceinline__ void flush_owned(const MainParams& p, const u64* slot, int q, int n) {
    const unsigned pos = atomicAdd(p.cnt + q, (unsigned)n);
    for (int i = 0; i < n; ++i)
        if (pos + i < (unsigned)kCap) p.cand[(size_t)q * kCap + pos + i] = slot[i * kMainEpiThreads];
}

// Rows of one 32-column group that passed the group bound (the warp's ballot
// `ev`; see the epilogue) go, up to kTRows at a time, through the warp's
// shared-memory transpose buffer: lane l then reads column l of each such row
// -- the query it owns -- and checks it exactly: score < tau_s decides without
// the key; on an exact score tie the row index decides against the threshold
// key. A qualifying key is staged in the lane's slots for that query; a full
// stage goes to the query's candidate buffer with one atomic.
// Lanes of `sel` (at most kTRows) write their rows' 32 values and (A, B, row) to
// the warp's transpose buffer, row `rank` = the lane's rank within `sel`.
__device__ __forceinline__ void stage_rows(const uint32_t (&v)[32], float A, float B, uint32_t row, unsigned sel,
                                           int lane, float* tbuf) {
    if ((sel >> lane) & 1u) {
        float4* dst = reinterpret_cast<float4*>(tbuf + __popc(sel & ((1u << lane) - 1u)) * kTStride);
#pragma unroll
        for (int j = 0; j < 8; ++j)
            dst[j] = make_float4(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]), __uint_as_float(v[4 * j + 2]),
                                 __uint_as_float(v[4 * j + 3]));
        dst[8] = make_float4(A, B, __uint_as_float(row), 0.f);
    }
}

// Lane l checks column l -- the query it owns -- of the nsel buffered rows.
__device__ __forceinline__ void check_rows(const MainParams& p, const float* tbuf, int nsel, int lane, u64* slot,
                                           const int* own_q, const float* own_tau, int& n_own) {
    const float tau_own = *own_tau;
    for (int r = 0; r < nsel; ++r) {
        const float x = tbuf[r * kTStride + lane];
        const float4 mt = *reinterpret_cast<const float4*>(tbuf + r * kTStride + 32);
        const float score = fmaf(mt.y, x, mt.x);
        if (score <= tau_own) {
            const int q_own = *own_q;
            const u64 key = score_key(score, __float_as_uint(mt.z));
            if (score < tau_own || key <= __ldg(p.tau_key + q_own)) {
                slot[n_own * kMainEpiThreads] = key;
                if (++n_own == kOwnSlots) {
                    flush_owned(p, slot, q_own, n_own);
                    n_own = 0;
                }
            }
        }
    }
}

// All rows of `ev`, kTRows at a time.
__device__ __forceinline__ void main_survivors(const MainParams& p, const uint32_t (&v)[32], float A, float B,
                                               unsigned ev, uint32_t row, int lane, float* tbuf, u64* slot,
                                               const int* own_q, const float* own_tau, int& n_own) {
    const unsigned lt = (1u << lane) - 1u;
    while (ev) {
        const unsigned sel = __ballot_sync(kFull, ((ev >> lane) & 1u) && __popc(ev & lt) < kTRows);
        stage_rows(v, A, B, row, sel, lane, tbuf);
        __syncwarp();
        check_rows(p, tbuf, __popc(sel), lane, slot, own_q, own_tau, n_own);
        __syncwarp();
        ev &= ~sel;
    }
}

// Main pass: every key <= tau_q of the chunk into query q's candidate buffer.
// The query block is kQTile = 256 queries in ascending-threshold order (the MMA's
// B operand, resident in shared memory); the database tile is the A operand,
// so a TMEM lane -- an epilogue thread -- is a database row and a column is a
// query. Two 256-column FP32 accumulators fill TMEM; the tensor core works on
// one tile while the epilogue reads the other.
// Sorted register network of kPilotR scores (static indices only).
__device__ __forceinline__ void fnet_insert(float (&net)[kPilotR], float x) {
    if (!(x < net[kPilotR - 1])) return;
#pragma unroll
    for (int i = kPilotR - 1; i > 0; --i) {
        const float prev = net[i - 1];
        net[i] = x < prev ? prev : (x < net[i] ? x : net[i]);
    }
    net[0] = fminf(x, net[0]);
}

// kPilot = false: the main pass (below). kPilot = true: the pilot over the
// database sample with the same pipeline: per 32-row bucket (a warp's rows of a
// tile) and query, the smallest score (column_min32), each query keeping its
// kPilotR smallest bucket minima per (chunk, lane quadrant). Every bucket
// minimum is a distinct row, so at least kPilotR sample rows score at most the
// kPilotR-th smallest of them (the threshold tau_kernel takes).
template <bool kFp8, bool kPilot>
__global__ void __launch_bounds__(kMainThreads, 1)
    tc_main_kernel(const __grid_constant__ CUtensorMap tmQ, const __grid_constant__ CUtensorMap tmX, const MainParams p) {
    extern __shared__ unsigned char smem_raw[];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int chunk = blockIdx.x, qblock = blockIdx.y;
    unsigned char* smem =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int stages = p.stages;
    constexpr int kQSlice = kQTile * kSliceBytes;               // 32 KB: one K slice of the query block
    unsigned char* sQ = smem;                                   // slices x 32 KB: the block's query codes
    unsigned char* sX = sQ + (size_t)p.slices * kQSlice;        // stages x 16 KB: database slices
    u64* own_slot = reinterpret_cast<u64*>(sX + (size_t)stages * kSliceTile);  // kMGroups kOwnSlots x threads
    float* tbuf_all = reinterpret_cast<float*>(own_slot + kMGroups * kOwnSlots * kMainEpiThreads);
    int* own_q_all = reinterpret_cast<int*>(tbuf_all + kMainEpiWarps * kTRows * kTStride);
    float* own_tau_all = reinterpret_cast<float*>(own_q_all + kMGroups * kMainEpiThreads);  // kMGroups x threads
    u64* full = reinterpret_cast<u64*>(own_tau_all + kMGroups * kMainEpiThreads);  // after the buffers below
    u64* empty = full + kMaxStages;
    u64* q_full = empty + kMaxStages;
    u64* acc_full = q_full + 1;
    u64* acc_empty = acc_full + kMainAcc;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(acc_empty + kMainAcc);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

    const int64_t row0 = (int64_t)chunk * p.chunk_rows;
    const int64_t row1 = min(p.n, row0 + p.chunk_rows);
    const int ntiles = row1 > row0 ? (int)((row1 - row0 + kTile - 1) / kTile) : 0;
    constexpr int kElemPerSlice = kFp8 ? 128 : 64;
    constexpr int kMmaK = kFp8 ? 32 : 16;
    constexpr int kMmaPerSlice = kElemPerSlice / kMmaK;
    constexpr uint32_t kIdesc = tc_idesc(kFp8, kQTile);

    // The cs CTAs of a cluster work on the same chunk for cs query blocks: each loads 1/cs of every
    // database slice and multicasts it to all of them, so a slot is free again once every CTA's
    // tensor core has read it (empty: one multicast commit from each CTA).
    const int cs = p.cs;
    const uint16_t cmask = (uint16_t)((1u << cs) - 1u);
    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], (uint32_t)cs);
        }
        mbar_init(q_full, 1);
        for (int i = 0; i < kMainAcc; ++i) {
            mbar_init(&acc_full[i], 1);
            mbar_init(&acc_empty[i], kMainEpiWarps);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(kMainAcc * kQTile)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    if (cs > 1) cluster_sync();  // every CTA's barriers exist before any multicast reaches them
    else __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    if (warp == 0) {
        if (lane == 0) {
            // the query block: per K slice two 128-row boxes, rows 0-127 and 128-255 of the slice
            mbar_arrive_expect_tx(q_full, (uint32_t)p.slices * kQSlice);
            for (int s = 0; s < p.slices; ++s)
                for (int hq = 0; hq < kQTile / kTile; ++hq)
                    tma_load_2d(sQ + (size_t)s * kQSlice + (size_t)hq * kSliceTile, &tmQ, s * kElemPerSlice,
                                qblock * kQTile + hq * kTile, q_full);
            const int rank = cs > 1 ? (int)cluster_ctarank() : 0;
            const int piece_rows = kTile / cs;
            const uint32_t piece_off = (uint32_t)(rank * piece_rows * kSliceBytes);
            int b_issued = 0, st = 0;
            uint32_t ph = 0;
            for (int t = 0; t < ntiles && !*abort_flag; ++t) {
                const int r = (int)(row0 + (int64_t)t * kTile);
                for (int s = 0; s < p.slices; ++s) {
                    if (!mbar_wait(&empty[st], ph ^ 1u, abort_flag)) {
                        *abort_flag = 1;
                        record_error(p.err, kErrTimeout);
                        break;
                    }
                    mbar_arrive_expect_tx(&full[st], kSliceTile);
                    if (cs > 1)
                        tma_load_2d_mc(sX + (size_t)st * kSliceTile + piece_off, &tmX, s * kElemPerSlice,
                                       r + rank * piece_rows, &full[st], cmask);
                    else
                        tma_load_2d(sX + (size_t)st * kSliceTile, &tmX, s * kElemPerSlice, r, &full[st]);
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
            if (cs > 1) {
                // every CTA's release of the last slots has reached this CTA's barriers (bounded waits)
                for (int it = b_issued > stages ? b_issued - stages : 0; it < b_issued; ++it)
                    mbar_wait(&empty[it % stages], (uint32_t)((it / stages) & 1), nullptr);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            bool ok = mbar_wait(q_full, 0u, abort_flag);
            int st = 0;
            uint32_t ph = 0;
            for (int t = 0; ok && t < ntiles; ++t) {
                const int a = t % kMainAcc;
                if (!mbar_wait(&acc_empty[a], (uint32_t)((t / kMainAcc) & 1) ^ 1u, abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(a * kQTile);
                for (int s = 0; s < p.slices; ++s) {
                    if (!mbar_wait(&full[st], ph, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t x_base = smem_u32(sX + (size_t)st * kSliceTile);
                    const uint32_t q_base = smem_u32(sQ + (size_t)s * kQSlice);
#pragma unroll
                    for (int kk = 0; kk < kMmaPerSlice; ++kk) {
                        const uint32_t off = (uint32_t)(kk * kMmaK * (kFp8 ? 1 : 2));
                        tc_mma<kFp8>(d_tmem, sw128_desc(x_base + off), sw128_desc(q_base + off), kIdesc,
                                     (s | kk) != 0 ? 1u : 0u);
                    }
                    if (cs > 1) tc_commit_mc(&empty[st], cmask);
                    else tc_commit(&empty[st]);
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
    } else if (kPilot) {
        // ------------------------------------------------ pilot epilogue: thread = sample row
        const int ew = warp - 2;
        const int quad = warp & 3;
        const int rl = quad * 32 + lane;
        const int cb = (ew / 4) * (32 * kMGroups);
        const int64_t q0 = (int64_t)qblock * kQTile + cb + lane;  // the queries this lane's columns end with
        const float kInfF = __int_as_float(0x7f800000);
        float net0[kPilotR], net1[kPilotR];
#pragma unroll
        for (int i = 0; i < kPilotR; ++i) net0[i] = net1[i] = kInfF;
        const float m = __ldg(p.qs + 1);
        const int rows_left = (int)(row1 - row0);
        const float2* snp = p.sn + row0 + rl;
        float2 sn_next = ntiles > 0 ? __ldg(snp) : make_float2(0.f, 0.f);
        for (int t = 0; t < ntiles; ++t) {
            const int a = t % kMainAcc;
            const float2 sn = sn_next;
            if (t + 1 < ntiles) sn_next = __ldg(snp + (t + 1) * kTile);
            if (!mbar_wait(&acc_full[a], (uint32_t)((t / kMainAcc) & 1), abort_flag)) {
                if (lane == 0) {
                    *abort_flag = 1;
                    record_error(p.err, kErrTimeout);
                }
                break;
            }
            tc_fence_after();
            const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(a * kQTile + cb);
            const float B = m * sn.x, A = sn.y;
            const bool rowvalid = t * kTile + rl < rows_left;
            uint32_t v[32];
            float c[32];
            tmem_ld32_issue(tbase, v);
            tmem_ld_wait(v);
#pragma unroll
            for (int j = 0; j < 32; ++j) c[j] = rowvalid ? fmaf(B, __uint_as_float(v[j]), A) : kInfF;
            fnet_insert(net0, column_min32(c, lane));
            tmem_ld32_issue(tbase + 32u, v);
            tmem_ld_wait(v);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[a]);
#pragma unroll
            for (int j = 0; j < 32; ++j) c[j] = rowvalid ? fmaf(B, __uint_as_float(v[j]), A) : kInfF;
            fnet_insert(net1, column_min32(c, lane));
        }
        // keys (score, row 0xffffffff): every key of that score is at most the threshold key
        const int list = chunk * 4 + quad;
#pragma unroll
        for (int g = 0; g < kMGroups; ++g) {
            const int64_t q = q0 + 32 * g;
            if (q < p.nq) {
                u64* dst = p.pilot_out + ((size_t)q * p.pilot_lists + list) * kPilotR;
#pragma unroll
                for (int i = 0; i < kPilotR; ++i) {
                    const float x = g == 0 ? net0[i] : net1[i];
                    dst[i] = x < kInfF ? score_key(x, 0xffffffffu) : kKeyEmpty;
                }
            }
        }
    } else {
        // ------------------------------------------------ epilogue: thread = database row
        const int ew = warp - 2;                        // epilogue warp 0 .. kMainEpiWarps - 1
        const int quad = warp & 3;                      // TMEM lane quadrant this warp may access
        const int rl = quad * 32 + lane;                // row within the tile
        const int cb = (ew / 4) * (32 * kMGroups);      // first column (query) of this warp's quarter
        const int64_t p0 = (int64_t)qblock * kQTile + cb;  // sorted position of that query
        float* tbuf = tbuf_all + ew * kTRows * kTStride;
        const int et = threadIdx.x - 64;                // epilogue thread 0 .. kMainEpiThreads - 1
        u64* slot0 = own_slot + et;
        u64* slot1 = slot0 + kOwnSlots * kMainEpiThreads;
        const float T0 = __ldg(p.tgrp + p0 / 32), T1 = __ldg(p.tgrp + p0 / 32 + 1);
        {
            // the queries this lane owns (column lane of each group) and their thresholds, read only
            // on the rare survivor path: kept in shared memory, not registers
            const float ninf = -__int_as_float(0x7f800000);
            for (int g = 0; g < kMGroups; ++g) {
                const int q = __ldg(p.perm + p0 + 32 * g + lane);
                own_q_all[g * kMainEpiThreads + et] = q;
                own_tau_all[g * kMainEpiThreads + et] = q >= 0 ? __ldg(p.tau_s + q) : ninf;
            }
        }
        int n0 = 0, n1 = 0;
        const float m = __ldg(p.qs + 1);
        const int rows_left = (int)(row1 - row0);       // rows of this chunk (< 2^31)
        const float2* snp = p.sn + row0 + rl;
        float2 sn_next = ntiles > 0 ? __ldg(snp) : make_float2(0.f, 0.f);
        for (int t = 0; t < ntiles; ++t) {
            const int a = t % kMainAcc;
            const float2 sn = sn_next;  // rows past the database read its zero padding
            if (t + 1 < ntiles) sn_next = __ldg(snp + (t + 1) * kTile);
            if (!mbar_wait(&acc_full[a], (uint32_t)((t / kMainAcc) & 1), abort_flag)) {
                if (lane == 0) {
                    *abort_flag = 1;
                    record_error(p.err, kErrTimeout);
                }
                break;
            }
            tc_fence_after();
            const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(a * kQTile + cb);
            const float B = m * sn.x, A = sn.y;
            const int rr = t * kTile + rl;                 // row within the chunk
            const bool rowvalid = rr < rows_left;
            const uint32_t row = (uint32_t)(row0 + rr);
            // per group: the row's smallest score over the group's queries is fma(B, max dot, A)
            // (B = m s_j <= 0, and a correctly rounded fma is monotone in each operand), tested
            // against the group's largest threshold.
            // one 32-column group in registers at a time: 18 warps leave 96 registers per thread.
            // Group 0's passing rows (at most kTRows; more is rare) wait in the transpose buffer, so
            // the accumulator goes back to the MMA issuer right after group 1 is in registers.
            uint32_t v[32];
            tmem_ld32_issue(tbase, v);
            tmem_ld_wait(v);
            const unsigned ev0 = __ballot_sync(kFull, rowvalid && fmaf(B, max32(v), A) <= T0);
            const int defer0 = __popc(ev0) <= kTRows ? __popc(ev0) : 0;
            if (defer0) stage_rows(v, A, B, row, ev0, lane, tbuf);
            else if (ev0) main_survivors(p, v, A, B, ev0, row, lane, tbuf, slot0, own_q_all + et, own_tau_all + et, n0);
            tmem_ld32_issue(tbase + 32u, v);
            tmem_ld_wait(v);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[a]);
            if (defer0) {
                check_rows(p, tbuf, defer0, lane, slot0, own_q_all + et, own_tau_all + et, n0);
                __syncwarp();
            }
            const unsigned ev1 = __ballot_sync(kFull, rowvalid && fmaf(B, max32(v), A) <= T1);
            if (ev1)
                main_survivors(p, v, A, B, ev1, row, lane, tbuf, slot1, own_q_all + kMainEpiThreads + et,
                               own_tau_all + kMainEpiThreads + et, n1);
        }
        if (n0) flush_owned(p, slot0, own_q_all[et], n0);
        if (n1) flush_owned(p, slot1, own_q_all[kMainEpiThreads + et], n1);
    }
    tc_fence_before();
    if (cs > 1) cluster_sync();  // no CTA leaves while another may still deliver to its shared memory
    else __syncthreads();
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kMainAcc * kQTile)
                     : "memory");
}

__device__ __forceinline__ u64 warp_min_u64(u64 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const u64 w = __shfl_xor_sync(kFull, v, o);
        v = w < v ? w : v;
    }
    return v;
}

// Per query (one warp): tau = the kPilotR-th smallest of its pilot keys (key
// and score); each lane keeps the kPilotR smallest of every 32nd list, then
// kPilotR rounds of a warp minimum pop the overall smallest. Padding queries
// get a score threshold of -inf, so nothing passes.
__global__ void tau_kernel(const u64* __restrict__ pilot, int lists, int nq, int nq_pad, u64* __restrict__ tau_key,
                           float* __restrict__ tau_s) {
    const int lane = threadIdx.x & 31;
    const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= nq_pad) return;
    if (q >= nq) {
        if (lane == 0) {
            tau_key[q] = 0;
            tau_s[q] = -__int_as_float(0x7f800000);
        }
        return;
    }
    u64 net[kPilotR];
#pragma unroll
    for (int i = 0; i < kPilotR; ++i) net[i] = kKeyEmpty;
    const u64* pl = pilot + (size_t)q * lists * kPilotR;
    // two of this lane's lists per pass: both lists' loads in flight together
    for (int c = lane; c < lists; c += 64) {
        u64 kk[2][kPilotR];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int ch = c + 32 * h;
#pragma unroll
            for (int i = 0; i < kPilotR; ++i) kk[h][i] = ch < lists ? __ldcg(pl + (size_t)ch * kPilotR + i) : kKeyEmpty;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int i = 0; i < kPilotR; ++i) net_insert(net, kk[h][i]);
    }
    u64 tau = kKeyEmpty;
    for (int r = 0; r < kPilotR; ++r) {
        const u64 head = net[0];
        tau = warp_min_u64(head);
        if (head == tau && tau != kKeyEmpty) {
            // the lane holding it (ties: keys are unique, (score, row)) pops its head
#pragma unroll
            for (int i = 0; i < kPilotR - 1; ++i) net[i] = net[i + 1];
            net[kPilotR - 1] = kKeyEmpty;
        }
    }
    if (lane == 0) {
        tau_key[q] = tau;
        tau_s[q] = tau == kKeyEmpty ? __int_as_float(0x7f800000) : key_score(tau);
    }
}

// Orders the batch's queries by threshold score for the main pass (CTA b
// writes sorted positions [256 b, 256 b + 256)): every CTA sorts all
// (threshold score, query) keys in shared memory with a bitonic network
// (batches of more than kSortMax queries keep their order), then writes, for
// its positions, the query there (perm, -1 = padding), its codes (a zero row
// for padding), and per 32 positions the largest threshold among their
// queries (tgrp). Adjacent thresholds make the main pass's per-group bound
// tight.
constexpr int kSortMax = 16384;
constexpr int kSortThreads = 512;
constexpr int kRegSort = 1024;  // up to this many keys: the bitonic network mostly in registers

__global__ void __launch_bounds__(kSortThreads) sort_queries_kernel(const float* __restrict__ tau_s, int nq,
                                                                    int n_sorted, const uint4* __restrict__ codes,
                                                                    int row_chunks, uint4* __restrict__ codes_s,
                                                                    int* __restrict__ perm, float* __restrict__ tgrp) {
    extern __shared__ u64 keys[];  // n2 >= n_sorted (a power of two), when sorting
    __shared__ int spos[kQTile];
    const int tid = threadIdx.x;
    const int base = blockIdx.x * kQTile;
    if (n_sorted <= kSortMax) {
        int n2 = 1;
        while (n2 < n_sorted) n2 <<= 1;
        for (int i = tid; i < n2; i += blockDim.x) {
            uint32_t u = 0xffffffffu;  // padding positions sort last, in index order
            if (i < nq) {
                u = __float_as_uint(tau_s[i]);
                u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
                u = min(u, 0xfffffffeu);
            }
            keys[i] = ((u64)u << 32) | (uint32_t)i;
        }
        __syncthreads();
        if (n2 <= kRegSort) {
            // 16 warps x 64 keys in registers (element 64 w + 32 e + lane in v[e]; ~0 past n2 sorts
            // last): strides below 32 by shuffles, 32 within the lane, 64 and up through shared memory
            static_assert(kSortThreads == 512 && kRegSort == 1024, "16 warps of 64 keys");
            const int warp = tid / 32, lane = tid % 32;
            u64 v[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int idx = 64 * warp + 32 * e + lane;
                v[e] = idx < n2 ? keys[idx] : ~0ull;
            }
            for (int size = 2; size <= kRegSort; size <<= 1) {
                for (int stride = size >> 1; stride > 0; stride >>= 1) {
                    if (stride >= 64) {
#pragma unroll
                        for (int e = 0; e < 2; ++e) keys[64 * warp + 32 * e + lane] = v[e];
                        __syncthreads();
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            const int idx = 64 * warp + 32 * e + lane;
                            const u64 o = keys[idx ^ stride];
                            const bool asc = (idx & size) == 0;
                            const bool keep_min = (idx < (idx ^ stride)) == asc;
                            v[e] = keep_min ? (o < v[e] ? o : v[e]) : (o > v[e] ? o : v[e]);
                        }
                        __syncthreads();
                    } else if (stride == 32) {
                        const bool asc = ((64 * warp + lane) & size) == 0;
                        const u64 lo = v[0] < v[1] ? v[0] : v[1], hi = v[0] < v[1] ? v[1] : v[0];
                        v[0] = asc ? lo : hi;
                        v[1] = asc ? hi : lo;
                    } else {
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            const int idx = 64 * warp + 32 * e + lane;
                            const u64 o = __shfl_xor_sync(kFull, v[e], stride);
                            const bool asc = (idx & size) == 0;
                            const bool keep_min = ((lane & stride) == 0) == asc;
                            v[e] = keep_min ? (o < v[e] ? o : v[e]) : (o > v[e] ? o : v[e]);
                        }
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int idx = 64 * warp + 32 * e + lane;
                if (idx < n2) keys[idx] = v[e];
            }
            __syncthreads();
        } else {
            for (int size = 2; size <= n2; size <<= 1) {
                for (int stride = size >> 1; stride > 0; stride >>= 1) {
                    for (int i = tid; i < n2 / 2; i += blockDim.x) {
                        const int lo = 2 * i - (i & (stride - 1));
                        const int hi = lo + stride;
                        const bool up = (lo & size) == 0;
                        const u64 x = keys[lo], y = keys[hi];
                        if ((x > y) == up) {
                            keys[lo] = y;
                            keys[hi] = x;
                        }
                    }
                    __syncthreads();
                }
            }
        }
        for (int i = tid; i < kQTile; i += blockDim.x) {
            const int q = (int)(uint32_t)keys[base + i];
            spos[i] = q < nq ? q : -1;
        }
    } else {
        for (int i = tid; i < kQTile; i += blockDim.x) spos[i] = base + i < nq ? base + i : -1;
    }
    __syncthreads();
    for (int i = tid; i < kQTile; i += blockDim.x) perm[base + i] = spos[i];
    const int warp = tid / 32, lane = tid % 32;
    for (int g = warp; g < kQTile / 32; g += blockDim.x / 32) {
        const int q = spos[g * 32 + lane];
        float t = q >= 0 ? tau_s[q] : -__int_as_float(0x7f800000);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t = fmaxf(t, __shfl_xor_sync(kFull, t, o));
        if (lane == 0) tgrp[(base >> 5) + g] = t;
    }
    for (int i = tid; i < kQTile * row_chunks; i += blockDim.x) {
        const int r = i / row_chunks, c = i % row_chunks;
        const int q = spos[r];
        codes_s[(size_t)(base + r) * row_chunks + c] = q >= 0 ? codes[(size_t)q * row_chunks + c] : make_uint4(0, 0, 0, 0);
    }
}

// max |q| over the batch into *amax_bits (the bits of a non-negative float
// order like unsigned integers; *amax_bits zeroed before the launch).
__global__ void __launch_bounds__(256) query_amax_kernel(const float* __restrict__ Q, int64_t count,
                                                          unsigned* __restrict__ amax_bits) {
    __shared__ float wmax[8];
    float amax = 0.f;
    // float4 loads when Q is 16-byte aligned (a caller's view may start anywhere), the rest one by one
    const int64_t count4 = (reinterpret_cast<uintptr_t>(Q) & 15u) == 0 ? count / 4 : 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count4; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(Q) + i);
        amax = fmaxf(amax, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
    for (int64_t i = count4 * 4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        amax = fmaxf(amax, fabsf(__ldg(Q + i)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(kFull, amax, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x / 32] = amax;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) m = fmaxf(m, wmax[w]);
        if (m > 0.f) atomicMax(amax_bits, __float_as_uint(m));  // one atomic per block
    }
}

// The batch's shared query scale from max |q|: s_Q = the smallest power of two
// >= max |q| / qmax (the divide in binary32; at least 2^-126; 1 for an
// all-zero batch).
__device__ __forceinline__ float query_scale(float amax, float qmax) {
    if (!(amax > 0.f)) return 1.0f;
    const float x = fmaxf(__fdiv_rn(amax, qmax), 1.17549435e-38f);  // 2^-126
    const uint32_t b = __float_as_uint(x);
    return (b & 0x7fffffu) == 0u ? x : __uint_as_float((b & 0x7f800000u) + 0x00800000u);
}

// Query codes q / s_Q (exact: s_Q is a power of two) rounded to the format;
// rows past nq (padding to the 128-query block) get zero codes. Also writes
// qs[0] = s_Q, qs[1] = m = -2 s_Q.
template <bool kFp8>
__global__ void quantize_queries_kernel(const float* Q, int nq, int nq_pad, int D, const unsigned* amax_bits,
                                        float qmax, float* qs, void* codes) {
    const int lane = threadIdx.x & 31;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= nq_pad) return;
    const float s = query_scale(__uint_as_float(*amax_bits), qmax);
    if (w == 0 && lane == 0) {
        qs[0] = s;
        qs[1] = -2.0f * s;
    }
    for (int j = lane; j < D; j += 32) {
        const float v = w < nq ? __fdiv_rn(Q[(size_t)w * D + j], s) : 0.f;
        if (kFp8)
            reinterpret_cast<__nv_fp8_storage_t*>(codes)[(size_t)w * D + j] =
                __nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
        else
            reinterpret_cast<__nv_bfloat16*>(codes)[(size_t)w * D + j] = __float2bfloat16_rn(v);
    }
}


// Warp bitonic sort of n (power of two) keys in shared memory, ascending.
__device__ void warp_sort(u64* a, int n, int lane) {
    for (int size = 2; size <= n; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = lane; i < n / 2; i += 32) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const bool up = (lo & size) == 0;
                const u64 x = a[lo], y = a[hi];
                if ((x > y) == up) {
                    a[lo] = y;
                    a[hi] = x;
                }
            }
            __syncwarp();
        }
    }
}

// Number of keys <= x among the query's per-chunk lists.
__device__ int count_le(const u64* P, int total, u64 x, int lane) {
    int c = 0;
    for (int i = lane; i < total; i += 32) {
        const u64 key = __ldcg(P + i);
        c += (key != kKeyEmpty && key <= x) ? 1 : 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
    return c;
}

template <int CPL>
__global__ void __launch_bounds__(kMergeWarps * 32) merge_rerank_kernel(
    const u64* __restrict__ partial, int nchunks, int W, const u64* __restrict__ cand,
    const unsigned* __restrict__ cnt, const float* __restrict__ X, int D, const float* __restrict__ Q, int nq, int k,
    int64_t* __restrict__ idx, float* __restrict__ dist) {
    extern __shared__ u64 merge_sm[];
    u64* cw = merge_sm;               // kCap: the shortlist
    u64* wl = merge_sm + kCap;        // kMergeWarps x 64: per-warp lists, then the exact keys
    __shared__ int s_n;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int qi = blockIdx.x;  // one query per block
    if (qi >= nq) return;
    const unsigned c = cand != nullptr ? cnt[qi] : 0u;
    if (cand != nullptr && c >= (unsigned)W && c <= (unsigned)kCap && W <= 64) {
        // the main pass collected every key <= tau, and there are W..kCap of them: each warp
        // keeps the 64 smallest of its share of the 64-key chunks (chunk w, w + kMergeWarps, ...;
        // the next chunk's loads in flight, chunks with nothing below its current 64th skipped),
        // then warp 0 merges the lists
        const int nc = (int)c;
        const u64* cq = cand + (size_t)qi * kCap;
        constexpr int kStep = 64 * kMergeWarps;
        u64 best[2] = {kKeyEmpty, kKeyEmpty}, nxt[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int i = warp * 64 + e * 32 + lane;
            nxt[e] = i < nc ? __ldcg(cq + i) : kKeyEmpty;
        }
        for (int base = warp * 64; base < nc; base += kStep) {
            u64 cur[2] = {nxt[0], nxt[1]};
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int i = base + kStep + e * 32 + lane;
                nxt[e] = i < nc ? __ldcg(cq + i) : kKeyEmpty;
            }
            const u64 worst = __shfl_sync(kFull, best[1], 31);
            if (!__any_sync(kFull, cur[0] < worst || cur[1] < worst)) continue;
            warp_sort64(cur, lane);
            warp_merge64(best, cur, lane);
        }
#pragma unroll
        for (int e = 0; e < 2; ++e) wl[warp * 64 + e * 32 + lane] = best[e];
        __syncthreads();
        if (warp == 0) {
            for (int w = 1; w < kMergeWarps; ++w) {
                const u64 cur[2] = {wl[w * 64 + lane], wl[w * 64 + 32 + lane]};
                warp_merge64(best, cur, lane);
            }
#pragma unroll
            for (int e = 0; e < 2; ++e) cw[e * 32 + lane] = best[e];
            if (lane == 0) s_n = W;
        }
    } else if (warp == 0) {
        int n = 0;
        if (cand != nullptr && c >= (unsigned)W && c <= (unsigned)kCap) {
            // the main pass collected every key <= tau, and there are W..kCap of them
            n = (int)c;
            for (int i = lane; i < n; i += 32) cw[i] = __ldcg(cand + (size_t)qi * kCap + i);
        } else {
            // per-chunk top-W lists of the full pass; every key of the global top W
            // is <= the smallest chunk's W-th key
            const u64* P = partial + (size_t)qi * nchunks * W;
            const int total = nchunks * W;
            u64 bound = kKeyEmpty;
            for (int ch = lane; ch < nchunks; ch += 32) {
                const u64 v = __ldcg(P + (size_t)ch * W + W - 1);
                bound = v < bound ? v : bound;
            }
            bound = warp_min_u64(bound);
            int cntle = count_le(P, total, bound, lane);
            if (cntle > kCap) {
                // many keys near the bound: bisect for the W-th smallest key
                u64 lo = 0, hi = bound;
                while (lo < hi) {
                    const u64 mid = lo + (hi - lo) / 2;
                    if (count_le(P, total, mid, lane) >= W) hi = mid;
                    else lo = mid + 1;
                }
                bound = lo;
            }
            for (int base = 0; base < total; base += 32) {
                const int i = base + lane;
                const u64 key = i < total ? __ldcg(P + i) : kKeyEmpty;
                const bool take = key != kKeyEmpty && key <= bound;
                const unsigned m = __ballot_sync(kFull, take);
                const int pos = n + __popc(m & ((1u << lane) - 1u));
                if (take && pos < kCap) cw[pos] = key;
                n += __popc(m);
            }
            n = min(n, kCap);
        }
        __syncwarp();
        int p2 = 32;
        while (p2 < n) p2 <<= 1;
        for (int i = n + lane; i < p2; i += 32) cw[i] = kKeyEmpty;
        __syncwarp();
        warp_sort(cw, p2, lane);
        if (lane == 0) s_n = n;
    }
    __syncthreads();
    const int take = min(s_n, W);
    // FP32 direct re-rank of the shortlist: warp w takes kInFlight rows at a time (rows
    // w * kInFlight + j kMergeWarps kInFlight ..), their keys into wl
    constexpr int kInFlight = CPL <= 2 ? 8 : 4;
    const int D4 = D / 4;
    float4 qv[CPL];
#pragma unroll
    for (int j = 0; j < CPL; ++j) {
        const int cc = lane + 32 * j;
        qv[j] = cc < D4 ? reinterpret_cast<const float4*>(Q + (size_t)qi * D)[cc] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const float2 neg1 = make_float2(-1.f, -1.f);
    for (int i0 = warp * kInFlight; i0 < take; i0 += kMergeWarps * kInFlight) {
        uint32_t r[kInFlight];
        float4 x[kInFlight][CPL];
#pragma unroll
        for (int b = 0; b < kInFlight; ++b) {
            r[b] = i0 + b < take ? (uint32_t)cw[i0 + b] : 0xffffffffu;
#pragma unroll
            for (int j = 0; j < CPL; ++j) {
                const int cc = lane + 32 * j;
                x[b][j] = (r[b] != 0xffffffffu && cc < D4)
                              ? __ldg(reinterpret_cast<const float4*>(X + (size_t)r[b] * D) + cc)
                              : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        float d[kInFlight];
#pragma unroll
        for (int b = 0; b < kInFlight; ++b) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < CPL; ++j) {
                float2 a = __ffma2_rn(make_float2(x[b][j].x, x[b][j].y), neg1, make_float2(qv[j].x, qv[j].y));
                float2 e = __ffma2_rn(make_float2(x[b][j].z, x[b][j].w), neg1, make_float2(qv[j].z, qv[j].w));
                acc = __ffma2_rn(a, a, acc);
                acc = __ffma2_rn(e, e, acc);
            }
            d[b] = acc.x + acc.y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int b = 0; b < kInFlight; ++b) d[b] += __shfl_xor_sync(kFull, d[b], o);
        }
        if (lane < kInFlight) {
#pragma unroll
            for (int b = 0; b < kInFlight; ++b)
                if (b == lane && r[b] != 0xffffffffu) wl[i0 + b] = make_key(d[b], r[b]);
        }
    }
    __syncthreads();
    if (warp == 0) {
        // the exact keys sorted; the first k are the answer
        int p2 = 32;
        while (p2 < take) p2 <<= 1;
        for (int i = take + lane; i < p2; i += 32) wl[i] = kKeyEmpty;
        __syncwarp();
        warp_sort(wl, p2, lane);
        if (lane < k) {
            const size_t o = (size_t)qi * k + lane;
            const u64 L = lane < take ? wl[lane] : kKeyEmpty;
            if (L == kKeyEmpty) {
                idx[o] = -1;
                dist[o] = __int_as_float(0x7f800000);
            } else {
                idx[o] = (int64_t)key_row(L);
                dist[o] = key_dist(L);
            }
        }
    }
}

// ------------------------------------------------------------------ host
bool make_map(CUtensorMap* map, const void* base, int64_t rows, int D, bool fp8, int box_rows = kTile) {
    return tc::make_map(map, base, rows, D, fp8 ? kTcFP8 : kTcBF16, box_rows);
}

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Chunking {
    int chunk_rows, nchunks;
};

// About one CTA per SM over qblocks x chunks; chunks are whole tiles.
Chunking chunking(int64_t rows, int qblocks, int sms) {
    Chunking c{};
    const int target = std::max(1, sms / qblocks);
    int64_t cr = (rows + target - 1) / target;
    cr = std::max<int64_t>(kTile, (cr + kTile - 1) / kTile * kTile);
    c.chunk_rows = (int)cr;
    c.nchunks = (int)((rows + cr - 1) / cr);
    return c;
}

struct LowpPlan {
    int nq_pad, qblocks, wmax;
    int nq_sorted, qblocks_main;  // main pass: 256-query blocks of threshold-sorted queries
    bool sampled;
    Chunking main, pilot;
    size_t codes_bytes, qs_bytes, pilot_bytes, tau_bytes, cnt_bytes, cand_bytes, partial_bytes, sort_bytes;
};

LowpPlan plan(const lhr_db* db, int nq, bool fp8, int W) {
    LowpPlan pl{};
    pl.nq_pad = (nq + kTile - 1) / kTile * kTile;
    pl.qblocks = pl.nq_pad / kTile;
    pl.nq_sorted = (nq + kQTile - 1) / kQTile * kQTile;
    pl.qblocks_main = pl.nq_sorted / kQTile;
    pl.wmax = W <= 32 ? 32 : (W <= 64 ? 64 : 128);
    pl.sampled = (fp8 ? db->X8_s : db->Xb_s) != nullptr;
    pl.main = chunking(db->n, pl.qblocks, db->sms);
    pl.pilot = chunking(std::max<int64_t>(db->n_sample, 1), pl.qblocks_main, db->sms);
    const int elem = fp8 ? 1 : 2;
    pl.codes_bytes = a256((size_t)pl.nq_pad * db->dim * elem);
    pl.qs_bytes = a256(4 * sizeof(float));  // s_Q, m, max |q| bits
    pl.pilot_bytes = pl.sampled ? a256((size_t)nq * pl.pilot.nchunks * 4 * kPilotR * sizeof(u64)) : 0;
    pl.tau_bytes = pl.sampled ? a256((size_t)pl.nq_pad * sizeof(u64)) + a256((size_t)pl.nq_pad * sizeof(float)) : 0;
    pl.cnt_bytes = pl.sampled ? a256((size_t)nq * sizeof(unsigned)) : 0;
    pl.cand_bytes = pl.sampled ? a256((size_t)nq * kCap * sizeof(u64)) : 0;
    pl.partial_bytes = a256((size_t)nq * pl.main.nchunks * kHalves * W * sizeof(u64));
    // sorted codes, perm, group thresholds
    pl.sort_bytes = pl.sampled ? a256((size_t)pl.nq_sorted * db->dim * elem) + a256((size_t)pl.nq_sorted * sizeof(int)) +
                                     a256((size_t)pl.nq_sorted / 32 * sizeof(float))
                               : 0;
    return pl;
}

constexpr size_t kSmemLimit = 227 * 1024;  // dynamic shared memory per CTA

size_t tc_smem_fixed(int slices, int mode) {
    return 1024 + (size_t)slices * kSliceTile + kSnSlots * kTile * sizeof(float2) +
           (size_t)kBuf * kEpiThreads * sizeof(u64) +
           (2 * kMaxStages + 1 + 2 * kAcc + 2 * kSnSlots) * sizeof(u64) + 16;
}

// Ring depth: as many slices as fit beside the resident query codes (>= 2).
int tc_stages(int slices, int mode) {
    const size_t fixed = tc_smem_fixed(slices, mode);
    const int fit = fixed < kSmemLimit ? (int)((kSmemLimit - fixed) / kSliceTile) : 0;
    return std::min(kMaxStages, fit);
}

size_t tc_smem(int slices, int stages, int mode) { return tc_smem_fixed(slices, mode) + (size_t)stages * kSliceTile; }

size_t main_smem(int slices, int stages) {
    return 1024 + (size_t)slices * kQTile * kSliceBytes + (size_t)stages * kSliceTile +
           (size_t)kMGroups * kOwnSlots * kMainEpiThreads * sizeof(u64) +
           (size_t)kMainEpiWarps * kTRows * kTStride * sizeof(float) + (size_t)2 * kMGroups * kMainEpiThreads * 4 +
           (2 * kMaxStages + 1 + 2 * kMainAcc) * sizeof(u64) + 16;
}

int main_stages(int slices) {
    const size_t fixed = main_smem(slices, 0);
    const int fit = fixed < kSmemLimit ? (int)((kSmemLimit - fixed) / kSliceTile) : 0;
    return std::min(kMaxStages, fit);
}

template <bool kFp8, bool kPilot = false>
cudaError_t launch_main(const CUtensorMap& mq, const CUtensorMap& mx, const MainParams& mp, int qblocks,
                        cudaStream_t stream) {
    auto kern = tc_main_kernel<kFp8, kPilot>;
    if (mp.stages < 2 || mp.stages > kMaxStages) return cudaErrorInvalidValue;
    if (mp.cs < 1 || qblocks % mp.cs || kTile % mp.cs) return cudaErrorInvalidValue;
    const size_t sm = main_smem(mp.slices, mp.stages);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    ProfScope ps(kPilot ? (kFp8 ? "tc_pilot_kernel_fp8" : "tc_pilot_kernel_bf16")
                        : (kFp8 ? "tc_main_kernel_fp8" : "tc_main_kernel_bf16"),
                 stream);
    // qblocks of kQTile queries; clusters of mp.cs CTAs along them
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(mp.nchunks, qblocks);
    cfg.blockDim = dim3(kMainThreads);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = (unsigned)mp.cs;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, mq, mx, mp);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// Clusters of cs main-pass CTAs that can be resident at once (cached per device, format and size).
template <bool kFp8>
cudaError_t main_max_clusters(size_t smem, int cs, int* out) {
    static std::mutex mu;
    static int cache[64][3] = {};  // [device][log2 cs]
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const int li = cs == 4 ? 2 : (cs == 2 ? 1 : 0);
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 64 && cache[dev][li] > 0) {
        *out = cache[dev][li];
        return cudaSuccess;
    }
    auto kern = tc_main_kernel<kFp8, false>;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs, 1);
    cfg.blockDim = dim3(kMainThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if ((e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg)) != cudaSuccess) return e;
    if (dev < 64) cache[dev][li] = n;
    *out = n;
    return cudaSuccess;
}

template <bool kFp8, int MODE, int WMAX>
cudaError_t launch_tc(const CUtensorMap& ma, const CUtensorMap& mb, const TcParams& tp, int qblocks,
                      cudaStream_t stream, const char* name) {
    auto kern = tc_kernel<kFp8, MODE, WMAX>;
    if (tp.stages < 2 || tp.stages > kMaxStages) return cudaErrorInvalidValue;
    const size_t sm = tc_smem(tp.slices, tp.stages, MODE);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    ProfScope ps(name, stream);
    kern<<<dim3(tp.nchunks, qblocks), kThreads, sm, stream>>>(ma, mb, tp);
    return cudaGetLastError();
}

template <bool kFp8>
cudaError_t launch_full(int wmax, const CUtensorMap& ma, const CUtensorMap& mb, const TcParams& tp, int qblocks,
                        cudaStream_t stream) {
    const char* name = kFp8 ? "tc_full_kernel_fp8" : "tc_full_kernel_bf16";
    if (wmax == 32) return launch_tc<kFp8, kModeFull, 32>(ma, mb, tp, qblocks, stream, name);
    if (wmax == 64) return launch_tc<kFp8, kModeFull, 64>(ma, mb, tp, qblocks, stream, name);
    return launch_tc<kFp8, kModeFull, 128>(ma, mb, tp, qblocks, stream, name);
}

}  // namespace

cudaError_t launch_sort_queries(const float* key, int nq, int n_sorted, const void* codes, int row_bytes,
                                void* codes_s, int* perm, float* gmax, cudaStream_t stream) {
    if (n_sorted % kQTile || row_bytes % 16) return cudaErrorInvalidValue;
    int n2 = 1;
    while (n2 < n_sorted) n2 <<= 1;
    const size_t ssm = n_sorted <= kSortMax ? (size_t)std::max(n2, kRegSort) * sizeof(u64) : 0;
    cudaError_t e = cudaFuncSetAttribute(sort_queries_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssm);
    if (e != cudaSuccess) return e;
    ProfScope ps("sort_queries_kernel", stream);
    sort_queries_kernel<<<n_sorted / kQTile, kSortThreads, ssm, stream>>>(
        key, nq, n_sorted, reinterpret_cast<const uint4*>(codes), row_bytes / 16, reinterpret_cast<uint4*>(codes_s),
        perm, gmax);
    return cudaGetLastError();
}

size_t lowp_scratch_bytes(const lhr_db* db, int nq, bool fp8, int W) {
    const LowpPlan pl = plan(db, nq, fp8, W);
    return pl.codes_bytes + pl.qs_bytes + pl.pilot_bytes + pl.tau_bytes + pl.cnt_bytes + pl.cand_bytes +
           pl.partial_bytes + pl.sort_bytes;
}

cudaError_t launch_lowp(const lhr_db* db, const float* q, int nq, bool fp8, int W, int k, int64_t* idx, float* dist,
                        void* scratch, cudaStream_t stream) {
    const LowpPlan pl = plan(db, nq, fp8, W);
    unsigned char* base = reinterpret_cast<unsigned char*>(scratch);
    void* codes = base;
    base += pl.codes_bytes;
    float* qs = reinterpret_cast<float*>(base);
    base += pl.qs_bytes;
    u64* pilot = reinterpret_cast<u64*>(base);
    base += pl.pilot_bytes;
    u64* tau_key = reinterpret_cast<u64*>(base);
    float* tau_s = reinterpret_cast<float*>(base + a256((size_t)pl.nq_pad * sizeof(u64)));
    base += pl.tau_bytes;
    unsigned* cnt = reinterpret_cast<unsigned*>(base);
    base += pl.cnt_bytes;
    u64* cand = reinterpret_cast<u64*>(base);
    base += pl.cand_bytes;
    u64* partial = reinterpret_cast<u64*>(base);
    base += pl.partial_bytes;
    void* codes_s = base;
    int* perm = reinterpret_cast<int*>(base + a256((size_t)pl.nq_sorted * db->dim * (fp8 ? 1 : 2)));
    float* tgrp = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(perm) +
                                           a256((size_t)pl.nq_sorted * sizeof(int)));
    cudaError_t e;
    {
        ProfScope ps("quantize_queries_kernel", stream);
        unsigned* amax_bits = reinterpret_cast<unsigned*>(qs + 2);
        if ((e = cudaMemsetAsync(amax_bits, 0, sizeof(unsigned), stream)) != cudaSuccess) return e;
        const int64_t count = (int64_t)nq * db->dim;
        const int ablocks = (int)std::min<int64_t>(std::max<int64_t>((count + 1023) / 1024, 1), db->sms);
        query_amax_kernel<<<ablocks, 256, 0, stream>>>(q, count, amax_bits);
        const float qmax = fp8 ? 448.0f : 1.0f;
        const int blocks = (pl.nq_pad * 32 + 255) / 256;
        if (fp8)
            quantize_queries_kernel<true><<<blocks, 256, 0, stream>>>(q, nq, pl.nq_pad, db->dim, amax_bits, qmax, qs, codes);
        else
            quantize_queries_kernel<false><<<blocks, 256, 0, stream>>>(q, nq, pl.nq_pad, db->dim, amax_bits, qmax, qs,
                                                                       codes);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    CUtensorMap ma, mb, ms;
    if (!make_map(&ma, codes, pl.nq_pad, db->dim, fp8) || !make_map(&mb, fp8 ? db->X8 : db->Xb, db->n, db->dim, fp8))
        return cudaErrorInvalidValue;
    TcParams tp{};
    tp.slices = db->dim * (fp8 ? 1 : 2) / kSliceBytes;
    tp.qs = qs;
    tp.nq = nq;
    tp.W = W;
    tp.err = db->err;
    if (pl.sampled) {
        if (!make_map(&ms, fp8 ? db->X8_s : db->Xb_s, db->n_sample, db->dim, fp8)) return cudaErrorInvalidValue;
        // pilot over the sample: the main pass's pipeline, 32-row bucket minima per query
        MainParams pm{};
        pm.n = db->n_sample;
        pm.slices = tp.slices;
        pm.stages = main_stages(tp.slices);
        pm.chunk_rows = pl.pilot.chunk_rows;
        pm.nchunks = pl.pilot.nchunks;
        pm.sn = fp8 ? db->sn8_s : db->snb_s;
        pm.qs = qs;
        pm.nq = nq;
        pm.cs = 1;
        pm.pilot_out = pilot;
        pm.pilot_lists = pl.pilot.nchunks * 4;
        pm.err = db->err;
        e = fp8 ? launch_main<true, true>(ma, ms, pm, pl.qblocks_main, stream)
                : launch_main<false, true>(ma, ms, pm, pl.qblocks_main, stream);
        if (e != cudaSuccess) return e;
        {
            ProfScope ps("tau_kernel", stream);
            tau_kernel<<<(pl.nq_pad + 7) / 8, 256, 0, stream>>>(pilot, pl.pilot.nchunks * 4, nq, pl.nq_pad,
                                                                 tau_key, tau_s);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        // queries in ascending-threshold order, in 256-query blocks, for the main pass
        if ((e = launch_sort_queries(tau_s, nq, pl.nq_sorted, codes, db->dim * (fp8 ? 1 : 2), codes_s, perm, tgrp,
                                     stream)) != cudaSuccess)
            return e;
        // one CTA per cluster: sharing each database tile across the query blocks of a cluster (each
        // CTA loading 1/cs of it) cuts L2 reads but couples the CTAs' pipelines, and measured slower
        const int cs = 1;
        CUtensorMap mqs, mxp;
        if (!make_map(&mqs, codes_s, pl.nq_sorted, db->dim, fp8) ||
            !make_map(&mxp, fp8 ? db->X8 : db->Xb, db->n, db->dim, fp8, kTile / cs))
            return cudaErrorInvalidValue;
        // main pass: every key <= tau into the candidate buffers
        if ((e = cudaMemsetAsync(cnt, 0, (size_t)nq * sizeof(unsigned), stream)) != cudaSuccess) return e;
        MainParams mp{};
        mp.n = db->n;
        mp.slices = tp.slices;
        mp.stages = main_stages(tp.slices);
        {
            // as many chunks as keep every cluster resident at once (clusters live inside one GPC,
            // so fewer than sms / cs clusters may fit): no second wave
            int max_clusters = 0;
            const size_t msm = main_smem(mp.slices, main_stages(mp.slices));
            if ((fp8 ? main_max_clusters<true>(msm, cs, &max_clusters)
                     : main_max_clusters<false>(msm, cs, &max_clusters)) != cudaSuccess ||
                max_clusters < 1)
                max_clusters = db->sms / cs;
            const int max_ctas = std::min(db->sms, max_clusters * cs);
            const Chunking c = chunking(db->n, pl.qblocks_main, max_ctas);
            mp.chunk_rows = c.chunk_rows;
            mp.nchunks = c.nchunks;
        }
        mp.perm = perm;
        mp.tgrp = tgrp;
        mp.cs = cs;
        mp.sn = fp8 ? db->sn8 : db->snb;
        mp.qs = qs;
        mp.tau_s = tau_s;
        mp.tau_key = tau_key;
        mp.cand = cand;
        mp.cnt = cnt;
        mp.nq = nq;
        mp.err = db->err;
        e = fp8 ? launch_main<true>(mqs, mxp, mp, pl.qblocks_main, stream)
                : launch_main<false>(mqs, mxp, mp, pl.qblocks_main, stream);
        if (e != cudaSuccess) return e;
    }
    // full pass: always without a sample, otherwise only where a main pass fell short
    TcParams fp = tp;
    fp.n = db->n;
    fp.chunk_rows = pl.main.chunk_rows;
    fp.nchunks = pl.main.nchunks;
    fp.sn = fp8 ? db->sn8 : db->snb;
    fp.partial = partial;
    fp.cnt = pl.sampled ? cnt : nullptr;
    fp.stages = tc_stages(fp.slices, kModeFull);
    e = fp8 ? launch_full<true>(pl.wmax, ma, mb, fp, pl.qblocks, stream)
            : launch_full<false>(pl.wmax, ma, mb, fp, pl.qblocks, stream);
    if (e != cudaSuccess) return e;
    const int d4 = db->dim / 4;
    const int cpl = d4 <= 32 ? 1 : (d4 <= 64 ? 2 : 4);
    const size_t msm = (size_t)(kCap + kMergeWarps * 64) * sizeof(u64);
    const u64* candp = pl.sampled ? cand : nullptr;
    const int blocks = nq;  // one query per block
#define LHR_MR(C)                                                                                              \
    do {                                                                                                       \
        e = cudaFuncSetAttribute(merge_rerank_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)msm); \
        if (e != cudaSuccess) return e;                                                                        \
        ProfScope ps("merge_rerank_kernel", stream);                                                           \
        merge_rerank_kernel<C><<<blocks, kMergeWarps * 32, msm, stream>>>(partial, pl.main.nchunks * kHalves, W, candp, cnt, \
                                                                            db->X, db->dim, q, nq, k, idx, dist); \
    } while (0)
    if (cpl == 1) LHR_MR(1);
    else if (cpl == 2) LHR_MR(2);
    else LHR_MR(4);
#undef LHR_MR
    return cudaGetLastError();
}

}  // namespace lhr
