// Exhaustive FP32 scan with fused per-frame, per-subspace top-N (§3.1,
// Algorithm 1: calculateDistance for every (query frame, database frame) pair,
// then selectTopCandidates; §4: Euclidean distance, top N).
//
// Design (GB300): for a handful of query frames the scan is bound by HBM, so
// every database byte is read once per launch and the arithmetic per byte is
// kept small.
//   * One CTA per (row chunk, block of QB query frames). A row chunk is a
//     contiguous range of one subspace; the chunk table is built with the
//     database. The frame block is the grid's fastest index, so the CTAs
//     resident together share chunks: with many frame blocks a chunk comes
//     from DRAM once and from L2 for the other blocks (chunk-fastest order
//     would stream the whole database from DRAM once per frame block).
//   * A producer thread streams the chunk through shared memory with 1-D bulk
//     copies (cp.async.bulk, 16 rows per stage) into an mbarrier ring; consumer
//     warp w owns the stages s with s % warps == w, so its parity waits always
//     see consecutive phases.
//   * Filter: lanes split the feature dimensions (float4 chunks,
//     conflict-free), the QB frames sit in registers, and each lane forms
//     partial dot products q.x with packed FP32 FMAs (one instruction per two
//     elements). A 5-step butterfly transpose-reduce leaves lane l with the
//     dot product of (row l / QB, frame l % QB), and
//     d~ = ||x||^2 + ||q||^2 - 2 q.x
//     (row norms built with the database). d~ differs from the exact value by
//     at most (gamma_D + 3u)(||x|| + ||q||)^2 (dot-product error bound, u =
//     2^-24), and so does the FP32 direct form; a row can only enter the list
//     if d~ <= threshold + 2 (gamma_D + 3u)(max||x|| + ||q||)^2.
//   * Rows that pass (rare once the lists fill) get their exact direct-form
//     distance sum_j (q_j - x_j)^2, recomputed by the warp from shared memory,
//     and are inserted into the warp's per-frame top-k list (shared memory,
//     lane i holds the i-th key). Keys are (distance bits << 32 | row): ties go
//     to the lower row. A per-frame threshold shared by the CTA's warps (the
//     smallest k-th distance of any warp) prunes further: an element above
//     another warp's k-th cannot be in the CTA's top k.
//   * Warp lists merge into a per-CTA list written to scratch; the last CTA of
//     a query block (atomic ticket) merges every chunk of each subspace, keys
//     above the smallest per-chunk k-th key being skipped, and writes the
//     final lists. One launch per call; the distance matrix never leaves the SM.
#include <math.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "common.cuh"
#include "internal.h"
#include "select.cuh"

namespace lhr {
namespace {

constexpr int kRPS = 16;           // rows per stage
constexpr int kMaxWarps = 12;      // consumer warps per CTA
constexpr int kMaxSmem = 227 * 1024;

struct ScanParams {
    const float* X;
    const float* xnorm;
    int D;
    const int4* chunks;
    int nchunks;
    const int32_t* chunk_off;
    int n_sub;
    const int32_t* perm;
    const float* Q;
    int nq;
    int k;
    int stages;
    const unsigned* bmin;  // nullable: [nq][n_sub][kPilotBuckets] pilot bucket minima (float bits; ~0u = empty)
    const float* w;        // nullable: per-dimension weights (>= 0) of the weighted distance; NULL = all 1
    const float* xmax_w;   // nullable: device max over rows of sum_j w_j x_j^2 (weighted scans)
    float xmax;          // sqrt(max ||x||^2)
    float margin_scale;  // 2 (gamma_D + 3u)
    u64* partial;        // [qblock][QB][nchunks][k]
    unsigned* counters;  // [qblock]
    unsigned* gthr;      // [qblock * QB][n_sub]: grid-wide k-th distance bound (float bits)
    int64_t* idx;        // [nq][n_sub][k]
    float* dist;
    int* err;
};

struct ScanConfig {
    int qb, cpl, warps, stages;
    size_t smem;
};

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

constexpr int kPilotBuckets = 128;

// Pilot bound of frame qi in subspace `sub`, by one warp. The pilot sample's
// rows were dealt into 128 buckets (row j -> j mod 128) and each bucket keeps
// its minimum distance; the k-th smallest non-empty bucket minimum (ties by
// bucket) is reached by k distinct database rows, so it bounds the frame's
// k-th distance from above, and it seldom exceeds the sample's own k-th (the
// best rows rarely share a bucket). Any k consecutive rows fill k buckets.
// The bound is widened by 2^-12 relative against a difference in the last
// bits between the two kernels' distances, and lowers *thr (float bits).
__device__ void pilot_bound(const ScanParams& p, int qi, int sub, int lane, unsigned* thr) {
    const unsigned* bm = p.bmin + ((size_t)qi * p.n_sub + sub) * kPilotBuckets;
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
    if (lane == 0 && b < 0x7f800000u) {
        const float w = __uint_as_float(b) * (1.0f + 1.0f / 4096.0f);
        atomicMin(thr, __float_as_uint(w));
    }
}

template <int QB, int CPL>
__global__ void __launch_bounds__((kMaxWarps + 1) * 32, 1) scan_topk_kernel(const ScanParams p) {
    constexpr int RW = 32 / QB;  // rows per reduction round
    constexpr int kRounds = kRPS / RW;
    static_assert(kRPS % RW == 0, "stage rows must hold whole rounds");
    extern __shared__ __align__(128) unsigned char smem[];
    const int warps = blockDim.x / 32 - 1;  // consumer warps; the last warp produces
    const int warp = threadIdx.x / 32;
    const int lane = threadIdx.x % 32;
    const int D = p.D;
    const int D4 = D / 4;
    const int NS = p.stages;
    const size_t stage_floats = (size_t)kRPS * D;

    float* stage_buf = reinterpret_cast<float*>(smem);
    float* qs = stage_buf + NS * stage_floats;                            // QB x D
    float* ws = qs + (size_t)QB * D;                                      // D weights
    u64* full = reinterpret_cast<u64*>(ws + D);
    u64* empty = full + NS;
    u64* lists = empty + NS;                                              // [warps][QB][32]
    unsigned* thr_sh = reinterpret_cast<unsigned*>(lists + (size_t)warps * QB * 32);  // QB float bits
    int* flags = reinterpret_cast<int*>(thr_sh + QB);
    volatile int* abort_flag = flags;

    const int qblock = blockIdx.x;
    const int chunk = blockIdx.y;
    const int4 ch = p.chunks[chunk];
    const int row0 = ch.x, row1 = ch.y;
    const int iters = (row1 - row0 + kRPS - 1) / kRPS;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        flags[0] = 0;
        flags[1] = 0;
        fence_mbar_init();
    }
    for (int i = threadIdx.x; i < QB * D4; i += blockDim.x) {
        const int q = i / D4, c = i % D4;
        const int qi = qblock * QB + q;
        reinterpret_cast<float4*>(qs)[i] =
            qi < p.nq ? reinterpret_cast<const float4*>(p.Q)[(size_t)qi * D4 + c] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int i = threadIdx.x; i < D; i += blockDim.x) ws[i] = p.w != nullptr ? p.w[i] : 1.f;
    for (int i = threadIdx.x; i < warps * QB * 32; i += blockDim.x) lists[i] = kKeyEmpty;
    if (threadIdx.x < QB) thr_sh[threadIdx.x] = 0x7f800000u;  // +inf
    __syncthreads();

    if (warp == warps) {
        // ------------------------------------------------ producer
        if (lane == 0) {
            int issued = 0;
            for (int it = 0; it < iters; ++it) {
                const int s = it % NS;
                const uint32_t ph = (uint32_t)(it / NS) & 1u;
                if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag)) {
                    *abort_flag = 1;
                    record_error(p.err, kErrTimeout);
                    break;
                }
                const int r = row0 + it * kRPS;
                const int nr = min(kRPS, row1 - r);
                const uint32_t bytes = (uint32_t)nr * (uint32_t)D * 4u;
                mbar_arrive_expect_tx(&full[s], bytes);
                bulk_g2s(stage_buf + s * stage_floats, p.X + (size_t)r * D, bytes, &full[s]);
                ++issued;
            }
            if (*abort_flag) {
                // Let the copies this thread issued land before the CTA exits.
                for (int it = max(0, issued - NS); it < issued; ++it)
                    mbar_wait(&full[it % NS], (uint32_t)(it / NS) & 1u, nullptr);
            }
        }
    } else {
        // ------------------------------------------------ consumers
        float4 qreg[QB][CPL];
        float qpart[QB];
#pragma unroll
        for (int q = 0; q < QB; ++q) {
            float a = 0.f;
#pragma unroll
            for (int j = 0; j < CPL; ++j) {
                // registers hold w * q; ||q||_w^2 = sum_j (w_j q_j) q_j
                const int c = lane + 32 * j;
                const float4 qv = c < D4 ? reinterpret_cast<const float4*>(qs + (size_t)q * D)[c]
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 wv = c < D4 ? reinterpret_cast<const float4*>(ws)[c] : make_float4(0.f, 0.f, 0.f, 0.f);
                qreg[q][j] = make_float4(wv.x * qv.x, wv.y * qv.y, wv.z * qv.z, wv.w * qv.w);
                a = fmaf(qreg[q][j].x, qv.x, a);
                a = fmaf(qreg[q][j].y, qv.y, a);
                a = fmaf(qreg[q][j].z, qv.z, a);
                a = fmaf(qreg[q][j].w, qv.w, a);
            }
            qpart[q] = a;
        }
        // ||q||^2 of this lane's frame (lane % QB), and its filter margin
        float qn = 0.f;
#pragma unroll
        for (int q = 0; q < QB; ++q) {
            float a = qpart[q];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(kFull, a, o);
            if ((lane % QB) == q) qn = a;
        }
        if (p.bmin != nullptr)
            for (int f = warp; f < QB && qblock * QB + f < p.nq; f += warps) pilot_bound(p, qblock * QB + f, ch.z, lane, &thr_sh[f]);
        const int myq = lane % QB;
        const bool q_valid = (qblock * QB + myq) < p.nq;
        const float rad = (p.xmax_w != nullptr ? sqrtf(__ldg(p.xmax_w)) * 1.0001f : p.xmax) + sqrtf(qn);
        const float margin = p.margin_scale * rad * rad;
        float thr_own = __int_as_float(0x7f800000);  // k-th distance of this warp's list for frame myq
        const int jr = (p.k + warps - 1) / warps;      // rank read from every warp's list for the CTA bound
        u64* wlist = lists + (size_t)warp * QB * 32;
        const volatile unsigned* thr_v = thr_sh;     // other warps lower it with atomicMin
        // grid-wide per-frame bound: the smallest k-th distance any warp of any
        // CTA of this subspace holds (float bits; 0xffffffff = none yet)
        unsigned* gthr = p.gthr + ((size_t)qblock * QB) * p.n_sub + ch.z;
        // row norms of this warp's next stage, loaded one stage ahead
        float xn_next = 0.f;
        if (warp < iters) {
            const int r = row0 + warp * kRPS;
            xn_next = lane < min(kRPS, row1 - r) ? __ldg(p.xnorm + r + lane) : 0.f;
        }

        for (int it = warp; it < iters; it += warps) {
            const int s = it % NS;
            const uint32_t ph = (uint32_t)(it / NS) & 1u;
            const int rbase = row0 + it * kRPS;
            const int nr = min(kRPS, row1 - rbase);
            const float xn_l = xn_next;
            if (it + warps < iters) {
                const int r = row0 + (it + warps) * kRPS;
                xn_next = lane < min(kRPS, row1 - r) ? __ldg(p.xnorm + r + lane) : 0.f;
            }
            const unsigned gbound = lane < QB ? __ldcg(gthr + (size_t)lane * p.n_sub) : 0xffffffffu;
            if (!mbar_wait(&full[s], ph, abort_flag)) {
                if (lane == 0) {
                    *abort_flag = 1;
                    record_error(p.err, kErrTimeout);
                }
                break;
            }
            const float* sbf = stage_buf + s * stage_floats;
            const float4* sb = reinterpret_cast<const float4*>(sbf);
#pragma unroll 1
            for (int rr = 0; rr < kRounds; ++rr) {
                const int rb = rr * RW;
                float part[32];
#pragma unroll
                for (int r = 0; r < RW; ++r) {
                    float4 x[CPL];
#pragma unroll
                    for (int j = 0; j < CPL; ++j) {
                        const int c = lane + 32 * j;
                        x[j] = (c < D4) ? sb[(rb + r) * D4 + c] : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
#pragma unroll
                    for (int q = 0; q < QB; ++q) {
                        float2 acc = f2(0.f, 0.f);
#pragma unroll
                        for (int j = 0; j < CPL; ++j) {
                            acc = __ffma2_rn(f2(x[j].x, x[j].y), f2(qreg[q][j].x, qreg[q][j].y), acc);
                            acc = __ffma2_rn(f2(x[j].z, x[j].w), f2(qreg[q][j].z, qreg[q][j].w), acc);
                        }
                        part[r * QB + q] = acc.x + acc.y;
                    }
                }
                // Butterfly transpose-reduce: lane l ends with value index l.
#pragma unroll
                for (int st = 16; st >= 1; st >>= 1) {
                    const bool upper = (lane & st) != 0;
#pragma unroll
                    for (int v = 0; v < st; ++v) {
                        const float send = upper ? part[v] : part[v + st];
                        const float keep = upper ? part[v + st] : part[v];
                        part[v] = keep + __shfl_xor_sync(kFull, send, st);
                    }
                }
                const int rl = rb + lane / QB;
                const float xn = __shfl_sync(kFull, xn_l, rl);
                const float approx = fmaf(-2.f, part[0], xn + qn);
                const float thr = fminf(thr_own, __uint_as_float(thr_v[myq]));
                const bool pass = q_valid && rl < nr && approx <= thr + margin;
                unsigned m = __ballot_sync(kFull, pass);
                while (m) {
                    const int j = __ffs(m) - 1;
                    m &= m - 1;
                    const int rj = rb + j / QB, qj = j % QB;
                    // exact direct-form distance of (row rj, frame qj)
                    const float4* xr = reinterpret_cast<const float4*>(sbf + (size_t)rj * D);
                    const float4* qr = reinterpret_cast<const float4*>(qs + (size_t)qj * D);
                    const float4* wr = reinterpret_cast<const float4*>(ws);
                    float2 acc = f2(0.f, 0.f);
#pragma unroll
                    for (int jj = 0; jj < CPL; ++jj) {
                        const int c = lane + 32 * jj;
                        if (c < D4) {
                            // w (q - x)^2; with w = 1 the product is exact and this is sum (q - x)^2
                            const float4 x = xr[c], qv = qr[c], wv = wr[c];
                            const float2 d0 = __ffma2_rn(f2(x.x, x.y), f2(-1.f, -1.f), f2(qv.x, qv.y));
                            const float2 d1 = __ffma2_rn(f2(x.z, x.w), f2(-1.f, -1.f), f2(qv.z, qv.w));
                            acc = __ffma2_rn(__fmul2_rn(d0, f2(wv.x, wv.y)), d0, acc);
                            acc = __ffma2_rn(__fmul2_rn(d1, f2(wv.z, wv.w)), d1, acc);
                        }
                    }
                    float de = acc.x + acc.y;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) de += __shfl_xor_sync(kFull, de, o);
                    if (de > __uint_as_float(thr_v[qj])) continue;  // another warp already holds k better
                    const u64 key = make_key(de, (uint32_t)(rbase + rj));
                    u64 L = wlist[qj * 32 + lane];
                    const u64 kth = __shfl_sync(kFull, L, p.k - 1);
                    if (key >= kth) continue;
                    list_insert(L, key, p.k, lane);
                    wlist[qj * 32 + lane] = L;
                    const u64 nk = __shfl_sync(kFull, L, p.k - 1);
                    if (nk != kKeyEmpty) {
                        const float nd = key_dist(nk);
                        if (myq == qj) thr_own = nd;
                        if (lane == 0) atomicMin(&thr_sh[qj], __float_as_uint(nd));
                    }
                    __syncwarp();
                }
            }
            // CTA bound from every warp's list: warp w's jr-th key has jr rows
            // at or below it, the warps' rows are disjoint and warps x jr >= k,
            // so the largest of those keys bounds the CTA's k-th. A list read
            // while its owner inserts is at worst stale, i.e. larger: still valid.
            // (With a pilot bound the lists rarely beat it: skipped.)
            if (p.bmin == nullptr && lane < QB) {
                u64 b = 0ull;
                for (int w = 0; w < warps; ++w) {
                    const u64 v = reinterpret_cast<const volatile u64*>(lists)[((size_t)w * QB + lane) * 32 + jr - 1];
                    b = v > b ? v : b;
                }
                if (b != kKeyEmpty) atomicMin(&thr_sh[lane], __float_as_uint(key_dist(b)));
            }
            // exchange bounds with the rest of the grid (gbound was loaded at the
            // stage's start): publish ours only when it is better, so the few
            // global words see rare atomics
            if (lane < QB) {
                const unsigned mine = thr_v[lane];
                if (mine < gbound) atomicMin(gthr + (size_t)lane * p.n_sub, mine);
                else if (gbound < mine) atomicMin(&thr_sh[lane], gbound);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
        }
    }
    __syncthreads();

    // ---------------------------------------------------- per-CTA merge
    const int nwarps = warps + 1;
    for (int q = warp; q < QB; q += nwarps) {
        u64 M = kKeyEmpty;
        for (int w = 0; w < warps; ++w) list_merge_keys<false>(M, &lists[((size_t)w * QB + q) * 32], p.k, p.k, lane);
        if (lane < p.k) p.partial[(((size_t)qblock * QB + q) * p.nchunks + chunk) * p.k + lane] = M;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned ticket = atomicAdd(&p.counters[qblock], 1u);
        flags[1] = (ticket == (unsigned)p.nchunks - 1u) ? 1 : 0;
    }
    __syncthreads();
    if (!flags[1]) return;
    __threadfence();

    // ---------------------------------------------------- last CTA: final lists
    // G warps share each (frame, subspace) pair: each merges a share of the
    // pair's chunk lists, then the pair's first warp merges the G results.
    const int pairs = min(QB, p.nq - qblock * QB) * p.n_sub;  // (frame, subspace) pairs of real frames
    const int G = max(1, nwarps / pairs);
    const int per_round = nwarps / G;
    u64* mlist = lists;  // free now: [nwarps][32]
    for (int pbase = 0; pbase < pairs; pbase += per_round) {
        const int pair = pbase + warp / G;
        const int g = warp % G;
        const bool active = warp / G < per_round && pair < pairs;
        const int q = active ? pair / p.n_sub : 0;
        const int sub = active ? pair % p.n_sub : 0;
        const int qi = qblock * QB + q;
        u64 M = kKeyEmpty;
        if (active && qi < p.nq) {
            const int c0 = p.chunk_off[sub], c1 = p.chunk_off[sub + 1];
            const u64* P = p.partial + (((size_t)qblock * QB + q) * p.nchunks + c0) * p.k;
            // every key of the subspace's top k is <= the smallest per-chunk k-th key
            u64 bound = kKeyEmpty;
            for (int c = lane; c < c1 - c0; c += 32) {
                const u64 v = __ldcg(P + (size_t)c * p.k + p.k - 1);
                bound = v < bound ? v : bound;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const u64 v = __shfl_xor_sync(kFull, bound, o);
                bound = v < bound ? v : bound;
            }
            const int nch = c1 - c0;
            const int ca = (int)((int64_t)nch * g / G), cb = (int)((int64_t)nch * (g + 1) / G);
            const u64* Pg = P + (size_t)ca * p.k;
            const int total = (cb - ca) * p.k;
            u64 thr = kKeyEmpty;
            for (int base = 0; base < total; base += 128) {
                u64 key[4];
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int i = base + b * 32 + lane;
                    key[b] = i < total ? __ldcg(Pg + i) : kKeyEmpty;
                }
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    unsigned m = __ballot_sync(kFull, key[b] <= bound && key[b] < thr);
                    while (m) {
                        const int j = __ffs(m) - 1;
                        m &= m - 1;
                        list_insert(M, __shfl_sync(kFull, key[b], j), p.k, lane);
                    }
                    thr = __shfl_sync(kFull, M, p.k - 1);
                }
            }
        }
        mlist[warp * 32 + lane] = M;
        __syncthreads();
        if (active && g == 0 && qi < p.nq) {
            for (int h = 1; h < G; ++h) list_merge_keys<false>(M, &mlist[(warp + h) * 32], p.k, p.k, lane);
            if (lane < p.k) {
                const size_t o = ((size_t)qi * p.n_sub + sub) * p.k + lane;
                if (M == kKeyEmpty) {
                    p.idx[o] = -1;
                    p.dist[o] = __int_as_float(0x7f800000);
                } else {
                    const uint32_t r = key_row(M);
                    p.idx[o] = p.perm ? (int64_t)p.perm[r] : (int64_t)r;
                    p.dist[o] = key_dist(M);
                }
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) p.counters[qblock] = 0u;
}

// Launch shape. With few frames per block (QB <= 4) the warps are
// latency-bound, so each keeps two stages in flight, even at half the warps;
// otherwise (or when that leaves fewer than 6 warps) the most warps that fit
// win, down to one stage each.
ScanConfig choose_config(const lhr_db* db, int nq) {
    ScanConfig c{};
    const int d4 = db->dim / 4;
    c.cpl = d4 <= 32 ? 1 : (d4 <= 64 ? 2 : 4);
    const int qb_max = 16 / c.cpl;
    int qb = 4;
    while (qb < nq && qb < qb_max) qb *= 2;
    c.qb = qb;
    const size_t stage_bytes = (size_t)kRPS * db->dim * sizeof(float);
    const size_t qs_bytes = (size_t)(qb + 1) * db->dim * sizeof(float);  // frames + weights
    auto smem_for = [&](int w, int per) {
        const int ns = per * w;
        return ns * stage_bytes + qs_bytes + 2 * ns * sizeof(u64) + (size_t)w * qb * 32 * sizeof(u64) +
               qb * sizeof(unsigned) + 16;
    };
    const size_t cap = (size_t)kMaxSmem - 1024;
    for (int pass = qb <= 4 ? 0 : 1; pass < 2; ++pass) {
        const int w_min = pass == 0 ? 6 : 1, per_min = pass == 0 ? 2 : 1;
        for (int w = kMaxWarps; w >= w_min; --w)
            for (int per = 3; per >= per_min; --per)
                if (smem_for(w, per) <= cap) {
                    c.warps = w;
                    c.stages = per * w;
                    c.smem = smem_for(w, per);
                    return c;
                }
    }
    c.warps = 1;
    c.stages = 1;
    c.smem = smem_for(1, 1);
    return c;
}

// ------------------------------------------------------------------ pilot
// Distances of every pilot-sample row to every frame (direct-form FP32, the
// arithmetic of the scan's exact step up to the summation order), folded into
// the bucket minima read by pilot_bound:
// bmin[(f * n_sub + sub_p[j]) * 128 + j % 128] (float bits, preset to ~0u).
// A warp takes 4 rows and 8 frames per round: 32 partial sums per lane, one
// butterfly transpose-reduce, and lane l then holds (row l / 8, frame l % 8).
// With many frames the grid's y splits them into slices of kPilotFrameSlice.
constexpr int kPilotFrameSlice = 64;

template <int CPL>
__global__ void __launch_bounds__(256) pilot_kernel(const float* Xp, const int32_t* sub_p, int64_t np, int D,
                                                    const float* Q, int nq, int n_sub, const float* w,
                                                    unsigned* bmin) {
    const int lane = threadIdx.x % 32;
    const int D4 = D / 4;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int64_t nw = (int64_t)gridDim.x * blockDim.x / 32;
    for (int64_t r0 = gw * 4; r0 < np; r0 += nw * 4) {
        float4 x[4][CPL];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float4* xr = reinterpret_cast<const float4*>(Xp + (r0 + i) * D);
#pragma unroll
            for (int j = 0; j < CPL; ++j) {
                const int c = lane + 32 * j;
                x[i][j] = (r0 + i < np && c < D4) ? __ldg(xr + c) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        const int64_t r = r0 + lane / 8;
        const int sub = r < np ? __ldg(sub_p + r) : 0;
        float4 wv[CPL];
#pragma unroll
        for (int j = 0; j < CPL; ++j) {
            const int c = lane + 32 * j;
            wv[j] = (w != nullptr && c < D4) ? __ldg(reinterpret_cast<const float4*>(w) + c)
                                             : make_float4(1.f, 1.f, 1.f, 1.f);
        }
        // this CTA's frames: a slice of kPilotFrameSlice (grid y), all of them
        // when the grid has one slice
        const int fb0 = blockIdx.y * kPilotFrameSlice, fb1 = gridDim.y == 1 ? nq : min(nq, fb0 + kPilotFrameSlice);
        for (int f0 = fb0; f0 < fb1; f0 += 8) {
            float part[32];
#pragma unroll
            for (int f = 0; f < 8; ++f) {
                float4 qv[CPL];
                const float4* qr = reinterpret_cast<const float4*>(Q + (size_t)min(f0 + f, nq - 1) * D);
#pragma unroll
                for (int j = 0; j < CPL; ++j) {
                    const int c = lane + 32 * j;
                    qv[j] = c < D4 ? __ldg(qr + c) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    float2 acc = f2(0.f, 0.f);
#pragma unroll
                    for (int j = 0; j < CPL; ++j) {
                        const float2 d0 = __ffma2_rn(f2(x[i][j].x, x[i][j].y), f2(-1.f, -1.f), f2(qv[j].x, qv[j].y));
                        const float2 d1 = __ffma2_rn(f2(x[i][j].z, x[i][j].w), f2(-1.f, -1.f), f2(qv[j].z, qv[j].w));
                        acc = __ffma2_rn(__fmul2_rn(d0, f2(wv[j].x, wv[j].y)), d0, acc);
                        acc = __ffma2_rn(__fmul2_rn(d1, f2(wv[j].z, wv[j].w)), d1, acc);
                    }
                    part[i * 8 + f] = acc.x + acc.y;
                }
            }
#pragma unroll
            for (int st = 16; st >= 1; st >>= 1) {
                const bool upper = (lane & st) != 0;
#pragma unroll
                for (int v = 0; v < st; ++v) {
                    const float send = upper ? part[v] : part[v + st];
                    const float keep = upper ? part[v + st] : part[v];
                    part[v] = keep + __shfl_xor_sync(kFull, send, st);
                }
            }
            const int f = f0 + lane % 8;
            if (r < np && f < fb1)
                atomicMin(bmin + ((size_t)f * n_sub + sub) * kPilotBuckets + (r % kPilotBuckets),
                          __float_as_uint(part[0]));
        }
    }
}

// Weighted row norms sum_j w_j x_j^2 (internal order) and their maximum (float
// bits, atomicMax; the values are >= 0); one warp per row. Block 0 also checks
// the weights: a negative or non-finite one records LHR_ERR_INVALID_ARG.
__global__ void __launch_bounds__(256) wnorm_kernel(const float* X, int64_t n, int D, const float* w, float* xnw,
                                                    unsigned* max_bits, int* err) {
    const int lane = threadIdx.x % 32;
    const int D4 = D / 4;
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < D; i += blockDim.x)
            if (!(w[i] >= 0.f && w[i] < __int_as_float(0x7f800000))) record_error(err, kErrInvalidArg);
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int64_t nw = (int64_t)gridDim.x * blockDim.x / 32;
    unsigned mx = 0u;
    for (int64_t r = gw; r < n; r += nw) {
        const float4* xr = reinterpret_cast<const float4*>(X + r * D);
        float a = 0.f;
        for (int c = lane; c < D4; c += 32) {
            const float4 x = __ldg(xr + c), wv = __ldg(reinterpret_cast<const float4*>(w) + c);
            a = fmaf(wv.x * x.x, x.x, a);
            a = fmaf(wv.y * x.y, x.y, a);
            a = fmaf(wv.z * x.z, x.z, a);
            a = fmaf(wv.w * x.w, x.w, a);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(kFull, a, o);
        if (lane == 0) xnw[r] = a;
        mx = max(mx, __float_as_uint(a));
    }
    if (lane == 0 && mx) atomicMax(max_bits, mx);
}

// ------------------------------------------------------------------ small databases
// Databases of at most kSmallRows rows: one CTA per (frame, subspace) scores
// every row of the subspace (a warp per row, four rows in flight, the scan's
// exact direct-form arithmetic, so the distances are the same to the bit),
// keeps the keys in shared memory and selects the top k by radix select; no
// per-warp lists, no merge tail.
constexpr int kSmallThreads = 512;
constexpr int64_t kSmallRows = 16384;

template <int CPL>
__global__ void __launch_bounds__(kSmallThreads) small_topk_kernel(const float* X, int D, const float* Q,
                                                                   const float* w, const int4* chunks,
                                                                   const int32_t* chunk_off, int n_sub,
                                                                   const int32_t* perm, int k, int64_t* idx,
                                                                   float* dist) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int f = blockIdx.x, sub = blockIdx.y, t = threadIdx.x, warp = t / 32, lane = t % 32;
    const int D4 = D / 4;
    const int c0 = chunk_off[sub], c1 = chunk_off[sub + 1];
    const int r0 = c1 > c0 ? chunks[c0].x : 0, r1 = c1 > c0 ? chunks[c1 - 1].y : 0;
    const int cnt = r1 - r0;
    float* qs = reinterpret_cast<float*>(smem);          // D
    float* ws = qs + D;                                   // D
    unsigned* hs = reinterpret_cast<unsigned*>(ws + D);   // kBins
    unsigned* res = hs + sel::kBins;                      // 4
    unsigned* tmp = res + 4;                              // kSmallThreads / 32
    u64* mm = reinterpret_cast<u64*>(tmp + kSmallThreads / 32);  // 2 x 16 (min, max per warp)
    u64* outk = mm + 32;                                  // 32
    u64* keys = outk + 32;                                // cnt
    for (int i = t; i < D; i += kSmallThreads) {
        qs[i] = Q[(size_t)f * D + i];
        ws[i] = w != nullptr ? w[i] : 1.f;
    }
    __syncthreads();
    const float4* qr = reinterpret_cast<const float4*>(qs);
    const float4* wr = reinterpret_cast<const float4*>(ws);
    u64 lo = ~0ull, hi = 0ull;
    for (int i0 = warp * 4; i0 < cnt; i0 += (kSmallThreads / 32) * 4) {
        float4 x[4][CPL];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float4* xr = reinterpret_cast<const float4*>(X + (size_t)(r0 + min(i0 + u, cnt - 1)) * D);
#pragma unroll
            for (int jj = 0; jj < CPL; ++jj) {
                const int c = lane + 32 * jj;
                x[u][jj] = c < D4 ? __ldg(xr + c) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            float2 acc = f2(0.f, 0.f);
#pragma unroll
            for (int jj = 0; jj < CPL; ++jj) {
                const int c = lane + 32 * jj;
                if (c < D4) {
                    const float4 qv = qr[c], wv = wr[c];
                    const float2 d0 = __ffma2_rn(f2(x[u][jj].x, x[u][jj].y), f2(-1.f, -1.f), f2(qv.x, qv.y));
                    const float2 d1 = __ffma2_rn(f2(x[u][jj].z, x[u][jj].w), f2(-1.f, -1.f), f2(qv.z, qv.w));
                    acc = __ffma2_rn(__fmul2_rn(d0, f2(wv.x, wv.y)), d0, acc);
                    acc = __ffma2_rn(__fmul2_rn(d1, f2(wv.z, wv.w)), d1, acc);
                }
            }
            float de = acc.x + acc.y;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) de += __shfl_xor_sync(kFull, de, o);
            if (i0 + u < cnt) {
                const u64 key = make_key(de, (uint32_t)(r0 + i0 + u));
                if (lane == 0) keys[i0 + u] = key;
                lo = key < lo ? key : lo;
                hi = key > hi ? key : hi;
            }
        }
    }
    if (lane == 0) {
        mm[warp] = lo;
        mm[16 + warp] = hi;
    }
    __syncthreads();
    const int kk = min(k, cnt);
    u64 kth = ~0ull;
    if (cnt > kk) {
        lo = ~0ull;
        hi = 0ull;
        for (int i = 0; i < kSmallThreads / 32; ++i) {
            lo = mm[i] < lo ? mm[i] : lo;
            hi = mm[16 + i] > hi ? mm[16 + i] : hi;
        }
        kth = sel::block_kth_key<kSmallThreads>(keys, (unsigned)cnt, (unsigned)kk, lo, hi, hs, res, tmp);
    }
    if (t == 0) res[3] = 0u;
    __syncthreads();
    for (int i = t; i < cnt; i += kSmallThreads)
        if (keys[i] <= kth) {
            const unsigned pos = atomicAdd(&res[3], 1u);
            if (pos < 32u) outk[pos] = keys[i];
        }
    __syncthreads();
    if (t < 32) {
        const unsigned n_out = min(res[3], 32u);
        u64 v = (unsigned)lane < n_out ? outk[lane] : kKeyEmpty;
#pragma unroll
        for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                const u64 o = __shfl_xor_sync(kFull, v, stride);
                const bool keep_min = ((lane & stride) == 0) == ((lane & size) == 0);
                v = keep_min ? (o < v ? o : v) : (o > v ? o : v);
            }
        }
        if (lane < k) {
            const size_t o = ((size_t)f * n_sub + sub) * k + lane;
            if (v == kKeyEmpty) {
                idx[o] = -1;
                dist[o] = __int_as_float(0x7f800000);
            } else {
                const uint32_t r = key_row(v);
                idx[o] = perm ? (int64_t)perm[r] : (int64_t)r;
                dist[o] = key_dist(v);
            }
        }
    }
}

cudaError_t launch_small(const lhr_db* db, const float* q, int nq, int k, const float* w, int64_t* idx, float* dist,
                         cudaStream_t stream) {
    const int d4 = db->dim / 4;
    const int cpl = d4 <= 32 ? 1 : (d4 <= 64 ? 2 : 4);
    int64_t rows_max = 0;
    for (int64_t r : db->sub_rows_h) rows_max = std::max(rows_max, r);
    const size_t smem = (size_t)(2 * db->dim + sel::kBins + 4 + kSmallThreads / 32) * sizeof(float) +
                        (64 + (size_t)std::max<int64_t>(rows_max, 1)) * sizeof(u64) + 16;
    const dim3 grid(nq, db->n_sub);
    ProfScope ps("small_topk_kernel", stream);
#define LHR_SMALL(C)                                                                                                  \
    do {                                                                                                              \
        cudaError_t e = cudaFuncSetAttribute(small_topk_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e != cudaSuccess) return e;                                                                               \
        small_topk_kernel<C><<<grid, kSmallThreads, smem, stream>>>(db->X, db->dim, q, w, db->chunks, db->chunk_off,  \
                                                                    db->n_sub, db->perm, k, idx, dist);               \
    } while (0)
    if (cpl == 1) LHR_SMALL(1);
    else if (cpl == 2) LHR_SMALL(2);
    else LHR_SMALL(4);
#undef LHR_SMALL
    return cudaGetLastError();
}

__global__ void check_weights_kernel(const float* w, int D, int* err) {
    for (int i = threadIdx.x; i < D; i += blockDim.x)
        if (!(w[i] >= 0.f && w[i] < __int_as_float(0x7f800000))) record_error(err, kErrInvalidArg);
}

template <int QB, int CPL>
cudaError_t launch_t(const ScanConfig& c, const ScanParams& p, int nqb, const char* label, cudaStream_t stream) {
    auto kern = scan_topk_kernel<QB, CPL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem);
    if (e != cudaSuccess) return e;
    if (p.nchunks > 65535) return cudaErrorInvalidValue;
    dim3 grid(nqb, p.nchunks);
    ProfScope ps(label, stream);
    kern<<<grid, (c.warps + 1) * 32, c.smem, stream>>>(p);
    return cudaGetLastError();
}

}  // namespace

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

namespace {

// The rows one scan pass streams: the database, or its pilot sample.
struct ScanSrc {
    const float* X;
    const float* xnorm;
    const int4* chunks;
    int nchunks;
    const int32_t* chunk_off;
    const int32_t* perm;  // nullable
};

// 2 (gamma_{D+4} + 3u) with u = 2^-24 and gamma_m = m u / (1 - m u), slightly
// rounded up (the weighted form rounds w q and w (q - x) once more): times
// (max ||x|| + ||q||)^2, it bounds the difference between the expanded-form
// distance and the exact direct form.
float scan_margin_scale(int dim) {
    const double u = 1.0 / 16777216.0;
    const double gamma = (dim + 4) * u / (1.0 - (dim + 4) * u);
    return (float)(2.0 * (gamma + 3.0 * u) * 1.0001);
}

size_t pass_bytes(const ScanConfig& c, int nchunks, int n_sub, int nq, int k) {
    const size_t nqb = (nq + c.qb - 1) / c.qb;
    return align256(nqb * c.qb * (size_t)nchunks * k * sizeof(u64)) + align256(nqb * sizeof(unsigned)) +
           align256(nqb * c.qb * (size_t)n_sub * sizeof(unsigned));
}

constexpr int kPilotMaxFrames = 4096;  // larger requests scan without the pilot

bool use_pilot(const lhr_db* db, int nq) { return db->Xp != nullptr && nq <= kPilotMaxFrames; }

size_t pilot_bytes(const lhr_db* db, int nq) { return align256((size_t)nq * db->n_sub * kPilotBuckets * sizeof(unsigned)); }

cudaError_t launch_pilot(const lhr_db* db, const float* q, int nq, const float* w, void* scratch,
                         unsigned** bmin_out, cudaStream_t stream) {
    unsigned* bmin = reinterpret_cast<unsigned*>(scratch);
    cudaError_t e = cudaMemsetAsync(bmin, 0xff, (size_t)nq * db->n_sub * kPilotBuckets * sizeof(unsigned), stream);
    if (e != cudaSuccess) return e;
    const int d4 = db->dim / 4;
    const int cpl = d4 <= 32 ? 1 : (d4 <= 64 ? 2 : 4);
    const int slices = nq > 2 * kPilotFrameSlice ? (nq + kPilotFrameSlice - 1) / kPilotFrameSlice : 1;
    const dim3 grid((unsigned)std::min<int64_t>((db->n_pilot + 31) / 32, (int64_t)db->sms * 8), (unsigned)slices);
    {
        ProfScope ps("scan_pilot", stream);
        if (cpl == 1)
            pilot_kernel<1><<<grid, 256, 0, stream>>>(db->Xp, db->sub_p, db->n_pilot, db->dim, q, nq, db->n_sub, w, bmin);
        else if (cpl == 2)
            pilot_kernel<2><<<grid, 256, 0, stream>>>(db->Xp, db->sub_p, db->n_pilot, db->dim, q, nq, db->n_sub, w, bmin);
        else
            pilot_kernel<4><<<grid, 256, 0, stream>>>(db->Xp, db->sub_p, db->n_pilot, db->dim, q, nq, db->n_sub, w, bmin);
    }
    *bmin_out = bmin;
    return cudaGetLastError();
}

// Weighted scans: the weights, the weighted row norms and their device max.
struct ScanWeights {
    const float* w;
    const float* xnw;
    const float* xmax_w;
};

cudaError_t scan_pass(const lhr_db* db, const ScanSrc& src, const char* label, const float* q, int nq, int k,
                      const unsigned* bmin, const ScanWeights* wt, int64_t* idx, float* dist, void* scratch,
                      cudaStream_t stream) {
    const ScanConfig c = choose_config(db, nq);
    const int nqb = (nq + c.qb - 1) / c.qb;
    ScanParams p{};
    p.X = src.X;
    p.xnorm = src.xnorm;
    p.D = db->dim;
    p.chunks = src.chunks;
    p.nchunks = src.nchunks;
    p.chunk_off = src.chunk_off;
    p.n_sub = db->n_sub;
    p.perm = src.perm;
    p.Q = q;
    p.nq = nq;
    p.k = k;
    p.stages = c.stages;
    p.bmin = bmin;
    if (wt != nullptr) {
        p.w = wt->w;
        p.xnorm = wt->xnw;
        p.xmax_w = wt->xmax_w;
    }
    p.margin_scale = scan_margin_scale(db->dim);
    // max ||x|| over the whole database bounds the sample's too
    p.xmax = (float)(sqrt((double)db->xnorm_max) * 1.0001);
    p.partial = reinterpret_cast<u64*>(scratch);
    const size_t part_bytes = align256((size_t)nqb * c.qb * src.nchunks * k * sizeof(u64));
    p.counters = reinterpret_cast<unsigned*>(reinterpret_cast<unsigned char*>(scratch) + part_bytes);
    p.gthr = reinterpret_cast<unsigned*>(reinterpret_cast<unsigned char*>(scratch) + part_bytes +
                                         align256(nqb * sizeof(unsigned)));
    p.idx = idx;
    p.dist = dist;
    p.err = db->err;
    cudaError_t e = cudaMemsetAsync(p.counters, 0, nqb * sizeof(unsigned), stream);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(p.gthr, 0xff, (size_t)nqb * c.qb * db->n_sub * sizeof(unsigned), stream);
    if (e != cudaSuccess) return e;
    switch (c.cpl * 100 + c.qb) {
        case 104: return launch_t<4, 1>(c, p, nqb, label, stream);
        case 108: return launch_t<8, 1>(c, p, nqb, label, stream);
        case 116: return launch_t<16, 1>(c, p, nqb, label, stream);
        case 204: return launch_t<4, 2>(c, p, nqb, label, stream);
        case 208: return launch_t<8, 2>(c, p, nqb, label, stream);
        case 404: return launch_t<4, 4>(c, p, nqb, label, stream);
        default: return cudaErrorInvalidConfiguration;
    }
}

}  // namespace

size_t scan_scratch_bytes(const lhr_db* db, int nq, int k, bool pilot) {
    if (pilot && many_eligible(db, nq, k)) return many_scratch_bytes(db, nq);
    const ScanConfig c = choose_config(db, nq);
    const size_t main = pass_bytes(c, db->nchunks, db->n_sub, nq, k);
    return pilot && use_pilot(db, nq) ? main + pilot_bytes(db, nq) : main;
}

namespace {

// With a pilot sample (every 64th row): a bound on each frame's k-th distance
// per subspace, taken from the sample (pilot_bound), seeds the full scan's
// thresholds, so only rows that can still reach a top k are ever recomputed
// and inserted. Every key of the final top k is <= that bound: the k sample
// rows reaching it are database rows the full scan meets again.
cudaError_t scan_with_pilot(const lhr_db* db, const float* q, int nq, int k, const ScanWeights* wt, int64_t* idx,
                            float* dist, void* scratch, bool pilot, cudaStream_t stream) {
    const ScanSrc full{db->X, db->xnorm, db->chunks, db->nchunks, db->chunk_off, db->perm};
    unsigned* bmin = nullptr;
    if (pilot && many_eligible(db, nq, k)) {
        // many frames: the tensor-core filter and the exact re-score (many.cu)
        return launch_many(db, q, nq, k, wt ? wt->w : nullptr, wt ? wt->xnw : db->xnorm, wt ? wt->xmax_w : nullptr,
                           scan_margin_scale(db->dim), idx, dist, scratch, stream);
    }
    if (pilot && use_pilot(db, nq)) {
        const ScanConfig c = choose_config(db, nq);
        unsigned char* ps = reinterpret_cast<unsigned char*>(scratch) + pass_bytes(c, db->nchunks, db->n_sub, nq, k);
        cudaError_t e = launch_pilot(db, q, nq, wt ? wt->w : nullptr, ps, &bmin, stream);
        if (e != cudaSuccess) return e;
    }
    return scan_pass(db, full, "scan_topk_kernel", q, nq, k, bmin, wt, idx, dist, scratch, stream);
}

}  // namespace

cudaError_t launch_scan(const lhr_db* db, const float* q, int nq, int k, int64_t* idx, float* dist, void* scratch,
                        bool pilot, cudaStream_t stream) {
    if (db->n <= kSmallRows) return launch_small(db, q, nq, k, nullptr, idx, dist, stream);
    return scan_with_pilot(db, q, nq, k, nullptr, idx, dist, scratch, pilot, stream);
}

size_t scan_weighted_scratch_bytes(const lhr_db* db, int nq, int k) {
    return align256(((size_t)db->n + 1) * sizeof(float)) + scan_scratch_bytes(db, nq, k, true);
}

cudaError_t launch_scan_weighted(const lhr_db* db, const float* q, int nq, int k, const float* w, int64_t* idx,
                                 float* dist, void* scratch, cudaStream_t stream) {
    if (db->n <= kSmallRows) {
        // the weights are checked here as the large path's norm kernel does
        cudaError_t e = launch_small(db, q, nq, k, w, idx, dist, stream);
        if (e != cudaSuccess) return e;
        check_weights_kernel<<<1, 256, 0, stream>>>(w, db->dim, db->err);
        return cudaGetLastError();
    }
    float* xnw = reinterpret_cast<float*>(scratch);
    float* xmax_w = xnw + db->n;
    void* rest = reinterpret_cast<unsigned char*>(scratch) + align256(((size_t)db->n + 1) * sizeof(float));
    cudaError_t e = cudaMemsetAsync(xmax_w, 0, sizeof(float), stream);
    if (e != cudaSuccess) return e;
    {
        ProfScope ps("wnorm_kernel", stream);
        const int grid = (int)std::min<int64_t>((db->n + 7) / 8, (int64_t)db->sms * 16);
        wnorm_kernel<<<grid, 256, 0, stream>>>(db->X, db->n, db->dim, w, xnw, reinterpret_cast<unsigned*>(xmax_w),
                                               db->err);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const ScanWeights wt{w, xnw, xmax_w};
    return scan_with_pilot(db, q, nq, k, &wt, idx, dist, rest, true, stream);
}

}  // namespace lhr

// ---------------------------------------------------------------------------
// Allocation-free variant of the exhaustive scan (lhr_query_static).
//
// Its scratch (per-chunk candidate lists and per-query-block tickets) lives in
// this fixed device array instead of memory allocated per call. The array is
// part of the library's device code, so every GPU that loads the library
// holds these bytes until the process exits. All calls share it.
static constexpr size_t kStaticScratchBytes = (size_t)4 << 20;  // 4 MiB
static __device__ __align__(256) unsigned char g_scan_static_scratch[kStaticScratchBytes];

namespace {

// Device address of g_scan_static_scratch, looked up once per device. In host
// code the array's name only stands in for the symbol: it is not a device
// address and must never be handed to a kernel.
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_addr[kMaxDevices] = {};

cudaError_t static_scratch_address(int dev, void** out) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (g_static_addr[dev] == nullptr) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scan_static_scratch);  // `dev` is current here
        if (e != cudaSuccess) return e;
        g_static_addr[dev] = p;
    }
    *out = g_static_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" lhr_status lhr_query_static(const lhr_db* db, const float* q, int32_t nq, int32_t k, int64_t* idx,
                                       float* dist, void* cuda_stream) {
    using namespace lhr;
    if (!db) return fail(LHR_ERR_INVALID_ARG, "db is NULL");
    if (!q || !idx || !dist) return fail(LHR_ERR_INVALID_ARG, "q, idx and dist must be non-NULL");
    if (reinterpret_cast<uintptr_t>(q) % 16) return fail(LHR_ERR_INVALID_ARG, "q must be 16-byte aligned");
    if (nq < 1) return fail(LHR_ERR_INVALID_ARG, "nq must be >= 1");
    if (k < 1 || k > 32) return fail(LHR_ERR_INVALID_ARG, "k must be in [1, 32]");
    const size_t need = scan_scratch_bytes(db, nq, k, false);
    if (need > kStaticScratchBytes)
        return fail(LHR_ERR_INVALID_ARG, "lhr_query_static: this request needs " + std::to_string(need) +
                                             " bytes of scratch, more than the fixed " +
                                             std::to_string(kStaticScratchBytes) +
                                             "-byte device array; use fewer query frames or lhr_query");
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return fail(LHR_ERR_CUDA, "cudaGetDevice failed");
    if (prev != db->device && cudaSetDevice(db->device) != cudaSuccess)
        return fail(LHR_ERR_CUDA, "cudaSetDevice failed");
    void* scratch = nullptr;
    cudaError_t e = static_scratch_address(db->device, &scratch);
    if (e == cudaSuccess)
        e = launch_scan(db, q, nq, k, idx, dist, scratch, false, reinterpret_cast<cudaStream_t>(cuda_stream));
    if (prev != db->device) cudaSetDevice(prev);
    if (e != cudaSuccess) return cuda_fail(e, "lhr_query_static");
    return LHR_OK;
}
