// Algorithm 2 (§3.2) for one window by a single warp -- shared by the
// aggregation kernel and the fused coarse-to-fine kernel. See aggregate.cu for
// the steps, tie rules and integer tests.
#pragma once

#include <math.h>

#include "common.cuh"
#include "internal.h"

namespace lhr {
namespace agg {

struct AggParams {
    AggArgs a;
    const int32_t* tile;  // n x 2
    const double* xy;     // n x 2
    int64_t n;
    long long rlim;       // floor(sqrt(r2max)): larger |dx| or |dy| is outside the circle
    int* err;
    const u64* tile_keys;  // nullable: tile key of each candidate slot (as a.idx), gathered by the producer
};

__device__ __forceinline__ u64 tile_key(int tx, int ty) {
    return ((u64)((uint32_t)ty ^ 0x80000000u) << 32) | (u64)((uint32_t)tx ^ 0x80000000u);
}
__device__ __forceinline__ int key_tx(u64 k) { return (int)((uint32_t)k ^ 0x80000000u); }
__device__ __forceinline__ int key_ty(u64 k) { return (int)((uint32_t)(k >> 32) ^ 0x80000000u); }

constexpr int kWarpCand = 1024;  // windows with at most this many candidate slots take the warp path

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ void write_invalid(const AggArgs& a, int w) {
    a.status[w] = kErrInvalidArg;
    a.xy_out[2 * w] = a.xy_out[2 * w + 1] = __longlong_as_double(0x7ff8000000000000ll);
}

// Sorts keys[0, 32 E) ascending in registers: element i = e * 32 + lane lives
// in v[e] (a bitonic network; strides below 32 cross lanes by shuffles, the
// others stay in the lane).
template <int E>
__device__ __forceinline__ void warp_sort_regs(u64 (&v)[E], int lane) {
#pragma unroll
    for (int size = 2; size <= 32 * E; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= 32) {
                const int es = stride / 32;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    if (e & es) continue;
                    const bool asc = ((e * 32) & size) == 0;
                    const u64 a = v[e], b = v[e + es];
                    const u64 lo = a < b ? a : b, hi = a < b ? b : a;
                    v[e] = asc ? lo : hi;
                    v[e + es] = asc ? hi : lo;
                }
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const u64 o = __shfl_xor_sync(kFull, v[e], stride);
                    const bool asc = ((e * 32 + lane) & size) == 0;
                    const bool keep_min = ((lane & stride) == 0) == asc;
                    v[e] = keep_min ? (o < v[e] ? o : v[e]) : (o > v[e] ? o : v[e]);
                }
            }
        }
    }
}

// keys[0, 32 E) sorted in place through registers (entries >= n read as empty).
template <int E>
__device__ __noinline__ void warp_sort_smem(u64* keys, int n, int lane) {
    u64 v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = e * 32 + lane < n ? keys[e * 32 + lane] : kKeyEmpty;
    warp_sort_regs<E>(v, lane);
#pragma unroll
    for (int e = 0; e < E; ++e) keys[e * 32 + lane] = v[e];
}

// Initialization and binning of a window of at most 32 E candidate slots in
// registers: every slot's row, distance and tile key loaded in one round,
// rows and distances compacted (padding rows skipped) into cand_rows /
// cand_d, and the tile keys sorted in registers with the padding slots' empty
// keys last, written to keys[0, 32 E). Returns the candidate count C.
template <int E>
__device__ __forceinline__ int init_sorted(const AggParams& p, long long b0, long long total, u64* keys,
                                           int* cand_rows, float* cand_d, int lane, bool sort) {
    const AggArgs& a = p.a;
    const unsigned below = (1u << lane) - 1u;
    int64_t r[E];
    float d[E];
    u64 v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const long long i = e * 32 + lane;
        r[e] = i < total ? __ldcg(a.idx + b0 + i) : -1;  // may come from another CTA of the launch
        d[e] = (i < total && a.dist != nullptr) ? __ldcg(a.dist + b0 + i) : 0.f;
        v[e] = (i < total && p.tile_keys != nullptr) ? __ldcg(p.tile_keys + b0 + i) : kKeyEmpty;
    }
    int C = 0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const bool bad = r[e] >= p.n;
        if (bad) record_error(p.err, kErrInvalidArg);
        const bool take = r[e] >= 0 && !bad;
        const unsigned m = __ballot_sync(kFull, take);
        const int pos = C + __popc(m & below);
        if (take) {
            cand_rows[pos] = (int)r[e];
            cand_d[pos] = d[e];
            if (p.tile_keys == nullptr) v[e] = tile_key(p.tile[2 * r[e]], p.tile[2 * r[e] + 1]);
        } else {
            v[e] = kKeyEmpty;
        }
        C += __popc(m);
    }
    if (sort) {
        warp_sort_regs<E>(v, lane);
#pragma unroll
        for (int e = 0; e < E; ++e) keys[e * 32 + lane] = v[e];
    }
    return C;
}

// Tile modes (0, 1) of Algorithm 2 for one window of at most 128 candidate
// slots, by one warp, without sorting (the short form for latency-bound
// callers): each candidate's tile key goes into a 256-slot open-addressing
// table in shared memory (one compare-and-swap, linear probing) whose counts
// are its bins; lane l keeps table slots l + 32 j, j < 8, in registers, and a
// draw takes the best untaken tile -- count descending, then key ascending,
// i.e. ty, tx ascending -- by warp reductions (redux.sync), not shuffles.
// The same draws, circle test, tie rules and outputs as aggregate_warp.
// `tab` holds 256 keys, `tcnt` 256 counts, `cand_rows` 128 rows.
__device__ __forceinline__ unsigned tab_hash(u64 k) {
    return (((unsigned)k * 0x9E3779B1u) ^ ((unsigned)(k >> 32) * 0x85EBCA77u)) >> 24;
}

__device__ inline void aggregate_warp_small(const AggParams& p, int w, long long b0, long long total, u64* tab,
                                            unsigned* tcnt, int* cand_rows) {
    const AggArgs& a = p.a;
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        tab[j * 32 + lane] = kKeyEmpty;
        tcnt[j * 32 + lane] = 0u;
    }
    // initialization: rows -> tiles, padding rows skipped, compacted in order
    int64_t r[4];
    u64 v[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const long long i = e * 32 + lane;
        r[e] = i < total ? __ldcg(a.idx + b0 + i) : -1;  // may come from another CTA of the launch
        v[e] = (i < total && p.tile_keys != nullptr) ? __ldcg(p.tile_keys + b0 + i) : kKeyEmpty;
    }
    __syncwarp();
    int C = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const bool bad = r[e] >= p.n;
        if (bad) record_error(p.err, kErrInvalidArg);
        const bool take = r[e] >= 0 && !bad;
        const unsigned m = __ballot_sync(kFull, take);
        if (take) {
            cand_rows[C + __popc(m & below)] = (int)r[e];
            if (p.tile_keys == nullptr) v[e] = tile_key(p.tile[2 * r[e]], p.tile[2 * r[e] + 1]);
            unsigned slot = tab_hash(v[e]);
            for (int probe = 0; probe < 256; ++probe) {  // at most 128 keys in 256 slots: a slot is found
                const u64 old = atomicCAS(reinterpret_cast<unsigned long long*>(tab + slot), kKeyEmpty, v[e]);
                if (old == kKeyEmpty || old == v[e]) {
                    atomicAdd(tcnt + slot, 1u);
                    break;
                }
                slot = (slot + 1u) & 255u;
            }
        }
        C += __popc(m);
    }
    __syncwarp();
    if (C == 0) {
        if (lane == 0) write_invalid(a, w);
        return;
    }
    u64 kk[8];
    unsigned cc[8], occupied = 0u;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        kk[j] = tab[j * 32 + lane];
        cc[j] = tcnt[j * 32 + lane];
        occupied += kk[j] != kKeyEmpty ? 1u : 0u;
    }
    const int U = (int)__reduce_add_sync(kFull, occupied);
    const double tm = a.tile_m;
    int status = 0, win_tx = 0, win_ty = 0, first_tx = 0, first_ty = 0;
    bool found = false;
    unsigned taken = 0u;
    const int ntop = min(a.top_c, U);
    for (int rr = 0; rr < ntop; ++rr) {
        unsigned bc = 0u;
        u64 bk = kKeyEmpty;
        int bj = -1;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const bool live = kk[j] != kKeyEmpty && !((taken >> j) & 1u);
            if (live && (cc[j] > bc || (cc[j] == bc && kk[j] < bk))) {
                bc = cc[j];
                bk = kk[j];
                bj = j;
            }
        }
        const unsigned mc = __reduce_max_sync(kFull, bc);
        const unsigned hi = __reduce_min_sync(kFull, bc == mc ? (unsigned)(bk >> 32) : 0xffffffffu);
        const unsigned lo =
            __reduce_min_sync(kFull, (bc == mc && (unsigned)(bk >> 32) == hi) ? (unsigned)bk : 0xffffffffu);
        const u64 ks = ((u64)hi << 32) | (u64)lo;
        if (bj >= 0 && bk == ks) taken |= 1u << bj;  // the table's keys are distinct: one lane holds ks
        const int tx0 = key_tx(ks), ty0 = key_ty(ks);
        if (rr == 0) {
            first_tx = tx0;
            first_ty = ty0;
        }
        unsigned circ = 0u;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (kk[j] == kKeyEmpty) continue;
            const long long dx = (long long)key_tx(kk[j]) - tx0, dy = (long long)key_ty(kk[j]) - ty0;
            if (dx > p.rlim || dx < -p.rlim || dy > p.rlim || dy < -p.rlim) continue;
            if (dx * dx + dy * dy <= a.r2max) circ += cc[j];
        }
        circ = __reduce_add_sync(kFull, circ);
        if (100ll * (long long)circ > (long long)a.toler_pct * (long long)C) {
            win_tx = tx0;
            win_ty = ty0;
            found = true;
            break;
        }
    }
    if (!found) {
        win_tx = first_tx;
        win_ty = first_ty;
        status = 1;
    }
    double ox, oy;
    if (a.mode == 0) {
        ox = ((double)win_tx + 0.5) * tm;
        oy = ((double)win_ty + 0.5) * tm;
    } else {
        double sx = 0.0, sy = 0.0;
        long long m = 0;
        for (int i = lane; i < C; i += 32) {
            const int rw = cand_rows[i];
            const long long dx = (long long)p.tile[2 * rw] - win_tx, dy = (long long)p.tile[2 * rw + 1] - win_ty;
            if (dx > p.rlim || dx < -p.rlim || dy > p.rlim || dy < -p.rlim) continue;
            if (dx * dx + dy * dy <= a.r2max) {
                sx += p.xy[2 * rw];
                sy += p.xy[2 * rw + 1];
                ++m;
            }
        }
        sx = warp_sum(sx);
        sy = warp_sum(sy);
        m = warp_sum(m);
        ox = sx / (double)m;
        oy = sy / (double)m;
    }
    if (lane == 0) {
        a.xy_out[2 * w] = ox;
        a.xy_out[2 * w + 1] = oy;
        a.status[w] = status;
    }
}

// Algorithm 2 for one window of at most kWarpCand candidate slots, by a single
// warp: the same steps, tie rules and integer tests as the block path of
// aggregate.cu, with warp shuffles in place of block barriers.
__device__ inline void aggregate_warp(const AggParams& p, int w, long long b0, long long total, u64* keys, int* cand_rows,
                               float* cand_d, int* cnt) {
    const AggArgs& a = p.a;
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    // initialization: rows -> tiles, padding rows skipped, compacted in order;
    // up to 128 slots in registers, sorted there for the binning below
    int C = 0;
    bool sorted = false;
    if (total <= 32) {
        C = init_sorted<1>(p, b0, total, keys, cand_rows, cand_d, lane, a.mode != 2);
        sorted = true;
    } else if (total <= 64) {
        C = init_sorted<2>(p, b0, total, keys, cand_rows, cand_d, lane, a.mode != 2);
        sorted = true;
    } else if (total <= 128) {
        C = init_sorted<4>(p, b0, total, keys, cand_rows, cand_d, lane, a.mode != 2);
        sorted = true;
    }
    for (long long base = 0; !sorted && base < total; base += 32) {
        const long long i = base + lane;
        const int64_t r = i < total ? __ldcg(a.idx + b0 + i) : -1;  // may come from another CTA of the launch
        const bool bad = r >= p.n;
        if (bad) record_error(p.err, kErrInvalidArg);
        const bool take = r >= 0 && !bad;
        const unsigned m = __ballot_sync(kFull, take);
        const int pos = C + __popc(m & below);
        if (take) {
            cand_rows[pos] = (int)r;
            cand_d[pos] = a.dist != nullptr ? __ldcg(a.dist + b0 + i) : 0.f;
            keys[pos] = p.tile_keys != nullptr ? __ldcg(p.tile_keys + b0 + i) : tile_key(p.tile[2 * r], p.tile[2 * r + 1]);
        }
        C += __popc(m);
    }
    __syncwarp();
    if (C == 0) {
        if (lane == 0) write_invalid(a, w);
        return;
    }
    const double tm = a.tile_m;
    int status = 0;
    int win_tx = 0, win_ty = 0;
    if (a.mode != 2) {
        // step 2: binning = sort the tile keys (in registers), count runs
        static_assert(kWarpCand == 32 * 32, "sort widths below cover kWarpCand");
        if (sorted) {
            // keys[0, C) hold the candidates' sorted keys (the empty keys follow)
        } else if (C <= 32) warp_sort_smem<1>(keys, C, lane);
        else if (C <= 64) warp_sort_smem<2>(keys, C, lane);
        else if (C <= 128) warp_sort_smem<4>(keys, C, lane);
        else if (C <= 256) warp_sort_smem<8>(keys, C, lane);
        else if (C <= 512) warp_sort_smem<16>(keys, C, lane);
        else warp_sort_smem<32>(keys, C, lane);
        __syncwarp();
        int U = 0;
        for (int base = 0; base < C; base += 32) {
            const int i = base + lane;
            const bool st = i < C && (i == 0 || keys[i] != keys[i - 1]);
            const unsigned m = __ballot_sync(kFull, st);
            if (st) cnt[U + __popc(m & below)] = i;
            U += __popc(m);
        }
        if (lane == 0) cnt[U] = C;
        int* taken = reinterpret_cast<int*>(cand_d);  // tile modes do not read distances
        for (int u = lane; u < U; u += 32) taken[u] = 0;
        __syncwarp();
        // steps 5-7: draw tiles by (count desc, ty asc, tx asc); first circle above the threshold wins
        const int ntop = min(a.top_c, U);
        int first_tx = 0, first_ty = 0;
        bool found = false;
        for (int r = 0; r < ntop; ++r) {
            long long best = -1;
            for (int u = lane; u < U; u += 32) {
                if (taken[u]) continue;
                const long long c = cnt[u + 1] - cnt[u];
                const long long v = (c << 32) | (long long)(0xffffffffu - (unsigned)u);
                best = v > best ? v : best;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const long long ov = __shfl_xor_sync(kFull, best, o);
                best = ov > best ? ov : best;
            }
            const int us = (int)(0xffffffffu - (unsigned)(best & 0xffffffffll));
            __syncwarp();
            if (lane == 0) taken[us] = 1;
            __syncwarp();
            const u64 ks = keys[cnt[us]];
            const int tx0 = key_tx(ks), ty0 = key_ty(ks);
            if (r == 0) {
                first_tx = tx0;
                first_ty = ty0;
            }
            long long circ = 0;
            for (int u = lane; u < U; u += 32) {
                const u64 ku = keys[cnt[u]];
                const long long dx = (long long)key_tx(ku) - tx0, dy = (long long)key_ty(ku) - ty0;
                if (dx > p.rlim || dx < -p.rlim || dy > p.rlim || dy < -p.rlim) continue;
                if (dx * dx + dy * dy <= a.r2max) circ += cnt[u + 1] - cnt[u];
            }
            circ = warp_sum(circ);
            if (100ll * circ > (long long)a.toler_pct * (long long)C) {
                win_tx = tx0;
                win_ty = ty0;
                found = true;
                break;
            }
        }
        if (!found) {
            win_tx = first_tx;
            win_ty = first_ty;
            status = 1;
        }
    }
    double ox, oy;
    if (a.mode == 0) {
        ox = ((double)win_tx + 0.5) * tm;
        oy = ((double)win_ty + 0.5) * tm;
    } else if (a.mode == 1) {
        double sx = 0.0, sy = 0.0;
        long long m = 0;
        for (int i = lane; i < C; i += 32) {
            const int r = cand_rows[i];
            const long long dx = (long long)p.tile[2 * r] - win_tx, dy = (long long)p.tile[2 * r + 1] - win_ty;
            if (dx > p.rlim || dx < -p.rlim || dy > p.rlim || dy < -p.rlim) continue;
            if (dx * dx + dy * dy <= a.r2max) {
                sx += p.xy[2 * r];
                sy += p.xy[2 * r + 1];
                ++m;
            }
        }
        sx = warp_sum(sx);
        sy = warp_sum(sy);
        m = warp_sum(m);
        ox = sx / (double)m;
        oy = sy / (double)m;
    } else {
        double mx = -INFINITY;
        for (int i = lane; i < C; i += 32) mx = fmax(mx, -(double)cand_d[i] / (double)a.tau);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(kFull, mx, o));
        double z = 0.0, sx = 0.0, sy = 0.0;
        for (int i = lane; i < C; i += 32) {
            const double e = exp(-(double)cand_d[i] / (double)a.tau - mx);
            const int r = cand_rows[i];
            z += e;
            sx += e * p.xy[2 * r];
            sy += e * p.xy[2 * r + 1];
        }
        z = warp_sum(z);
        sx = warp_sum(sx);
        sy = warp_sum(sy);
        ox = sx / z;
        oy = sy / z;
    }
    if (lane == 0) {
        a.xy_out[2 * w] = ox;
        a.xy_out[2 * w + 1] = oy;
        a.status[w] = status;
    }
}


}  // namespace agg
}  // namespace lhr
