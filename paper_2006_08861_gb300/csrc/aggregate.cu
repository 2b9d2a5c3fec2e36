// Algorithm 2 (§3.2): 2-D multi-frame localization candidate aggregation,
// one warp per window (one CTA for windows of more than 1,024 candidate
// slots), entirely on the device so a window's answer never makes a host
// round trip.
//
//   initialization  candidate row -> floor-plan tile through the database's
//                   geo-referenced table (tiles precomputed at build:
//                   tx = floor(x / t), ty = floor(y / t), IEEE double divide)
//   step 2          2-D binning: the window's tile keys are sorted (bitonic,
//                   shared memory) and run-length counted -> locationDistriArray
//                   as a sparse list of (tile, count)
//   steps 5-6       rank by count descending, ties by (ty, tx) ascending; the
//                   first TopC tiles are drawn by repeated block-wide argmax
//   step 7          tolerance circle of each drawn tile in rank order:
//                   sum of counts of tiles with dx^2 + dy^2 <= r2max (integer
//                   test); the first with 100 * circle > tolerPer * C wins
// If no drawn tile passes, the top-ranked tile is returned with status
// LHR_WARN_LOW_CONFIDENCE. The reported position is the tile centre, or the
// FP64 mean position of the candidates inside the winner's circle
// (TILE_CENTROID), or the softmax(-d / tau)-weighted mean (SOFTMAX).
#include <math.h>

#include "common.cuh"
#include "internal.h"

#include "aggregate.cuh"

namespace lhr {
namespace {

using namespace agg;

constexpr int kAggThreads = 256;
constexpr int kMaxCand = 8192;

template <typename T>
__device__ T block_sum(T v, T* red) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    T s = 0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
        red[0] = s;
    }
    __syncthreads();
    s = red[0];
    __syncthreads();
    return s;
}

// Window w (kWarpCand < total <= kMaxCand candidate slots from b0) by the whole block.
__device__ void aggregate_block(const AggParams& p, int w, long long b0, long long total, unsigned char* smem) {
    u64* keys = reinterpret_cast<u64*>(smem);                      // kMaxCand tile keys (sorted)
    int* cand_rows = reinterpret_cast<int*>(keys + kMaxCand);      // kMaxCand candidate rows
    float* cand_d = reinterpret_cast<float*>(cand_rows + kMaxCand);  // kMaxCand distances
    int* cnt = reinterpret_cast<int*>(cand_d + kMaxCand);          // kMaxCand + 1 run starts
    double* redd = reinterpret_cast<double*>(cnt + kMaxCand + 2);  // 32
    long long* redl = reinterpret_cast<long long*>(redd + 32);     // 32
    int* ctl = reinterpret_cast<int*>(redl + 32);                  // control words

    const AggArgs& a = p.a;
    const int t = threadIdx.x;
    if (t == 0) ctl[0] = 0;
    __syncthreads();
    // initialization: rows -> tiles (padding rows -1 are skipped)
    for (long long i = t; i < total; i += blockDim.x) {
        const int64_t r = a.idx[b0 + i];
        if (r < 0) continue;
        if (r >= p.n) {
            record_error(p.err, kErrInvalidArg);
            continue;
        }
        const int pos = atomicAdd(&ctl[0], 1);
        cand_rows[pos] = (int)r;
        cand_d[pos] = a.dist != nullptr ? a.dist[b0 + i] : 0.f;
        keys[pos] = tile_key(p.tile[2 * r], p.tile[2 * r + 1]);
    }
    __syncthreads();
    const int C = ctl[0];
    if (C == 0) {
        if (t == 0) {
            a.status[w] = kErrInvalidArg;
            a.xy_out[2 * w] = a.xy_out[2 * w + 1] = __longlong_as_double(0x7ff8000000000000ll);
        }
        return;
    }
    const double tm = a.tile_m;
    int status = 0;
    int win_tx = 0, win_ty = 0;
    if (a.mode != 2) {
        // step 2: binning = sort the tile keys and count runs
        int p2 = 1;
        while (p2 < C) p2 <<= 1;
        for (int i = C + t; i < p2; i += blockDim.x) keys[i] = kKeyEmpty;
        __syncthreads();
        for (int size = 2; size <= p2; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int i = t; i < p2 / 2; i += blockDim.x) {
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
        // compact run starts in key order: cnt[u] = first index of unique tile u
        {
            constexpr int kPer = kMaxCand / kAggThreads;  // 32 sorted keys per thread
            const int i0 = t * kPer;
            int local = 0;
            for (int i = i0; i < min(i0 + kPer, C); ++i) local += (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
            // exclusive block scan of `local`
            int incl = local;
            const int lane = t & 31, wi = t >> 5;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += v;
            }
            if (lane == 31) ctl[8 + wi] = incl;
            __syncthreads();
            if (t == 0) {
                int run = 0;
                for (int i = 0; i < kAggThreads / 32; ++i) {
                    const int v = ctl[8 + i];
                    ctl[8 + i] = run;
                    run += v;
                }
                ctl[1] = run;
                cnt[run] = C;
            }
            __syncthreads();
            int u = ctl[8 + wi] + incl - local;
            for (int i = i0; i < min(i0 + kPer, C); ++i)
                if (i == 0 || keys[i] != keys[i - 1]) cnt[u++] = i;
        }
        __syncthreads();
        const int U = ctl[1];
        // Tile u has key keys[cnt[u]] and count cnt[u + 1] - cnt[u].
        const int ntop = min(a.top_c, U);
        // taken[u]: tile u already drawn. Aliases cand_d, which the tile modes
        // do not read (U <= C).
        int* taken = reinterpret_cast<int*>(cand_d);
        for (int u = t; u < U; u += blockDim.x) taken[u] = 0;
        __syncthreads();
        int first_tx = 0, first_ty = 0;
        bool found = false;
        for (int r = 0; r < ntop; ++r) {
            // argmax of (count desc, u asc) over tiles not taken
            long long best = -1;  // (count << 32) | (0xffffffff - u)
            for (int u = t; u < U; u += blockDim.x) {
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
            __syncthreads();
            if ((t & 31) == 0) redl[t >> 5] = best;
            __syncthreads();
            if (t == 0) {
                long long b = redl[0];
                for (int i = 1; i < (int)(blockDim.x >> 5); ++i) b = redl[i] > b ? redl[i] : b;
                const int u = (int)(0xffffffffu - (unsigned)(b & 0xffffffffll));
                taken[u] = 1;
                ctl[2] = u;
            }
            __syncthreads();
            const int us = ctl[2];
            const u64 ks = keys[cnt[us]];
            const int tx0 = key_tx(ks), ty0 = key_ty(ks);
            if (r == 0) {
                first_tx = tx0;
                first_ty = ty0;
            }
            long long circ = 0;
            for (int u = t; u < U; u += blockDim.x) {
                const u64 ku = keys[cnt[u]];
                const long long dx = (long long)key_tx(ku) - tx0, dy = (long long)key_ty(ku) - ty0;
                if (dx > p.rlim || dx < -p.rlim || dy > p.rlim || dy < -p.rlim) continue;
                if (dx * dx + dy * dy <= a.r2max) circ += cnt[u + 1] - cnt[u];
            }
            circ = block_sum<long long>(circ, redl);
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
        for (int i = t; i < C; i += blockDim.x) {
            const int r = cand_rows[i];
            const long long dx = (long long)p.tile[2 * r] - win_tx, dy = (long long)p.tile[2 * r + 1] - win_ty;
            if (dx > p.rlim || dx < -p.rlim || dy > p.rlim || dy < -p.rlim) continue;
            if (dx * dx + dy * dy <= a.r2max) {
                sx += p.xy[2 * r];
                sy += p.xy[2 * r + 1];
                ++m;
            }
        }
        sx = block_sum<double>(sx, redd);
        sy = block_sum<double>(sy, redd);
        m = block_sum<long long>(m, redl);
        ox = sx / (double)m;
        oy = sy / (double)m;
    } else {
        // softmax(-d / tau) over the window's candidates, FP64 sums
        double mx = -INFINITY;
        for (int i = t; i < C; i += blockDim.x) mx = fmax(mx, -(double)cand_d[i] / (double)a.tau);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(kFull, mx, o));
        __syncthreads();
        if ((t & 31) == 0) redd[t >> 5] = mx;
        __syncthreads();
        if (t == 0) {
            double m2 = redd[0];
            for (int i = 1; i < (int)(blockDim.x >> 5); ++i) m2 = fmax(m2, redd[i]);
            redd[0] = m2;
        }
        __syncthreads();
        mx = redd[0];
        __syncthreads();
        double z = 0.0, sx = 0.0, sy = 0.0;
        for (int i = t; i < C; i += blockDim.x) {
            const double e = exp(-(double)cand_d[i] / (double)a.tau - mx);
            const int r = cand_rows[i];
            z += e;
            sx += e * p.xy[2 * r];
            sy += e * p.xy[2 * r + 1];
        }
        z = block_sum<double>(z, redd);
        sx = block_sum<double>(sx, redd);
        sy = block_sum<double>(sy, redd);
        ox = sx / z;
        oy = sy / z;
    }
    if (t == 0) {
        a.xy_out[2 * w] = ox;
        a.xy_out[2 * w + 1] = oy;
        a.status[w] = status;
    }
}

// Per-warp shared memory of the warp path: tile keys, rows and distances of up
// to kWarpCand slots, and kWarpCand + 1 run starts (16-byte multiple).
constexpr size_t kWarpSlice = ((size_t)kWarpCand * (sizeof(u64) + 2 * sizeof(int)) + (kWarpCand + 1) * sizeof(int) + 15) / 16 * 16;
constexpr int kAggWindows = kAggThreads / 32;  // windows per CTA: one per warp

// Algorithm 2 for kAggWindows windows per CTA: each warp takes one window of at
// most kWarpCand slots in its own slice of shared memory; larger windows are
// then run one at a time by the whole block over all of it.
__global__ void __launch_bounds__(kAggThreads) aggregate_kernel(const AggParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int large_w[kAggWindows];
    __shared__ long long large_b0[kAggWindows], large_n[kAggWindows];
    const AggArgs& a = p.a;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int w = blockIdx.x * kAggWindows + warp;
    bool large = false;
    long long b0 = 0, total = 0;
    if (w < a.nw) {
        b0 = a.offsets[w];
        long long b1 = a.offsets[w + 1];
        if (a.per_frame > 0) {
            b0 *= a.per_frame;
            b1 *= a.per_frame;
        }
        total = b1 - b0;
        if (total <= 0 || total > kMaxCand || b0 < 0 || b1 > a.limit) {
            if (lane == 0) write_invalid(a, w);
        } else if (total <= kWarpCand) {
            unsigned char* sl = smem + (size_t)warp * kWarpSlice;
            u64* keys = reinterpret_cast<u64*>(sl);
            int* rows = reinterpret_cast<int*>(keys + kWarpCand);
            float* dd = reinterpret_cast<float*>(rows + kWarpCand);
            int* cnt = reinterpret_cast<int*>(dd + kWarpCand);
            aggregate_warp(p, w, b0, total, keys, rows, dd, cnt);
        } else {
            large = true;
        }
    }
    if (lane == 0) {
        large_w[warp] = large ? w : -1;
        large_b0[warp] = b0;
        large_n[warp] = total;
    }
    __syncthreads();
    for (int k = 0; k < kAggWindows; ++k) {
        if (large_w[k] >= 0) aggregate_block(p, large_w[k], large_b0[k], large_n[k], smem);
        __syncthreads();
    }
}

constexpr size_t agg_smem() {
    return kMaxCand * (sizeof(u64) + sizeof(int) + sizeof(float) + sizeof(int)) + 2 * sizeof(int) +
           32 * (sizeof(double) + sizeof(long long)) + (8 + kAggThreads / 32) * sizeof(int);
}

}  // namespace

long long circle_r2_limit(double radius_m, double tile_m) {
    auto snap = [](double v) {
        const double r = nearbyint(v);
        return fabs(v - r) <= 1e-9 * fmax(1.0, fabs(v)) ? r : v;
    };
    const double rt = snap(radius_m / tile_m);
    return (long long)floor(snap(rt * rt));
}

cudaError_t launch_aggregate(const lhr_db* db, const AggArgs& a, cudaStream_t stream) {
    AggParams p{};
    p.a = a;
    p.tile = db->tile;
    p.xy = db->xy;
    p.n = db->n;
    p.rlim = (long long)floor(sqrt((double)a.r2max)) + 1;
    p.err = db->err;
    const size_t sm = agg_smem();
    static_assert(kAggWindows * kWarpSlice <= agg_smem(), "the warps' slices fit in the block path's shared memory");
    cudaError_t e = cudaFuncSetAttribute(aggregate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    ProfScope ps("aggregate_kernel", stream);
    aggregate_kernel<<<(a.nw + kAggWindows - 1) / kAggWindows, kAggThreads, sm, stream>>>(p);
    return cudaGetLastError();
}

}  // namespace lhr
