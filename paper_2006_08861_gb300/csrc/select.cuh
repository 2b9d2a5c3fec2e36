// Radix-select building blocks shared by the coarse-to-fine kernels: the key
// of a row under a per-frame distance array, the block-wide search for the
// histogram bin holding a given rank, and warp-aggregated list appends.
#pragma once

#include "common.cuh"

namespace lhr {
namespace sel {

constexpr int kBins = 2048;  // 11-bit digits

// Finds the bin holding the `need`-th smallest key of a 2048-bin histogram in
// shared memory, with a block of THREADS threads. Writes (bin, keys below it,
// keys in it) to out[0..2]. `tmp` holds THREADS / 32 words.
template <int THREADS>
__device__ void find_bin(const unsigned* hsm, unsigned need, unsigned* out, unsigned* tmp) {
    constexpr int kPer = kBins / THREADS;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    unsigned own = 0;
#pragma unroll
    for (int i = 0; i < kPer; ++i) own += hsm[t * kPer + i];
    unsigned s = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned v = __shfl_up_sync(kFull, s, o);
        if (lane >= o) s += v;
    }
    if (lane == 31) tmp[w] = s;
    __syncthreads();
    if (w == 0) {
        unsigned v = lane < THREADS / 32 ? tmp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned u = __shfl_up_sync(kFull, v, o);
            if (lane >= o) v += u;
        }
        if (lane < THREADS / 32) tmp[lane] = v;
    }
    __syncthreads();
    unsigned before = (w > 0 ? tmp[w - 1] : 0u) + s - own;  // keys below this thread's first bin
    if (before < need && need <= before + own) {
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const unsigned c = hsm[t * kPer + i];
            if (before < need && need <= before + c) {
                out[0] = t * kPer + i;
                out[1] = before;
                out[2] = c;
            }
            before += c;
        }
    }
    __syncthreads();
}

// The same search over a histogram in global memory, by one warp. The loads
// are coalesced (instruction i reads bins [128 i, 128 i + 128), lane l four
// of them: every SM reads the same histogram at once, so the requests per
// line matter); the 16 chunk totals come from warp reductions, the chunk
// holding the need-th key from static selects, the lane and bin inside it
// from one warp scan. Returns (bin, keys below it, keys in it) on every lane;
// zeros when the histogram holds fewer than `need` keys.
__device__ __forceinline__ uint3 warp_find_bin(const unsigned* hist, unsigned need, int lane) {
    static_assert(kBins == 16 * 128, "16 chunks of 128 bins");
    const uint4* h4 = reinterpret_cast<const uint4*>(hist);
    uint4 v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __ldcg(h4 + i * 32 + lane);
    unsigned c[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) c[i] = __reduce_add_sync(kFull, v[i].x + v[i].y + v[i].z + v[i].w);
    // the chunk is the last one starting below `need`
    unsigned run = 0, cbefore = 0;
    int ci = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        if (run < need) {
            ci = i;
            cbefore = run;
        }
        run += c[i];
    }
    uint4 q = v[0];
#pragma unroll
    for (int i = 1; i < 16; ++i)
        if (i == ci) q = v[i];
    const unsigned own = q.x + q.y + q.z + q.w;
    unsigned s = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned u = __shfl_up_sync(kFull, s, o);
        if (lane >= o) s += u;
    }
    const unsigned before = cbefore + s - own;
    const bool mine = before < need && need <= before + own;
    uint3 out = make_uint3(0u, 0u, 0u);
    if (mine) {
        const unsigned cq[4] = {q.x, q.y, q.z, q.w};
        unsigned bj = 0, bb = before, bc = q.x, r = before;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (r < need) {
                bj = (unsigned)j;
                bb = r;
                bc = cq[j];
            }
            r += cq[j];
        }
        out = make_uint3((unsigned)(ci * 128 + lane * 4) + bj, bb, bc);
    }
    const unsigned m = __ballot_sync(kFull, mine);
    const int src = m ? __ffs(m) - 1 : 0;
    out.x = __shfl_sync(kFull, out.x, src);
    out.y = __shfl_sync(kFull, out.y, src);
    out.z = __shfl_sync(kFull, out.z, src);
    return out;
}

// The need-th smallest (1-based) of the nb distinct keys keys[0, nb) in shared
// memory, all of which lie in [lo, hi] (inclusive; any range): radix
// refinement, each pass histogramming the keys still in range on the 11-bit
// digit (key - lo) >> shift (shift chosen so the range fits 2048 bins), until
// one key is left. `hsm` holds kBins words, `res` 4 and `tmp` THREADS / 32;
// every thread of the block calls it and gets the key.
template <int THREADS>
__device__ u64 block_kth_key(const u64* keys, unsigned nb, unsigned need, u64 lo, u64 hi, unsigned* hsm,
                             unsigned* res, unsigned* tmp) {
    const int t = threadIdx.x;
    for (;;) {
        const u64 span = hi - lo;
        if (span == 0) return lo;
        const int bits = 64 - __clzll((long long)span);
        const int shift = bits > 11 ? bits - 11 : 0;
        for (int i = t; i < kBins; i += THREADS) hsm[i] = 0u;
        __syncthreads();
        for (unsigned i = t; i < nb; i += THREADS) {
            const u64 key = keys[i];
            if (key >= lo && key <= hi) atomicAdd(&hsm[(unsigned)((key - lo) >> shift)], 1u);
        }
        __syncthreads();
        find_bin<THREADS>(hsm, need, res, tmp);
        const u64 nlo = lo + ((u64)res[0] << shift);
        const u64 room = hi - nlo, width = (1ull << shift) - 1ull;
        hi = nlo + (room < width ? room : width);
        lo = nlo;
        need -= res[1];
        if (shift == 0) return lo;
        if (res[2] == 1u) break;
    }
    // one key left in [lo, hi]
    u64* found = reinterpret_cast<u64*>(hsm);
    __syncthreads();
    for (unsigned i = t; i < nb; i += THREADS) {
        const u64 key = keys[i];
        if (key >= lo && key <= hi) *found = key;
    }
    __syncthreads();
    const u64 key = *found;
    __syncthreads();
    return key;
}

__device__ __forceinline__ u64 coarse_key(const float* dcf, int64_t row) {
    return ((u64)__float_as_uint(dcf[row]) << 32) | (u64)row;
}

// Appends `take` rows / keys of a warp at consecutive positions of a list.
__device__ __forceinline__ void warp_append(bool take, unsigned* counter, unsigned cap, int* rows, u64* keys,
                                            int64_t row, u64 key, int lane) {
    const unsigned m = __ballot_sync(kFull, take);
    if (!m) return;
    unsigned base = 0;
    const int leader = __ffs(m) - 1;
    if (lane == leader) base = atomicAdd(counter, (unsigned)__popc(m));
    base = __shfl_sync(kFull, base, leader);
    const unsigned pos = base + __popc(m & ((1u << lane) - 1u));
    if (take && pos < cap) {
        if (rows) rows[pos] = (int)row;
        else keys[pos] = key;
    }
}

}  // namespace sel
}  // namespace lhr
