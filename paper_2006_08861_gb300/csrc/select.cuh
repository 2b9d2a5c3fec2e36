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
