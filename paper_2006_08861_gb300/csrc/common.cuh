// Device-side building blocks shared by the library's kernels: candidate
// keys, warp-register top-N lists, mbarrier / bulk-copy wrappers (inline PTX)
// and bounded waits.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lhr {

typedef unsigned long long u64;

constexpr unsigned kFull = 0xffffffffu;
constexpr u64 kKeyEmpty = 0xffffffffffffffffull;
// Device-side waits give up after this long and record LHR_ERR_TIMEOUT.
constexpr u64 kWaitLimitNs = 1000000000ull;

// Error codes written to a database's device error word (match lhr_status).
constexpr int kErrInvalidArg = -1;
constexpr int kErrTimeout = -4;

// A candidate is packed as (distance bits << 32 | row). Squared distances are
// >= 0, so their IEEE bits order like the values; the row in the low word
// breaks ties toward the lower row, which is the library's tie rule.
__device__ __forceinline__ u64 make_key(float d, uint32_t row) {
    return ((u64)__float_as_uint(d) << 32) | (u64)row;
}
__device__ __forceinline__ float key_dist(u64 k) { return __uint_as_float((uint32_t)(k >> 32)); }
__device__ __forceinline__ uint32_t key_row(u64 k) { return (uint32_t)k; }

// Warp-register sorted list of the k (<= 32) smallest keys: lane i holds the
// i-th smallest, lanes >= k hold kKeyEmpty. Inserts one warp-uniform key.
__device__ __forceinline__ void list_insert(u64& L, u64 key, int k, int lane) {
    const unsigned lt = __ballot_sync(kFull, L < key);
    const int pos = __popc(lt);
    const u64 up = __shfl_up_sync(kFull, L, 1);
    if (pos < k) {
        if (lane == pos) L = key;
        else if (lane > pos && lane < k) L = up;
    }
}

// Merge `n` keys from memory (any order) into the warp list L.
// `thr` is kept equal to L's k-th key so most keys are rejected with one compare.
template <bool kCacheGlobal>
__device__ __forceinline__ void list_merge_keys(u64& L, const u64* keys, int n, int k, int lane) {
    u64 thr = __shfl_sync(kFull, L, k - 1);
    for (int base = 0; base < n; base += 32) {
        const int i = base + lane;
        u64 key = kKeyEmpty;
        if (i < n) key = kCacheGlobal ? __ldcg(keys + i) : keys[i];
        unsigned m = __ballot_sync(kFull, key < thr);
        while (m) {
            const int j = __ffs(m) - 1;
            m &= m - 1;
            const u64 kj = __shfl_sync(kFull, key, j);
            list_insert(L, kj, k, lane);
        }
        thr = __shfl_sync(kFull, L, k - 1);
    }
}

// ---------------------------------------------------------------- PTX wrappers
// 64 keys of a warp, element e * 32 + lane in v[e], sorted ascending (bitonic).
__device__ __forceinline__ void warp_sort64(u64 (&v)[2], int lane) {
#pragma unroll
    for (int size = 2; size <= 64; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride == 32) {
                const u64 lo = v[0] < v[1] ? v[0] : v[1], hi = v[0] < v[1] ? v[1] : v[0];
                v[0] = lo;
                v[1] = hi;
            } else {
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const u64 o = __shfl_xor_sync(kFull, v[e], stride);
                    const bool asc = ((e * 32 + lane) & size) == 0;
                    const bool keep_min = ((lane & stride) == 0) == asc;
                    v[e] = keep_min ? (o < v[e] ? o : v[e]) : (o > v[e] ? o : v[e]);
                }
            }
        }
    }
}

// best (64 sorted keys, layout of warp_sort64) becomes the 64 smallest of best
// and c (also sorted): min(best_i, c_{63-i}) is a bitonic sequence holding
// them, which a half-cleaner cascade sorts.
__device__ __forceinline__ void warp_merge64(u64 (&best)[2], const u64 (&c)[2], int lane) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const u64 r = __shfl_sync(kFull, c[1 - e], 31 - lane);
        best[e] = best[e] < r ? best[e] : r;
    }
    const u64 lo = best[0] < best[1] ? best[0] : best[1], hi = best[0] < best[1] ? best[1] : best[0];
    best[0] = lo;
    best[1] = hi;
#pragma unroll
    for (int stride = 16; stride > 0; stride >>= 1) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const u64 o = __shfl_xor_sync(kFull, best[e], stride);
            const bool keep_min = (lane & stride) == 0;
            best[e] = keep_min ? (o < best[e] ? o : best[e]) : (o > best[e] ? o : best[e]);
        }
    }
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ u64 globaltimer() {
    u64 t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(u64* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(u64* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(u64* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(u64* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// try_wait with a suspend-time hint: the thread sleeps (issuing nothing) until
// the phase completes or about `ns` nanoseconds pass.
__device__ __forceinline__ bool mbar_try_wait_sleep(u64* bar, uint32_t parity, uint32_t ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}

// Waits for the phase of `bar` with the given parity; false if it did not
// complete within kWaitLimitNs or if `abort` was raised meanwhile. Between
// checks the thread sleeps in the barrier (up to 20 us at a time), so waiting
// warps take no issue slots from the warps that work.
__device__ __forceinline__ bool mbar_wait(u64* bar, uint32_t parity, volatile int* abort) {
    if (mbar_try_wait(bar, parity)) return true;
    const u64 t0 = globaltimer();
    for (;;) {
        if (mbar_try_wait_sleep(bar, parity, 20000u)) return true;
        if (abort != nullptr && *abort) return false;
        if (globaltimer() - t0 > kWaitLimitNs) return false;
    }
}

// 1-D bulk copy global -> shared (async proxy), completing `bytes` of
// transaction count on `bar`. dst / src 16-byte aligned, bytes % 16 == 0.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, u64* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Hint: bring `bytes` (multiple of 16, 16-byte aligned) of global memory into L2.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ void record_error(int* err_word, int code) {
    if (err_word != nullptr) atomicCAS(err_word, 0, code);
}

}  // namespace lhr
