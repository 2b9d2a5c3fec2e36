// tcgen05 / TMA building blocks shared by the tensor-core kernels (inline PTX):
// 2-D tensor copies into shared memory (plain and cluster multicast), the
// tensor core's fences, commits and MMA issue for BF16, FP8-e4m3 and TF32
// operands, TMEM loads, the K-major 128-byte-swizzle shared-memory matrix
// descriptor, the instruction descriptor, and the host-side tensor-map encoder.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "common.cuh"

namespace lhr {
namespace tc {

constexpr int kTcM = 128;         // rows of A per MMA (M), one TMEM lane each
constexpr int kTcSliceBytes = 128;  // K bytes per shared-memory row (one 128-byte swizzle atom)

// Operand kinds: tcgen05.mma kind and the format code of A and B in the instruction descriptor.
enum TcKind { kTcBF16 = 0, kTcFP8 = 1, kTcTF32 = 2, kTcF16 = 3 };
__host__ __device__ constexpr int tc_elem_bytes(TcKind k) {
    return k == kTcFP8 ? 1 : (k == kTcTF32 ? 4 : 2);
}
// A / B format code in the instruction descriptor: E4M3 0 (kind::f8f6f4), F16 0
// and BF16 1 (kind::f16), TF32 2 (kind::tf32).
__host__ __device__ constexpr uint32_t tc_format(TcKind k) {
    return k == kTcBF16 ? 1u : (k == kTcTF32 ? 2u : 0u);
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1, u64* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

// The same tile box delivered to the shared memory of every CTA of the cluster
// in `mask` (same offsets in each), completing bytes on each CTA's barrier at
// `bar`'s offset.
__device__ __forceinline__ void tma_load_2d_mc(void* dst, const CUtensorMap* map, int c0, int c1, u64* bar,
                                               uint16_t mask) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster [%0], [%1, {%2, "
        "%3}], [%4], %5;" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar)), "h"(mask)
        : "memory");
}

__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// All threads of every CTA of the cluster (a plain block barrier when the cluster is one CTA).
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_commit(u64* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// Arrival, once this thread's earlier tcgen05 operations complete, on the barrier
// at `bar`'s offset in every CTA of the cluster in `mask`.
__device__ __forceinline__ void tc_commit_mc(u64* bar, uint16_t mask) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
                     smem_u32(bar)),
                 "h"(mask)
                 : "memory");
}

template <TcKind K>
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, u64 adesc, u64 bdesc, uint32_t idesc, uint32_t accum) {
    if (K == kTcFP8) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
            : "memory");
    } else if (K == kTcBF16 || K == kTcF16) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
            : "memory");
    }
}

// MMA with the A operand in tensor memory: M rows x K, a row per TMEM lane,
// from column a_tmem on 32 bits per column (one TF32 element, or two 16-bit
// elements, the lower-indexed in the low half).
template <TcKind K>
__device__ __forceinline__ void tc_mma_tmem_a(uint32_t d_tmem, uint32_t a_tmem, u64 bdesc, uint32_t idesc,
                                              uint32_t accum) {
    if (K == kTcTF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
            "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accum)
            : "memory");
    } else {
        static_assert(K == kTcTF32 || K == kTcF16 || K == kTcBF16, "16- or 32-bit operands");
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
            "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accum)
            : "memory");
    }
}

// tcgen05.st of 32 columns: this thread's lane of columns taddr .. taddr + 31.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
        "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]),
        "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]),
        "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}

__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// tcgen05.ld of 32 columns without the wait: the registers are valid only after
// tmem_ld_wait on the same array, which names them so nothing reads them earlier.
__device__ __forceinline__ void tmem_ld32_issue(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld_wait(uint32_t (&r)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                   "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row core groups 1024 bytes apart.
__device__ __forceinline__ u64 sw128_desc(uint32_t saddr) {
    u64 d = (u64)((saddr >> 4) & 0x3FFFu);
    d |= (u64)1 << 16;              // leading-dimension offset (unused with this swizzle)
    d |= (u64)(1024 >> 4) << 32;    // stride-dimension offset: 1024 B between 8-row groups
    d |= (u64)1 << 46;              // descriptor version for tcgen05
    d |= (u64)2 << 61;              // 128-byte swizzle
    return d;
}

// Instruction descriptor: dense, FP32 accumulate, A/B K-major, M = 128, N = n
// (a multiple of 16, <= 256), operand formats by tc_format.
__host__ __device__ constexpr uint32_t tc_idesc(TcKind k, int n) {
    return (1u << 4)                                                        // D format: F32
           | (tc_format(k) << 7)                                              // A format
           | (tc_format(k) << 10)                                             // B format
           | ((uint32_t)(n >> 3) << 17)                                     // N >> 3
           | ((uint32_t)(kTcM >> 4) << 24);                                 // M >> 4
}

// Three-input maximum (one instruction on this architecture).
__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Three-input minimum.
__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Minimum over the warp's 32 rows of each of 32 columns (c[j] = this lane's
// row, column j): a butterfly in which every step exchanges half of the
// remaining columns with the partner lane; lane l ends with column l's minimum.
__device__ __forceinline__ float column_min32(float (&c)[32], int lane) {
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const bool upper = (lane & s) != 0;
#pragma unroll
        for (int i = 0; i < s; ++i) {
            const float send = upper ? c[i] : c[i + s];
            const float keep = upper ? c[i + s] : c[i];
            c[i] = fminf(keep, __shfl_xor_sync(0xffffffffu, send, s));
        }
    }
    return c[0];
}

// Maximum of 32 accumulator values in four interleaved chains of three-input
// maxima (few live temporaries).
__device__ __forceinline__ float max32(const uint32_t (&v)[32]) {
    float c[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) c[i] = fmax3(__uint_as_float(v[i]), __uint_as_float(v[4 + i]), __uint_as_float(v[8 + i]));
#pragma unroll
    for (int j = 12; j < 28; j += 8)
#pragma unroll
        for (int i = 0; i < 4; ++i) c[i] = fmax3(c[i], __uint_as_float(v[j + i]), __uint_as_float(v[j + 4 + i]));
#pragma unroll
    for (int i = 0; i < 4; ++i) c[i] = fmaxf(c[i], __uint_as_float(v[28 + i]));
    return fmax3(c[0], c[1], fmaxf(c[2], c[3]));
}

// ------------------------------------------------------------------ host
inline PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void* f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    });
    return fn;
}

// 2-D map over a row-major rows x D array of operands of kind k; box = 128
// bytes of K by box_rows rows, 128-byte swizzle, zero fill past the last row.
// row_pitch: elements from one mapped row to the next (0 = D; a multiple of D
// maps every (row_pitch / D)-th row of a larger array).
inline bool make_map(CUtensorMap* map, const void* base, int64_t rows, int D, TcKind k, int box_rows,
                     int64_t row_pitch = 0) {
    auto fn = encode_fn();
    if (!fn) return false;
    const int elem = tc_elem_bytes(k);
    cuuint64_t dims[2] = {(cuuint64_t)D, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(row_pitch > 0 ? row_pitch : D) * elem};
    cuuint32_t box[2] = {(cuuint32_t)(kTcSliceBytes / elem), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    const CUtensorMapDataType dt = k == kTcFP8    ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                   : k == kTcBF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                   : k == kTcF16  ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                  : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const CUresult r = fn(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace tc
}  // namespace lhr
