// Coarse-to-fine retrieval: a prefix of the feature scored over every row,
// an S-row shortlist per frame, the full feature re-scored on the shortlist,
// top N of those. (The paper scores full features, §3.1; the prefix level is
// this library's hierarchical form. The FFT-magnitude feature of §3 puts its
// low frequencies first, which is what a prefix keeps.)
//
// The candidate key of a row is (prefix distance bits << 32 | row); the
// shortlist is the S smallest keys, found by a radix select on 11-bit digits.
//
// K1 coarse_kernel: thread per row (grid-stride), squared prefix distance to
//   up to 8 frames with packed FP32 FMAs, written to scratch (frames x n
//   floats, L2-resident at building scale), and a per-frame 2048-bin
//   histogram of the key's top digit (shared-memory bins, flushed once per
//   CTA).
// K2 collect_kernel: 16 CTAs per frame. Each finds, from the histogram, the
//   bin holding the S-th key, then scans its slice of the frame's distances
//   and appends (warp-aggregated atomics) every row below that bin to the
//   frame's direct list and every key inside it to the frame's boundary list.
//   If the boundary bin holds more keys than one CTA can sort (kBinCap), the
//   frame is flagged and left to K3's refinement path.
// K3 shortlist_kernel: one CTA per frame. Sorts the boundary keys (bitonic,
//   shared memory) to take exactly S rows (or, for a flagged frame, refines
//   the radix select by further 11-bit digits over the frame's distances and
//   collects in place), re-scores the S rows on the full feature (warp per
//   row, loads batched four rows deep) and keeps the top k in warp-register
//   lists merged at the end.
#include "common.cuh"
#include "internal.h"
#include "select.cuh"

namespace lhr {
namespace {

using namespace sel;

constexpr int kFB = 8;           // frames per coarse CTA
constexpr int kBinCap = 4096;    // boundary-bin keys sorted in shared memory
constexpr int kSelThreads = 1024;
constexpr int kMaxShortlist = 4096;
constexpr int kParts = 16;       // collect CTAs per frame
constexpr int kColThreads = 256;
constexpr int kCtl = 8;          // control words per frame

// Per-frame control words written by K2, read by K3.
enum { kDirect = 0, kInBin = 1, kRefine = 2, kNeed = 3, kLo = 4 /* u64 at 4..5 */, kHi = 6 /* u64 at 6..7 */ };

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

template <int DC4>
__global__ void __launch_bounds__(256) coarse_kernel(const float* __restrict__ Xc, int64_t n, int dc,
                                                     const float* __restrict__ Q, int qld, int nq,
                                                     float* __restrict__ dcout, unsigned* __restrict__ hist) {
    extern __shared__ __align__(16) unsigned char csm[];
    float4(*qs)[DC4] = reinterpret_cast<float4(*)[DC4]>(csm);
    unsigned(*h)[kBins] = reinterpret_cast<unsigned(*)[kBins]>(csm + sizeof(float4) * kFB * DC4);
    const int f0 = blockIdx.y * kFB;
    const int nf = min(kFB, nq - f0);
    const int d4 = dc / 4;
    for (int i = threadIdx.x; i < kFB * DC4; i += blockDim.x) {
        const int f = i / DC4, c = i % DC4;
        qs[f][c] = (f < nf && c < d4) ? reinterpret_cast<const float4*>(Q + (size_t)(f0 + f) * qld)[c]
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int i = threadIdx.x; i < nf * kBins; i += blockDim.x) (&h[0][0])[i] = 0u;
    __syncthreads();
    const float2 neg1 = f2(-1.f, -1.f);
    for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < n;
         row += (int64_t)gridDim.x * blockDim.x) {
        float4 x[DC4];
        const float4* xr = reinterpret_cast<const float4*>(Xc + row * dc);
#pragma unroll
        for (int c = 0; c < DC4; ++c) x[c] = c < d4 ? __ldg(xr + c) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int f = 0; f < kFB; ++f) {
            if (f < nf) {
                float2 acc = f2(0.f, 0.f);
#pragma unroll
                for (int c = 0; c < DC4; ++c) {
                    const float4 qv = qs[f][c];
                    float2 a = __ffma2_rn(f2(x[c].x, x[c].y), neg1, f2(qv.x, qv.y));
                    float2 b = __ffma2_rn(f2(x[c].z, x[c].w), neg1, f2(qv.z, qv.w));
                    acc = __ffma2_rn(a, a, acc);
                    acc = __ffma2_rn(b, b, acc);
                }
                const float d = acc.x + acc.y;
                dcout[(size_t)(f0 + f) * n + row] = d;
                atomicAdd(&h[f][__float_as_uint(d) >> 20], 1u);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nf * kBins; i += blockDim.x) {
        const unsigned v = (&h[0][0])[i];
        if (v) atomicAdd(&hist[(size_t)(f0 + i / kBins) * kBins + (i % kBins)], v);
    }
}


__global__ void __launch_bounds__(kColThreads) collect_kernel(const float* __restrict__ dcall, int64_t n,
                                                              const unsigned* __restrict__ hist, int S,
                                                              unsigned* __restrict__ ctl_all,
                                                              int* __restrict__ direct_all,
                                                              u64* __restrict__ bin_all) {
    __shared__ unsigned hsm[kBins];
    __shared__ unsigned res[4];
    __shared__ unsigned tmp[kColThreads / 32];
    const int f = blockIdx.y, part = blockIdx.x;
    const int t = threadIdx.x, lane = t & 31;
    const float* dcf = dcall + (size_t)f * n;
    unsigned* ctl = ctl_all + (size_t)f * kCtl;
    int* direct = direct_all + (size_t)f * kMaxShortlist;
    u64* bins = bin_all + (size_t)f * kBinCap;
    const bool take_all = n <= S;
    u64 lo = ~0ull, hi = ~0ull;
    if (!take_all) {
        for (int i = t; i < kBins; i += kColThreads) hsm[i] = hist[(size_t)f * kBins + i];
        __syncthreads();
        find_bin<kColThreads>(hsm, (unsigned)S, res, tmp);
        if (res[2] > (unsigned)kBinCap) {
            if (part == 0 && t == 0) ctl[kRefine] = 1u;
            return;
        }
        lo = (u64)res[0] << 52;
        hi = lo + (1ull << 52);
        if (part == 0 && t == 0) {
            ctl[kNeed] = (unsigned)S - res[1];
            *reinterpret_cast<u64*>(&ctl[kLo]) = lo;
            *reinterpret_cast<u64*>(&ctl[kHi]) = hi;
        }
    }
    const int64_t per = (n + kParts - 1) / kParts;
    const int64_t r0 = part * per, r1 = min(n, r0 + per);
    // four rows per thread per pass keep several loads in flight
    for (int64_t base = r0; base < r1; base += 4 * kColThreads) {
        u64 key[4];
        int64_t row[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            row[j] = base + j * kColThreads + t;
            key[j] = row[j] < r1 ? coarse_key(dcf, row[j]) : kKeyEmpty;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool valid = row[j] < r1;
            const bool d = valid && (take_all || key[j] < lo);
            const bool b = valid && !d && key[j] < hi;
            warp_append(d, &ctl[kDirect], kMaxShortlist, direct, nullptr, row[j], 0, lane);
            warp_append(b, &ctl[kInBin], kBinCap, nullptr, bins, row[j], key[j], lane);
        }
    }
}

template <int CPL>
__global__ void __launch_bounds__(kSelThreads, 1)
    shortlist_kernel(const float* __restrict__ X, int D, int64_t n, const float* __restrict__ Q,
                     const float* __restrict__ dcall, const unsigned* __restrict__ hist, int S, int k,
                     const unsigned* __restrict__ ctl_all, const int* __restrict__ direct_all,
                     const u64* __restrict__ bin_all, int64_t* __restrict__ idx, float* __restrict__ dist) {
    extern __shared__ __align__(16) unsigned char smem[];
    u64* bin_keys = reinterpret_cast<u64*>(smem);                       // kBinCap
    int* short_rows = reinterpret_cast<int*>(bin_keys + kBinCap);       // kMaxShortlist
    unsigned* hsm = reinterpret_cast<unsigned*>(short_rows + kMaxShortlist);  // kBins
    u64* wl = reinterpret_cast<u64*>(hsm + kBins);                      // 32 warps x 32
    unsigned* ctl = reinterpret_cast<unsigned*>(wl + 32 * 32);          // control words
    unsigned* tmp = ctl + 8;                                            // 32 scan partials

    const int f = blockIdx.x;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const float* dcf = dcall + (size_t)f * n;
    const unsigned* gctl = ctl_all + (size_t)f * kCtl;
    const bool take_all = n <= S;
    const bool refine = !take_all && gctl[kRefine] != 0u;
    unsigned direct, need = 0, nb = 0;

    if (!refine) {
        // K2 collected the shortlist's rows below the boundary bin and the bin's keys
        direct = min(gctl[kDirect], (unsigned)kMaxShortlist);
        for (unsigned i = t; i < direct; i += blockDim.x) short_rows[i] = direct_all[(size_t)f * kMaxShortlist + i];
        if (!take_all) {
            need = gctl[kNeed];
            nb = min(gctl[kInBin], (unsigned)kBinCap);
            for (unsigned i = t; i < nb; i += blockDim.x) bin_keys[i] = bin_all[(size_t)f * kBinCap + i];
        }
    } else {
        // The boundary bin overflows: refine by further digits over the frame's keys.
        const int sel = (int)((int64_t)S < n ? (int64_t)S : n);
        need = (unsigned)sel;
        for (int i = t; i < kBins; i += blockDim.x) hsm[i] = hist[(size_t)f * kBins + i];
        __syncthreads();
        find_bin<kSelThreads>(hsm, need, ctl, tmp);
        int shift = 52;
        u64 lo = (u64)ctl[0] << shift;
        u64 hi = lo + (1ull << shift);
        need -= ctl[1];
        unsigned in_bin = ctl[2];
        while (in_bin > (unsigned)kBinCap && shift > 0) {
            const int nshift = shift >= 11 ? shift - 11 : 0;
            const int dbits = shift - nshift;
            __syncthreads();
            for (int i = t; i < kBins; i += blockDim.x) hsm[i] = 0u;
            __syncthreads();
            for (int64_t r = t; r < n; r += blockDim.x) {
                const u64 key = coarse_key(dcf, r);
                if (key >= lo && key < hi)
                    atomicAdd(&hsm[(unsigned)((key >> nshift) & ((1ull << dbits) - 1))], 1u);
            }
            __syncthreads();
            find_bin<kSelThreads>(hsm, need, ctl, tmp);
            lo += (u64)ctl[0] << nshift;
            hi = lo + (1ull << nshift);
            need -= ctl[1];
            in_bin = ctl[2];
            shift = nshift;
        }
        if (t == 0) {
            ctl[4] = 0u;
            ctl[5] = 0u;
        }
        __syncthreads();
        for (int64_t r = t; r < n; r += blockDim.x) {
            const u64 key = coarse_key(dcf, r);
            if (key < lo) {
                const unsigned pos = atomicAdd(&ctl[4], 1u);
                if (pos < (unsigned)kMaxShortlist) short_rows[pos] = (int)r;
            } else if (key < hi) {
                const unsigned pos = atomicAdd(&ctl[5], 1u);
                if (pos < (unsigned)kBinCap) bin_keys[pos] = key;
            }
        }
        __syncthreads();
        direct = min(ctl[4], (unsigned)kMaxShortlist);
        nb = min(ctl[5], (unsigned)kBinCap);
    }
    __syncthreads();
    if (!take_all) {
        unsigned p2 = 1;
        while (p2 < nb) p2 <<= 1;
        for (unsigned i = nb + t; i < p2; i += blockDim.x) bin_keys[i] = kKeyEmpty;
        __syncthreads();
        // bitonic sort of bin_keys[0, p2)
        for (unsigned size = 2; size <= p2; size <<= 1) {
            for (unsigned stride = size >> 1; stride > 0; stride >>= 1) {
                for (unsigned i = t; i < p2 / 2; i += blockDim.x) {
                    const unsigned lo_i = 2 * i - (i & (stride - 1));
                    const unsigned hi_i = lo_i + stride;
                    const bool up = ((lo_i & size) == 0);
                    const u64 a = bin_keys[lo_i], b = bin_keys[hi_i];
                    if ((a > b) == up) {
                        bin_keys[lo_i] = b;
                        bin_keys[hi_i] = a;
                    }
                }
                __syncthreads();
            }
        }
        need = min(need, nb);
        for (unsigned i = t; i < need && direct + i < (unsigned)kMaxShortlist; i += blockDim.x)
            short_rows[direct + i] = (int)key_row(bin_keys[i]);
        __syncthreads();
    }
    const int total = (int)min(direct + need, (unsigned)kMaxShortlist);

    // Re-rank on the full feature: warp per shortlisted row, four rows in flight.
    const int D4 = D / 4;
    float4 qv[CPL];
#pragma unroll
    for (int j = 0; j < CPL; ++j) {
        const int c = lane + 32 * j;
        qv[j] = c < D4 ? reinterpret_cast<const float4*>(Q + (size_t)f * D)[c] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const float2 neg1 = f2(-1.f, -1.f);
    u64 L = kKeyEmpty;
    u64 thr = kKeyEmpty;
    constexpr int kWarps = kSelThreads / 32;
    for (int i0 = warp; i0 < total; i0 += 4 * kWarps) {
        int r[4];
        float4 x[4][CPL];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = i0 + b * kWarps;
            r[b] = i < total ? short_rows[i] : -1;
#pragma unroll
            for (int j = 0; j < CPL; ++j) {
                const int c = lane + 32 * j;
                x[b][j] = (r[b] >= 0 && c < D4) ? __ldg(reinterpret_cast<const float4*>(X + (size_t)r[b] * D) + c)
                                                : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        float d[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            float2 acc = f2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < CPL; ++j) {
                float2 a = __ffma2_rn(f2(x[b][j].x, x[b][j].y), neg1, f2(qv[j].x, qv[j].y));
                float2 c2 = __ffma2_rn(f2(x[b][j].z, x[b][j].w), neg1, f2(qv[j].z, qv[j].w));
                acc = __ffma2_rn(a, a, acc);
                acc = __ffma2_rn(c2, c2, acc);
            }
            d[b] = acc.x + acc.y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int b = 0; b < 4; ++b) d[b] += __shfl_xor_sync(kFull, d[b], o);
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            if (r[b] < 0) continue;
            const u64 key = make_key(d[b], (uint32_t)r[b]);
            if (key < thr) {
                list_insert(L, key, k, lane);
                thr = __shfl_sync(kFull, L, k - 1);
            }
        }
    }
    wl[warp * 32 + lane] = L;
    __syncthreads();
    if (warp == 0) {
        u64 M = kKeyEmpty;
        list_merge_keys<false>(M, wl, 32 * 32, k, lane);
        if (lane < k) {
            const size_t o = (size_t)f * k + lane;
            if (M == kKeyEmpty) {
                idx[o] = -1;
                dist[o] = __int_as_float(0x7f800000);
            } else {
                idx[o] = (int64_t)key_row(M);
                dist[o] = key_dist(M);
            }
        }
    }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t shortlist_smem() {
    return kBinCap * sizeof(u64) + kMaxShortlist * sizeof(int) + kBins * sizeof(unsigned) + 32 * 32 * sizeof(u64) +
           (8 + 32) * sizeof(unsigned);
}

struct CoarseLayout {
    size_t dc, hist, ctl, direct, bins, total;
};

CoarseLayout layout(const lhr_db* db, int nq) {
    CoarseLayout L{};
    L.dc = 0;
    L.hist = align256((size_t)nq * db->n * sizeof(float));
    L.ctl = L.hist + (size_t)nq * kBins * sizeof(unsigned);  // hist and ctl are cleared together
    L.direct = align256(L.ctl + (size_t)nq * kCtl * sizeof(unsigned));
    L.bins = align256(L.direct + (size_t)nq * kMaxShortlist * sizeof(int));
    L.total = align256(L.bins + (size_t)nq * kBinCap * sizeof(u64));
    return L;
}

}  // namespace

size_t coarse_scratch_bytes(const lhr_db* db, int nq, int /*shortlist*/) { return layout(db, nq).total; }

namespace {
// One subspace's [nq][k] result (rows relative to the subspace's first internal
// row `off`) into slot s of the [nq][n_sub][k] output, in the caller's rows.
__global__ void subspace_remap_kernel(const int64_t* __restrict__ tidx, const float* __restrict__ tdist, int nq, int k,
                                      int n_sub, int s, int64_t off, const int32_t* __restrict__ perm,
                                      int64_t* __restrict__ idx, float* __restrict__ dist) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nq * k) return;
    const int f = i / k, j = i % k;
    const int64_t r = tidx[i];
    const size_t o = ((size_t)f * n_sub + s) * k + j;
    idx[o] = r < 0 ? -1 : (perm != nullptr ? (int64_t)perm[off + r] : off + r);
    dist[o] = tdist[i];
}
}  // namespace

cudaError_t launch_subspace_remap(const int64_t* tidx, const float* tdist, int nq, int k, int n_sub, int s, int64_t off,
                                  const int32_t* perm, int64_t* idx, float* dist, cudaStream_t stream) {
    const int n = nq * k;
    subspace_remap_kernel<<<(n + 255) / 256, 256, 0, stream>>>(tidx, tdist, nq, k, n_sub, s, off, perm, idx, dist);
    return cudaGetLastError();
}

cudaError_t launch_coarse(const lhr_db* db, const float* q, int nq, int shortlist, int k, int64_t* idx, float* dist,
                          void* scratch, cudaStream_t stream) {
    const CoarseLayout Lo = layout(db, nq);
    unsigned char* base = reinterpret_cast<unsigned char*>(scratch);
    float* dcbuf = reinterpret_cast<float*>(base + Lo.dc);
    unsigned* hist = reinterpret_cast<unsigned*>(base + Lo.hist);
    unsigned* ctl = reinterpret_cast<unsigned*>(base + Lo.ctl);
    int* direct = reinterpret_cast<int*>(base + Lo.direct);
    u64* bins = reinterpret_cast<u64*>(base + Lo.bins);
    cudaError_t e = cudaMemsetAsync(hist, 0, Lo.direct - Lo.hist, stream);
    if (e != cudaSuccess) return e;
    const int64_t nblk = (db->n + 255) / 256;
    dim3 g1((unsigned)std::min<int64_t>(nblk, (int64_t)db->sms * 2), (nq + kFB - 1) / kFB);
    const int dc4 = db->coarse_dim / 4;
#define LHR_CK(C)                                                                                                \
    do {                                                                                                         \
        const size_t csm = sizeof(float4) * kFB * (C) + sizeof(unsigned) * kFB * kBins;                          \
        e = cudaFuncSetAttribute(coarse_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm);       \
        if (e != cudaSuccess) return e;                                                                          \
        ProfScope ps("coarse_kernel", stream);                                                                   \
        coarse_kernel<C><<<g1, 256, csm, stream>>>(db->Xc, db->n, db->coarse_dim, q, db->dim, nq, dcbuf, hist); \
    } while (0)
    if (dc4 <= 8) LHR_CK(8);
    else if (dc4 <= 16) LHR_CK(16);
    else if (dc4 <= 32) LHR_CK(32);
    else return cudaErrorInvalidValue;
#undef LHR_CK
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    {
        ProfScope ps("collect_kernel", stream);
        collect_kernel<<<dim3(kParts, nq), kColThreads, 0, stream>>>(dcbuf, db->n, hist, shortlist, ctl, direct, bins);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const size_t sm = shortlist_smem();
    const int d4 = db->dim / 4;
    const int cpl = d4 <= 32 ? 1 : (d4 <= 64 ? 2 : 4);
#define LHR_SL(C)                                                                                            \
    do {                                                                                                     \
        e = cudaFuncSetAttribute(shortlist_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
        if (e != cudaSuccess) return e;                                                                      \
        ProfScope ps("shortlist_kernel", stream);                                                            \
        shortlist_kernel<C><<<nq, kSelThreads, sm, stream>>>(db->X, db->dim, db->n, q, dcbuf, hist,          \
                                                             shortlist, k, ctl, direct, bins, idx, dist);    \
    } while (0)
    if (cpl == 1) LHR_SL(1);
    else if (cpl == 2) LHR_SL(2);
    else LHR_SL(4);
#undef LHR_SL
    return cudaGetLastError();
}

}  // namespace lhr
