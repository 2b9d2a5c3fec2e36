// Exhaustive FP32 scan with fused per-frame, per-subspace top-N (§3.1,
// Algorithm 1: calculateDistance for every (query frame, database frame) pair,
// then selectTopCandidates; §4: Euclidean distance, top N).
//
// Design (GB300): the database is memory-bound work for a handful of query
// frames, so every byte of it is read once per launch.
//   * One CTA per (row chunk, query block). A row chunk is a contiguous range
//     of one subspace; the chunk table is built with the database.
//   * A producer thread streams the chunk through shared memory with 1-D bulk
//     copies (cp.async.bulk, 16 rows per stage) into an mbarrier ring; each
//     consumer warp owns the stages s with s % warps == warp, so its parity
//     waits always see consecutive phases.
//   * Lanes split the feature dimensions (float4 chunks, conflict-free), the
//     block's QB query frames sit in registers, and (q - x)^2 runs as packed
//     FP32 pairs (FFMA2). A 5-step butterfly transpose-reduce leaves lane l
//     with the full distance of (row l / QB, query l % QB): 31 shuffles for 32
//     distances.
//   * Each warp keeps, per query, a sorted top-k list in registers (lane i
//     holds the i-th key); a ballot against the list's k-th key rejects almost
//     every distance with one compare. The distance matrix never leaves the SM.
//   * Warp lists merge into a per-CTA list written to scratch; the last CTA of
//     a query block (atomic ticket) merges every chunk of each subspace and
//     writes the final lists. One launch per call.
#include <mutex>
#include <string>

#include "common.cuh"
#include "internal.h"

namespace lhr {
namespace {

constexpr int kRowsPerStage = 16;
constexpr int kMaxSmem = 227 * 1024;

struct ScanParams {
    const float* X;
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
    u64* partial;        // [qblock][QB][nchunks][k]
    unsigned* counters;  // [qblock]
    int64_t* idx;        // [nq][n_sub][k]
    float* dist;
    int* err;
};

struct ScanConfig {
    int qb, cpl, warps, stages;
    size_t smem;
};

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

template <int QB, int CPL>
__global__ void __launch_bounds__(288, 1) scan_topk_kernel(const ScanParams p) {
    constexpr int RW = 32 / QB;  // rows per reduction round
    extern __shared__ __align__(128) unsigned char smem[];
    const int warps = blockDim.x / 32 - 1;  // consumer warps; the last warp produces
    const int warp = threadIdx.x / 32;
    const int lane = threadIdx.x % 32;
    const int D4 = p.D / 4;
    const int NS = p.stages;
    const size_t stage_floats = (size_t)kRowsPerStage * p.D;

    float* stage_buf = reinterpret_cast<float*>(smem);
    u64* full = reinterpret_cast<u64*>(smem + NS * stage_floats * sizeof(float));
    u64* empty = full + NS;
    u64* lists = empty + NS;  // [warps][QB][32]
    int* flags = reinterpret_cast<int*>(lists + (size_t)warps * QB * 32);
    volatile int* abort_flag = flags;

    const int chunk = blockIdx.x;
    const int qblock = blockIdx.y;
    const int4 ch = p.chunks[chunk];
    const int row0 = ch.x, row1 = ch.y;
    const int iters = (row1 - row0 + kRowsPerStage - 1) / kRowsPerStage;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        flags[0] = 0;
        flags[1] = 0;
        fence_mbar_init();
    }
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
                const int r = row0 + it * kRowsPerStage;
                const int nr = min(kRowsPerStage, row1 - r);
                const uint32_t bytes = (uint32_t)nr * (uint32_t)p.D * 4u;
                mbar_arrive_expect_tx(&full[s], bytes);
                bulk_g2s(stage_buf + s * stage_floats, p.X + (size_t)r * p.D, bytes, &full[s]);
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
#pragma unroll
        for (int q = 0; q < QB; ++q) {
            const int qi = qblock * QB + q;
#pragma unroll
            for (int j = 0; j < CPL; ++j) {
                const int c = lane + 32 * j;
                qreg[q][j] = (qi < p.nq && c < D4)
                                 ? reinterpret_cast<const float4*>(p.Q)[(size_t)qi * D4 + c]
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        u64 L[QB];
#pragma unroll
        for (int q = 0; q < QB; ++q) L[q] = kKeyEmpty;
        u64 thr = kKeyEmpty;  // k-th key of the list of query (lane % QB)
        const bool q_valid = (qblock * QB + (lane % QB)) < p.nq;
        const float2 neg1 = f2(-1.f, -1.f);

        for (int it = warp; it < iters; it += warps) {
            const int s = it % NS;
            const uint32_t ph = (uint32_t)(it / NS) & 1u;
            if (!mbar_wait(&full[s], ph, abort_flag)) {
                if (lane == 0) {
                    *abort_flag = 1;
                    record_error(p.err, kErrTimeout);
                }
                break;
            }
            const float4* sb = reinterpret_cast<const float4*>(stage_buf + s * stage_floats);
            const int rbase = row0 + it * kRowsPerStage;
            const int nr = min(kRowsPerStage, row1 - rbase);
#pragma unroll 1
            for (int rb = 0; rb < kRowsPerStage; rb += RW) {
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
                            float2 d0 = __ffma2_rn(f2(x[j].x, x[j].y), neg1, f2(qreg[q][j].x, qreg[q][j].y));
                            float2 d1 = __ffma2_rn(f2(x[j].z, x[j].w), neg1, f2(qreg[q][j].z, qreg[q][j].w));
                            acc = __ffma2_rn(d0, d0, acc);
                            acc = __ffma2_rn(d1, d1, acc);
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
                const u64 key = (q_valid && rl < nr) ? make_key(part[0], (uint32_t)(rbase + rl)) : kKeyEmpty;
                unsigned m = __ballot_sync(kFull, key < thr);
                while (m) {
                    const int j = __ffs(m) - 1;
                    m &= m - 1;
                    const u64 kj = __shfl_sync(kFull, key, j);
                    const int qj = j % QB;
                    u64 t = kKeyEmpty;
#pragma unroll
                    for (int q = 0; q < QB; ++q) {
                        if (q == qj) {
                            list_insert(L[q], kj, p.k, lane);
                            t = __shfl_sync(kFull, L[q], p.k - 1);
                        }
                    }
                    if ((lane % QB) == qj) thr = t;
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
        }
#pragma unroll
        for (int q = 0; q < QB; ++q) lists[((size_t)warp * QB + q) * 32 + lane] = L[q];
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
    for (int pair = warp; pair < QB * p.n_sub; pair += nwarps) {
        const int q = pair / p.n_sub;
        const int sub = pair % p.n_sub;
        const int qi = qblock * QB + q;
        if (qi >= p.nq) continue;
        const int c0 = p.chunk_off[sub], c1 = p.chunk_off[sub + 1];
        u64 M = kKeyEmpty;
        list_merge_keys<true>(M, p.partial + (((size_t)qblock * QB + q) * p.nchunks + c0) * p.k, (c1 - c0) * p.k,
                              p.k, lane);
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
    if (threadIdx.x == 0) p.counters[qblock] = 0u;
}

ScanConfig choose_config(const lhr_db* db, int nq) {
    ScanConfig c{};
    const int d4 = db->dim / 4;
    c.cpl = d4 <= 32 ? 1 : (d4 <= 64 ? 2 : 4);
    const int qb_max = 16 / c.cpl;
    int qb = 2;
    while (qb < nq && qb < qb_max) qb *= 2;
    c.qb = qb;
    const size_t stage_bytes = (size_t)kRowsPerStage * db->dim * sizeof(float);
    const int warps_pref = 8;
    // shared memory: stages + 2 barriers per stage + lists + flags
    for (int w = warps_pref; w >= 1; --w) {
        const size_t lists = (size_t)w * qb * 32 * sizeof(u64);
        const size_t budget = kMaxSmem - 1024 - lists;
        int ns = (int)(budget / (stage_bytes + 16));
        ns = (ns / w) * w;
        if (ns >= 2 * w) {
            c.warps = w;
            c.stages = ns;
            c.smem = ns * stage_bytes + 2 * ns * sizeof(u64) + lists + 16;
            return c;
        }
    }
    c.warps = 1;
    c.stages = 2;
    c.smem = 2 * stage_bytes + 4 * sizeof(u64) + (size_t)qb * 32 * sizeof(u64) + 16;
    return c;
}

template <int QB, int CPL>
cudaError_t launch_t(const ScanConfig& c, const ScanParams& p, int nqb, cudaStream_t stream) {
    auto kern = scan_topk_kernel<QB, CPL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem);
    if (e != cudaSuccess) return e;
    dim3 grid(p.nchunks, nqb);
    ProfScope ps("scan_topk_kernel", stream);
    kern<<<grid, (c.warps + 1) * 32, c.smem, stream>>>(p);
    return cudaGetLastError();
}

}  // namespace

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t scan_scratch_bytes(const lhr_db* db, int nq, int k) {
    const ScanConfig c = choose_config(db, nq);
    const size_t nqb = (nq + c.qb - 1) / c.qb;
    return align256(nqb * c.qb * (size_t)db->nchunks * k * sizeof(u64)) + align256(nqb * sizeof(unsigned));
}

cudaError_t launch_scan(const lhr_db* db, const float* q, int nq, int k, int64_t* idx, float* dist, void* scratch,
                        cudaStream_t stream) {
    const ScanConfig c = choose_config(db, nq);
    const int nqb = (nq + c.qb - 1) / c.qb;
    ScanParams p{};
    p.X = db->X;
    p.D = db->dim;
    p.chunks = db->chunks;
    p.nchunks = db->nchunks;
    p.chunk_off = db->chunk_off;
    p.n_sub = db->n_sub;
    p.perm = db->perm;
    p.Q = q;
    p.nq = nq;
    p.k = k;
    p.stages = c.stages;
    p.partial = reinterpret_cast<u64*>(scratch);
    const size_t part_bytes = align256((size_t)nqb * c.qb * db->nchunks * k * sizeof(u64));
    p.counters = reinterpret_cast<unsigned*>(reinterpret_cast<unsigned char*>(scratch) + part_bytes);
    p.idx = idx;
    p.dist = dist;
    p.err = db->err;
    cudaError_t e = cudaMemsetAsync(p.counters, 0, nqb * sizeof(unsigned), stream);
    if (e != cudaSuccess) return e;
    switch (c.cpl * 100 + c.qb) {
        case 102: return launch_t<2, 1>(c, p, nqb, stream);
        case 104: return launch_t<4, 1>(c, p, nqb, stream);
        case 108: return launch_t<8, 1>(c, p, nqb, stream);
        case 116: return launch_t<16, 1>(c, p, nqb, stream);
        case 202: return launch_t<2, 2>(c, p, nqb, stream);
        case 204: return launch_t<4, 2>(c, p, nqb, stream);
        case 208: return launch_t<8, 2>(c, p, nqb, stream);
        case 402: return launch_t<2, 4>(c, p, nqb, stream);
        case 404: return launch_t<4, 4>(c, p, nqb, stream);
        default: return cudaErrorInvalidConfiguration;
    }
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
    const size_t need = scan_scratch_bytes(db, nq, k);
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
        e = launch_scan(db, q, nq, k, idx, dist, scratch, reinterpret_cast<cudaStream_t>(cuda_stream));
    if (prev != db->device) cudaSetDevice(prev);
    if (e != cudaSuccess) return cuda_fail(e, "lhr_query_static");
    return LHR_OK;
}
