// The C ABI (include/lhr.h): argument validation on the host, the database
// handle, stream-ordered scratch, and dispatch to the kernels.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

namespace lhr {

static thread_local std::string g_last_error;

lhr_status fail(lhr_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

lhr_status cuda_fail(cudaError_t e, const char* what) {
    cudaGetLastError();  // clear a sticky launch error of this thread's context, if any
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(e == cudaErrorMemoryAllocation ? LHR_ERR_OOM : LHR_ERR_CUDA, m);
}

// One library-owned memory pool per device, kept warm (no release threshold),
// so per-call scratch is a stream-ordered sub-allocation, not a cudaMalloc.
static cudaError_t device_pool(int dev, cudaMemPool_t* out) {
    static std::mutex mu;
    static std::map<int, cudaMemPool_t> pools;
    std::lock_guard<std::mutex> lk(mu);
    auto it = pools.find(dev);
    if (it != pools.end()) {
        *out = it->second;
        return cudaSuccess;
    }
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool;
    cudaError_t e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    uint64_t thr = ~0ull;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    if (e != cudaSuccess) return e;
    pools[dev] = pool;
    *out = pool;
    return cudaSuccess;
}

cudaError_t Scratch::alloc(size_t bytes, cudaStream_t s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaMemPool_t pool;
    e = device_pool(dev, &pool);
    if (e != cudaSuccess) return e;
    stream = s;
    return cudaMallocFromPoolAsync(&ptr, std::max<size_t>(bytes, 256), pool, s);
}

void Scratch::release() {
    if (ptr) cudaFreeAsync(ptr, stream);
    ptr = nullptr;
}

// ---------------------------------------------------------------- profiling
namespace {
struct ProfRec {
    std::string name;
    cudaEvent_t a = nullptr, b = nullptr;
};
std::atomic<bool> g_prof{false};
std::mutex g_prof_mu;
std::vector<ProfRec> g_prof_recs;
}  // namespace

ProfScope::ProfScope(const char* kernel, cudaStream_t s) : stream(s) {
    if (!g_prof.load(std::memory_order_relaxed)) return;
    ProfRec r;
    r.name = kernel;
    if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) return;
    // under stream capture the pair becomes event-record nodes of the graph, re-recorded by every replay
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) cs = cudaStreamCaptureStatusNone;
    capturing = cs == cudaStreamCaptureStatusActive;
    if (capturing) cudaEventRecordWithFlags(r.a, s, cudaEventRecordExternal);
    else cudaEventRecord(r.a, s);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    slot = (int)g_prof_recs.size();
    g_prof_recs.push_back(r);
}

ProfScope::~ProfScope() {
    if (slot < 0) return;
    cudaEvent_t b;
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        b = g_prof_recs[slot].b;
    }
    if (capturing) cudaEventRecordWithFlags(b, stream, cudaEventRecordExternal);
    else cudaEventRecord(b, stream);
}

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

static bool is_device_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

static void free_db(lhr_db* db) {
    if (!db) return;
    void* bufs[] = {db->X, db->xnorm, db->Xc, db->perm, db->iperm, db->xy, db->tile, db->chunks, db->chunk_off,
                    db->Xb, db->snb, db->X8, db->sn8, db->Xb_s, db->snb_s, db->X8_s, db->sn8_s,
                    db->Xh, db->Xp, db->sub_p, db->err, db->hws};
    for (void* b : bufs)
        if (b) cudaFree(b);
    delete db->hws_map;
    delete db;
}

template <typename T>
static cudaError_t dalloc(T** p, size_t count) {
    return cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(count * sizeof(T), 16));
}

lhr_status check_query_params(const lhr_db* db, const lhr_query_params* p) {
    if (!p) return fail(LHR_ERR_INVALID_ARG, "query params are NULL");
    if (p->k < 1 || p->k > 32) return fail(LHR_ERR_INVALID_ARG, "k must be in [1, 32]");
    if (p->shortlist < 0) return fail(LHR_ERR_INVALID_ARG, "shortlist must be >= 0");
    if (p->score != LHR_F32 && p->score != LHR_BF16 && p->score != LHR_FP8_E4M3)
        return fail(LHR_ERR_INVALID_ARG, "unknown score dtype");
    if (p->shortlist > 0) {
        if (p->score != LHR_F32) return fail(LHR_ERR_INVALID_ARG, "coarse-to-fine scores are FP32");
        if (p->shortlist < p->k || p->shortlist > 4096)
            return fail(LHR_ERR_INVALID_ARG, "shortlist must be in [k, 4096]");
        if (!db->Xc) return fail(LHR_ERR_INVALID_ARG, "database was built without a coarse level (coarse_dim = 0)");
        for (int64_t rows : db->sub_rows_h)
            if (rows < p->shortlist)
                return fail(LHR_ERR_INVALID_ARG, "shortlist must not exceed the rows of any subspace");
    }
    if (p->score != LHR_F32) {
        if (p->rerank_width < p->k || p->rerank_width > 128)
            return fail(LHR_ERR_INVALID_ARG, "rerank_width must be in [k, 128]");
        if (db->n_sub != 1) return fail(LHR_ERR_INVALID_ARG, "low-precision scores need a single-subspace database");
        if (p->score == LHR_BF16 && !db->Xb) return fail(LHR_ERR_INVALID_ARG, "database has no BF16 copy");
        if (p->score == LHR_FP8_E4M3 && !db->X8) return fail(LHR_ERR_INVALID_ARG, "database has no FP8 copy");
    }
    return LHR_OK;
}

// Retrieval for `nq` frames into idx/dist ([nq][n_sub][k]).
lhr_status run_retrieval(const lhr_db* db, const float* q, int nq, const lhr_query_params* p, int64_t* idx,
                         float* dist, cudaStream_t s) {
    Scratch scr;
    cudaError_t e;
    if (p->score != LHR_F32) {
        const bool fp8 = p->score == LHR_FP8_E4M3;
        e = scr.alloc(lowp_scratch_bytes(db, nq, fp8, p->rerank_width), s);
        if (e != cudaSuccess) return cuda_fail(e, "scratch allocation");
        e = launch_lowp(db, q, nq, fp8, p->rerank_width, p->k, idx, dist, scr.ptr, s);
        if (e != cudaSuccess) return cuda_fail(e, "low-precision launch");
    } else if (p->shortlist > 0 && db->n_sub > 1) {
        // subspaces are searched independently (§3.1): the coarse-to-fine path over each
        // subspace's contiguous internal rows, its rows then mapped into slot s of the output
        int64_t off = 0;
        for (int s2 = 0; s2 < db->n_sub; ++s2) {
            lhr_db view = *db;
            const int64_t rows = db->sub_rows_h[s2];
            view.X = db->X + off * db->dim;
            view.Xc = db->Xc + off * db->coarse_dim;
            view.xnorm = db->xnorm + off;
            view.n = rows;
            view.n_sub = 1;
            view.perm = view.iperm = nullptr;
            const bool fused = hier_fused_eligible(&view, nq, p->shortlist);
            const size_t tbytes = ((size_t)nq * p->k * (sizeof(int64_t) + sizeof(float)) + 255) / 256 * 256;
            const size_t pbytes = fused ? hier_scratch_bytes(&view, nq) : coarse_scratch_bytes(&view, nq, p->shortlist);
            e = scr.alloc(tbytes + pbytes, s);
            if (e != cudaSuccess) return cuda_fail(e, "scratch allocation");
            int64_t* tidx = reinterpret_cast<int64_t*>(scr.ptr);
            float* tdist = reinterpret_cast<float*>(tidx + (size_t)nq * p->k);
            void* pscr = reinterpret_cast<unsigned char*>(scr.ptr) + tbytes;
            e = fused ? launch_hier_fused(&view, q, nq, p->shortlist, p->k, tidx, tdist, nullptr, pscr, s)
                      : launch_coarse(&view, q, nq, p->shortlist, p->k, tidx, tdist, pscr, s);
            if (e != cudaSuccess) return cuda_fail(e, "coarse-to-fine launch");
            e = launch_subspace_remap(tidx, tdist, nq, p->k, db->n_sub, s2, off, db->perm, idx, dist, s);
            if (e != cudaSuccess) return cuda_fail(e, "subspace remap launch");
            scr.release();
            off += rows;
        }
    } else if (p->shortlist > 0 && hier_fused_eligible(db, nq, p->shortlist)) {
        e = scr.alloc(hier_scratch_bytes(db, nq), s);
        if (e != cudaSuccess) return cuda_fail(e, "scratch allocation");
        e = launch_hier_fused(db, q, nq, p->shortlist, p->k, idx, dist, nullptr, scr.ptr, s);
        if (e != cudaSuccess) return cuda_fail(e, "fused coarse-to-fine launch");
    } else if (p->shortlist > 0) {
        e = scr.alloc(coarse_scratch_bytes(db, nq, p->shortlist), s);
        if (e != cudaSuccess) return cuda_fail(e, "scratch allocation");
        e = launch_coarse(db, q, nq, p->shortlist, p->k, idx, dist, scr.ptr, s);
        if (e != cudaSuccess) return cuda_fail(e, "coarse-to-fine launch");
    } else {
        e = scr.alloc(scan_scratch_bytes(db, nq, p->k, true), s);
        if (e != cudaSuccess) return cuda_fail(e, "scratch allocation");
        e = launch_scan(db, q, nq, p->k, idx, dist, scr.ptr, true, s);
        if (e != cudaSuccess) return cuda_fail(e, "scan launch");
    }
    return LHR_OK;
}

lhr_status check_agg_params(const lhr_agg_params* a) {
    if (!a) return fail(LHR_ERR_INVALID_ARG, "aggregation params are NULL");
    if (a->mode != LHR_AGG_TILE && a->mode != LHR_AGG_TILE_CENTROID && a->mode != LHR_AGG_SOFTMAX)
        return fail(LHR_ERR_INVALID_ARG, "unknown aggregation mode");
    if (a->top_c < 1) return fail(LHR_ERR_INVALID_ARG, "top_c must be >= 1");
    if (!(a->radius_m >= 0.0) || !isfinite(a->radius_m)) return fail(LHR_ERR_INVALID_ARG, "radius_m must be >= 0");
    if (a->toler_pct < 0 || a->toler_pct > 100) return fail(LHR_ERR_INVALID_ARG, "toler_pct must be in [0, 100]");
    if (a->mode == LHR_AGG_SOFTMAX && !(a->tau > 0.f && isfinite(a->tau)))
        return fail(LHR_ERR_INVALID_ARG, "tau must be > 0");
    return LHR_OK;
}

AggArgs make_agg(const lhr_db* db, const lhr_agg_params* a) {
    AggArgs g{};
    g.mode = (int)a->mode;
    g.top_c = a->top_c;
    g.toler_pct = a->toler_pct;
    g.r2max = circle_r2_limit(a->radius_m, db->tile_m);
    g.tau = a->tau;
    g.tile_m = db->tile_m;
    return g;
}

}  // namespace lhr

using namespace lhr;

extern "C" {

const char* lhr_last_error(void) { return g_last_error.c_str(); }

lhr_status lhr_build_db(const float* feats, const double* xy, const int32_t* subspace, int64_t n,
                        const lhr_db_config* cfg, void* cuda_stream, lhr_db** out) {
    if (!out) return fail(LHR_ERR_INVALID_ARG, "out is NULL");
    if (!feats || !xy || !cfg) return fail(LHR_ERR_INVALID_ARG, "feats, xy and cfg must be non-NULL");
    if (n < 1 || n >= (int64_t)1 << 31) return fail(LHR_ERR_INVALID_ARG, "n must be in [1, 2^31)");
    const int D = cfg->dim, Dc = cfg->coarse_dim;
    if (D < 4 || D > 512 || D % 4) return fail(LHR_ERR_INVALID_ARG, "dim must be a multiple of 4 in [4, 512]");
    if (Dc != 0 && (Dc < 4 || Dc > D || Dc % 4 || Dc > 128))
        return fail(LHR_ERR_INVALID_ARG, "coarse_dim must be 0 or a multiple of 4 in [4, min(dim, 128)]");
    if (cfg->lowp & ~(LHR_LOWP_BF16 | LHR_LOWP_FP8)) return fail(LHR_ERR_INVALID_ARG, "unknown lowp bits");
    if ((cfg->lowp & LHR_LOWP_BF16) && (D % 64 || D > 256))
        return fail(LHR_ERR_INVALID_ARG, "a BF16 copy needs dim % 64 == 0 and dim <= 256");
    if ((cfg->lowp & LHR_LOWP_FP8) && D % 128)
        return fail(LHR_ERR_INVALID_ARG, "an FP8 copy needs dim % 128 == 0");
    if (cfg->reserved != 0) return fail(LHR_ERR_INVALID_ARG, "reserved must be 0");
    if (!(cfg->tile_m > 0.0) || !isfinite(cfg->tile_m)) return fail(LHR_ERR_INVALID_ARG, "tile_m must be > 0");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);

    lhr_db* db = new (std::nothrow) lhr_db();
    if (!db) return fail(LHR_ERR_OOM, "host allocation");
    cudaError_t e = cudaGetDevice(&db->device);
    if (e != cudaSuccess) {
        delete db;
        return cuda_fail(e, "cudaGetDevice");
    }
    cudaDeviceGetAttribute(&db->sms, cudaDevAttrMultiProcessorCount, db->device);
    db->n = n;
    db->dim = D;
    db->coarse_dim = Dc;
    db->lowp = cfg->lowp;
    db->tile_m = cfg->tile_m;

    // Subspaces: stable grouping of rows by id.
    std::vector<int32_t> sub_h;
    std::vector<int32_t> perm_h;
    bool need_perm = false;
    if (subspace) {
        sub_h.resize(n);
        e = cudaMemcpy(sub_h.data(), subspace, n * sizeof(int32_t), cudaMemcpyDefault);
        if (e != cudaSuccess) {
            free_db(db);
            return cuda_fail(e, "copy subspace ids");
        }
        int32_t mx = 0;
        for (int64_t i = 0; i < n; ++i) {
            if (sub_h[i] < 0) {
                free_db(db);
                return fail(LHR_ERR_INVALID_ARG, "subspace ids must be >= 0");
            }
            mx = std::max(mx, sub_h[i]);
        }
        if (mx >= 65536) {
            free_db(db);
            return fail(LHR_ERR_INVALID_ARG, "at most 65536 subspaces");
        }
        db->n_sub = mx + 1;
        db->sub_rows_h.assign(db->n_sub, 0);
        for (int64_t i = 0; i < n; ++i) db->sub_rows_h[sub_h[i]]++;
        std::vector<int64_t> start(db->n_sub + 1, 0);
        for (int s2 = 0; s2 < db->n_sub; ++s2) start[s2 + 1] = start[s2] + db->sub_rows_h[s2];
        perm_h.resize(n);
        for (int64_t i = 0; i < n; ++i) {
            perm_h[start[sub_h[i]]++] = (int32_t)i;
            if (i > 0 && sub_h[i] < sub_h[i - 1]) need_perm = true;
        }
    } else {
        db->n_sub = 1;
        db->sub_rows_h.assign(1, n);
    }

    int32_t* flag = nullptr;
    float* tmp = nullptr;
    auto bail = [&](lhr_status st) {
        if (flag) cudaFree(flag);
        if (tmp) cudaFree(tmp);
        free_db(db);
        return st;
    };
    if ((e = dalloc(&db->X, (size_t)n * D)) != cudaSuccess) return bail(cuda_fail(e, "allocate features"));
    if ((e = dalloc(&db->xy, (size_t)n * 2)) != cudaSuccess) return bail(cuda_fail(e, "allocate xy"));
    if ((e = dalloc(&db->tile, (size_t)n * 2)) != cudaSuccess) return bail(cuda_fail(e, "allocate tiles"));
    if ((e = dalloc(&db->err, 1)) != cudaSuccess) return bail(cuda_fail(e, "allocate error word"));
    if ((e = dalloc(&flag, 3)) != cudaSuccess) return bail(cuda_fail(e, "allocate flag"));
    if ((e = dalloc(&db->xnorm, (size_t)n + kSnPad)) != cudaSuccess ||
        (e = cudaMemsetAsync(db->xnorm, 0, ((size_t)n + kSnPad) * sizeof(float), s)) != cudaSuccess)
        return bail(cuda_fail(e, "allocate norms"));
    if (Dc && (e = dalloc(&db->Xc, (size_t)n * Dc)) != cudaSuccess) return bail(cuda_fail(e, "allocate coarse slab"));
    if (Dc) {
        const size_t hb = kHierWsBlocks * hier_ws_block_bytes();
        if ((e = cudaMalloc(&db->hws, hb)) != cudaSuccess || (e = cudaMemsetAsync(db->hws, 0, hb, s)) != cudaSuccess)
            return bail(cuda_fail(e, "allocate fused-kernel control blocks"));
        db->hws_map = new (std::nothrow) HierWsMap();
        if (!db->hws_map) return bail(fail(LHR_ERR_OOM, "host allocation"));
    }
    if (cfg->lowp & LHR_LOWP_BF16) {
        if ((e = cudaMalloc(&db->Xb, (size_t)n * D * 2)) != cudaSuccess ||
            (e = dalloc(&db->snb, (size_t)n + kSnPad)) != cudaSuccess ||
            (e = cudaMemsetAsync(db->snb, 0, ((size_t)n + kSnPad) * sizeof(float2), s)) != cudaSuccess)
            return bail(cuda_fail(e, "allocate BF16 copy"));
    }
    if (half_copy_wanted(n, D) && (e = cudaMalloc(&db->Xh, (size_t)n * D * 2)) != cudaSuccess)
        return bail(cuda_fail(e, "allocate FP16 copy"));
    if (cfg->lowp & LHR_LOWP_FP8) {
        if ((e = cudaMalloc(&db->X8, (size_t)n * D)) != cudaSuccess ||
            (e = dalloc(&db->sn8, (size_t)n + kSnPad)) != cudaSuccess ||
            (e = cudaMemsetAsync(db->sn8, 0, ((size_t)n + kSnPad) * sizeof(float2), s)) != cudaSuccess)
            return bail(cuda_fail(e, "allocate FP8 copy"));
    }
    if (cfg->lowp && n >= (int64_t)kSampleStride * kSampleMinRows) {
        // every 64th row of each copy, for the pilot pass of the low-precision path
        db->sample_stride = kSampleStride;
        db->n_sample = (n + kSampleStride - 1) / kSampleStride;
        const size_t ns = (size_t)db->n_sample;
        if ((cfg->lowp & LHR_LOWP_BF16) &&
            ((e = cudaMalloc(&db->Xb_s, ns * D * 2)) != cudaSuccess ||
             (e = dalloc(&db->snb_s, ns + kSnPad)) != cudaSuccess ||
             (e = cudaMemsetAsync(db->snb_s, 0, (ns + kSnPad) * sizeof(float2), s)) != cudaSuccess))
            return bail(cuda_fail(e, "allocate BF16 sample"));
        if ((cfg->lowp & LHR_LOWP_FP8) &&
            ((e = cudaMalloc(&db->X8_s, ns * D)) != cudaSuccess ||
             (e = dalloc(&db->sn8_s, ns + kSnPad)) != cudaSuccess ||
             (e = cudaMemsetAsync(db->sn8_s, 0, (ns + kSnPad) * sizeof(float2), s)) != cudaSuccess))
            return bail(cuda_fail(e, "allocate FP8 sample"));
    }
    cudaMemsetAsync(db->err, 0, sizeof(int32_t), s);
    cudaMemsetAsync(flag, 0, 3 * sizeof(int32_t), s);
    const bool feats_dev = is_device_ptr(feats);
    if (need_perm) {
        if ((e = dalloc(&db->perm, (size_t)n)) != cudaSuccess) return bail(cuda_fail(e, "allocate perm"));
        cudaMemcpyAsync(db->perm, perm_h.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, s);
        std::vector<int32_t> iperm_h(n);
        for (int64_t i = 0; i < n; ++i) iperm_h[perm_h[i]] = (int32_t)i;
        if ((e = dalloc(&db->iperm, (size_t)n)) != cudaSuccess) return bail(cuda_fail(e, "allocate inverse perm"));
        cudaMemcpyAsync(db->iperm, iperm_h.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, s);
        // iperm_h is read by the copy: finish it before the vector goes out of scope
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return bail(cuda_fail(e, "copy inverse perm"));
        const float* src = feats;
        if (!feats_dev) {
            if ((e = dalloc(&tmp, (size_t)n * D)) != cudaSuccess) return bail(cuda_fail(e, "allocate staging"));
            cudaMemcpyAsync(tmp, feats, (size_t)n * D * sizeof(float), cudaMemcpyHostToDevice, s);
            src = tmp;
        }
        if ((e = launch_gather_rows(src, db->perm, n, D, db->X, s)) != cudaSuccess)
            return bail(cuda_fail(e, "gather rows"));
    } else {
        e = cudaMemcpyAsync(db->X, feats, (size_t)n * D * sizeof(float), cudaMemcpyDefault, s);
        if (e != cudaSuccess) return bail(cuda_fail(e, "copy features"));
    }
    e = cudaMemcpyAsync(db->xy, xy, (size_t)n * 2 * sizeof(double), cudaMemcpyDefault, s);
    if (e != cudaSuccess) return bail(cuda_fail(e, "copy xy"));
    if ((e = launch_check_finite(db->X, (int64_t)n * D, flag, s)) != cudaSuccess)
        return bail(cuda_fail(e, "finite check"));
    if ((e = launch_tiles(db->xy, n, db->tile_m, db->tile, flag, s)) != cudaSuccess)
        return bail(cuda_fail(e, "tiles"));

    // Scan partition: about one chunk per SM over the whole database, never
    // crossing a subspace boundary.
    int64_t cr = (n + db->sms - 1) / db->sms;
    cr = std::max<int64_t>(256, (cr + 15) / 16 * 16);  // small databases: fewer, longer chunks (short merge tail)
    db->chunk_rows = (int)cr;
    std::vector<int4> chunks;
    db->chunk_off_h.assign(db->n_sub + 1, 0);
    int64_t row = 0;
    for (int s2 = 0; s2 < db->n_sub; ++s2) {
        db->chunk_off_h[s2] = (int32_t)chunks.size();
        const int64_t end = row + db->sub_rows_h[s2];
        for (int64_t r = row; r < end; r += cr) chunks.push_back(make_int4((int)r, (int)std::min(end, r + cr), s2, 0));
        row = end;
    }
    db->chunk_off_h[db->n_sub] = (int32_t)chunks.size();
    db->nchunks = (int)chunks.size();
    if ((e = dalloc(&db->chunks, chunks.size())) != cudaSuccess) return bail(cuda_fail(e, "allocate chunks"));
    if ((e = dalloc(&db->chunk_off, db->chunk_off_h.size())) != cudaSuccess)
        return bail(cuda_fail(e, "allocate chunk offsets"));
    cudaMemcpyAsync(db->chunks, chunks.data(), chunks.size() * sizeof(int4), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(db->chunk_off, db->chunk_off_h.data(), db->chunk_off_h.size() * sizeof(int32_t),
                    cudaMemcpyHostToDevice, s);
    if (n >= kPilotMinRows) {
        // Pilot sample of the exhaustive scan: internal rows j * 64, each with
        // the subspace of its row (subspaces are contiguous in internal order).
        db->n_pilot = (n + kSampleStride - 1) / kSampleStride;
        std::vector<int32_t> sub_p(db->n_pilot);
        int64_t r0 = 0;
        for (int s2 = 0; s2 < db->n_sub; ++s2) {
            const int64_t r1 = r0 + db->sub_rows_h[s2];
            for (int64_t j = (r0 + kSampleStride - 1) / kSampleStride; j * kSampleStride < r1; ++j) sub_p[j] = s2;
            r0 = r1;
        }
        if ((e = dalloc(&db->Xp, (size_t)db->n_pilot * D)) != cudaSuccess ||
            (e = dalloc(&db->sub_p, (size_t)db->n_pilot)) != cudaSuccess)
            return bail(cuda_fail(e, "allocate pilot sample"));
        e = cudaMemcpyAsync(db->sub_p, sub_p.data(), sub_p.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
        // sub_p is read by the copy: finish it before the vector goes out of scope
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return bail(cuda_fail(e, "pilot sample"));
    }
    if ((e = launch_build_derived(db, s)) != cudaSuccess) return bail(cuda_fail(e, "derived arrays"));
    if ((e = launch_norms(db, reinterpret_cast<unsigned*>(flag + 1), s)) != cudaSuccess)
        return bail(cuda_fail(e, "norms"));
    if ((e = launch_pilot_sample(db, s)) != cudaSuccess) return bail(cuda_fail(e, "pilot sample"));
    if ((e = launch_half_copy(db, reinterpret_cast<unsigned*>(flag + 2), s)) != cudaSuccess)
        return bail(cuda_fail(e, "FP16 copy"));
    int32_t flag_h2[3] = {0, 0, 0};
    cudaMemcpyAsync(flag_h2, flag, 3 * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return bail(cuda_fail(e, "build"));
    if ((e = cudaGetLastError()) != cudaSuccess) return bail(cuda_fail(e, "build"));
    const int32_t flag_h = flag_h2[0];
    std::memcpy(&db->xnorm_max, &flag_h2[1], sizeof(float));
    if (db->Xh) {
        // the scale the copy kernel derived from the same maximum
        float amax;
        std::memcpy(&amax, &flag_h2[2], sizeof(float));
        int ex = 0;
        std::frexp(amax, &ex);
        db->xh_scale = std::ldexp(1.0f, 15 - ex);
    }
    if (flag_h & 1) return bail(fail(LHR_ERR_INVALID_ARG, "features contain a non-finite value"));
    if (flag_h & 2) return bail(fail(LHR_ERR_INVALID_ARG, "xy contains a non-finite value or a tile outside int32"));
    cudaFree(flag);
    flag = nullptr;
    if (tmp) {
        cudaFree(tmp);
        tmp = nullptr;
    }
    *out = db;
    return LHR_OK;
}

lhr_status lhr_free_db(lhr_db* db) {
    if (!db) return LHR_OK;
    DeviceGuard g(db->device);
    cudaDeviceSynchronize();
    free_db(db);
    return LHR_OK;
}

lhr_status lhr_db_info(const lhr_db* db, int64_t* n, int32_t* dim, int32_t* coarse_dim, int32_t* n_subspaces) {
    if (!db) return fail(LHR_ERR_INVALID_ARG, "db is NULL");
    if (n) *n = db->n;
    if (dim) *dim = db->dim;
    if (coarse_dim) *coarse_dim = db->coarse_dim;
    if (n_subspaces) *n_subspaces = db->n_sub;
    return LHR_OK;
}

lhr_status lhr_query(const lhr_db* db, const float* q, int32_t nq, const lhr_query_params* p, int64_t* idx,
                     float* dist, void* cuda_stream) {
    if (!db) return fail(LHR_ERR_INVALID_ARG, "db is NULL");
    if (!q || !idx || !dist) return fail(LHR_ERR_INVALID_ARG, "q, idx and dist must be non-NULL");
    if (reinterpret_cast<uintptr_t>(q) % 16) return fail(LHR_ERR_INVALID_ARG, "q must be 16-byte aligned");
    if (nq < 1) return fail(LHR_ERR_INVALID_ARG, "nq must be >= 1");
    lhr_status st = check_query_params(db, p);
    if (st != LHR_OK) return st;
    DeviceGuard g(db->device);
    return run_retrieval(db, q, nq, p, idx, dist, reinterpret_cast<cudaStream_t>(cuda_stream));
}

lhr_status lhr_query_window(const lhr_db* db, const float* frames, const int32_t* offsets, int32_t W, int32_t nw,
                            const lhr_query_params* p, const lhr_agg_params* a, int64_t* idx, float* dist,
                            double* xy, int32_t* status, void* cuda_stream) {
    if (!db) return fail(LHR_ERR_INVALID_ARG, "db is NULL");
    if (!frames || !offsets || !idx || !dist || !xy || !status)
        return fail(LHR_ERR_INVALID_ARG, "frames, offsets, idx, dist, xy and status must be non-NULL");
    if (reinterpret_cast<uintptr_t>(frames) % 16) return fail(LHR_ERR_INVALID_ARG, "frames must be 16-byte aligned");
    if (W < 1 || nw < 1) return fail(LHR_ERR_INVALID_ARG, "W and nw must be >= 1");
    lhr_status st = check_query_params(db, p);
    if (st != LHR_OK) return st;
    if ((st = check_agg_params(a)) != LHR_OK) return st;
    DeviceGuard g(db->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    if (p->score == LHR_F32 && p->shortlist > 0 && nw <= W && hier_fused_eligible(db, W, p->shortlist)) {
        // the whole request -- retrieval and Algorithm 2 -- in one cooperative launch
        AggArgs ag = make_agg(db, a);
        ag.idx = idx;
        ag.dist = dist;
        ag.offsets = offsets;
        ag.per_frame = p->k;
        ag.limit = (long long)W * p->k;
        ag.nw = nw;
        ag.xy_out = xy;
        ag.status = status;
        Scratch scr;
        cudaError_t e = scr.alloc(hier_scratch_bytes(db, W), s);
        if (e != cudaSuccess) return cuda_fail(e, "scratch allocation");
        e = launch_hier_fused(db, frames, W, p->shortlist, p->k, idx, dist, &ag, scr.ptr, s);
        if (e != cudaSuccess) return cuda_fail(e, "fused coarse-to-fine launch");
        return LHR_OK;
    }
    if ((st = run_retrieval(db, frames, W, p, idx, dist, s)) != LHR_OK) return st;
    AggArgs ag = make_agg(db, a);
    ag.idx = idx;
    ag.dist = dist;
    ag.offsets = offsets;
    ag.per_frame = db->n_sub * p->k;
    ag.limit = (long long)W * ag.per_frame;
    ag.nw = nw;
    ag.xy_out = xy;
    ag.status = status;
    cudaError_t e = launch_aggregate(db, ag, s);
    if (e != cudaSuccess) return cuda_fail(e, "aggregation launch");
    return LHR_OK;
}

lhr_status lhr_aggregate_2d(const lhr_db* db, const int64_t* idx, const float* dist, int64_t n_cand,
                            const int32_t* cand_offsets, int32_t nw, const lhr_agg_params* a, double* xy,
                            int32_t* status, void* cuda_stream) {
    if (!db) return fail(LHR_ERR_INVALID_ARG, "db is NULL");
    if (!idx || !cand_offsets || !xy || !status)
        return fail(LHR_ERR_INVALID_ARG, "idx, cand_offsets, xy and status must be non-NULL");
    if (n_cand < 1 || nw < 1) return fail(LHR_ERR_INVALID_ARG, "n_cand and nw must be >= 1");
    lhr_status st = check_agg_params(a);
    if (st != LHR_OK) return st;
    if (a->mode == LHR_AGG_SOFTMAX && !dist) return fail(LHR_ERR_INVALID_ARG, "softmax mode needs dist");
    DeviceGuard g(db->device);
    AggArgs ag = make_agg(db, a);
    ag.idx = idx;
    ag.dist = dist;
    ag.offsets = cand_offsets;
    ag.per_frame = 0;
    ag.limit = n_cand;
    ag.nw = nw;
    ag.xy_out = xy;
    ag.status = status;
    cudaError_t e = launch_aggregate(db, ag, reinterpret_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return cuda_fail(e, "aggregation launch");
    return LHR_OK;
}

// ---------------------------------------------------------------- soft retrieval
static lhr_status check_soft(const lhr_db* db, int32_t k, const float* w, const float* tau) {
    if (!db) return fail(LHR_ERR_INVALID_ARG, "db is NULL");
    if (!w || !tau) return fail(LHR_ERR_INVALID_ARG, "w and tau must be non-NULL");
    if (reinterpret_cast<uintptr_t>(w) % 16) return fail(LHR_ERR_INVALID_ARG, "w must be 16-byte aligned");
    if (k < 1 || k > 32) return fail(LHR_ERR_INVALID_ARG, "k must be in [1, 32]");
    if (db->dim > 1024) return fail(LHR_ERR_UNSUPPORTED, "soft retrieval supports D <= 1024");
    if ((int64_t)db->n_sub * k > 1024) return fail(LHR_ERR_UNSUPPORTED, "soft retrieval supports n_s * k <= 1024");
    return LHR_OK;
}

lhr_status lhr_query_weighted(const lhr_db* db, const float* q, int32_t nq, int32_t k, const float* w,
                              int64_t* idx, float* dist, void* cuda_stream) {
    if (!db) return fail(LHR_ERR_INVALID_ARG, "db is NULL");
    if (!q || !w || !idx || !dist) return fail(LHR_ERR_INVALID_ARG, "q, w, idx and dist must be non-NULL");
    if (reinterpret_cast<uintptr_t>(q) % 16 || reinterpret_cast<uintptr_t>(w) % 16)
        return fail(LHR_ERR_INVALID_ARG, "q and w must be 16-byte aligned");
    if (nq < 1) return fail(LHR_ERR_INVALID_ARG, "nq must be >= 1");
    if (k < 1 || k > 32) return fail(LHR_ERR_INVALID_ARG, "k must be in [1, 32]");
    DeviceGuard g(db->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    Scratch scr;
    cudaError_t e = scr.alloc(scan_weighted_scratch_bytes(db, nq, k), s);
    if (e != cudaSuccess) return cuda_fail(e, "scratch allocation");
    e = launch_scan_weighted(db, q, nq, k, w, idx, dist, scr.ptr, s);
    if (e != cudaSuccess) return cuda_fail(e, "weighted scan launch");
    return LHR_OK;
}

lhr_status lhr_soft_forward(const lhr_db* db, const float* frames, const int32_t* offsets, int32_t W, int32_t nw,
                            int32_t k, const float* w, const float* tau, int64_t* idx, float* dist, double* p,
                            double* yhat, void* cuda_stream) {
    lhr_status st = check_soft(db, k, w, tau);
    if (st != LHR_OK) return st;
    if (!frames || !offsets || !idx || !dist || !p || !yhat)
        return fail(LHR_ERR_INVALID_ARG, "frames, offsets, idx, dist, p and yhat must be non-NULL");
    if (reinterpret_cast<uintptr_t>(frames) % 16) return fail(LHR_ERR_INVALID_ARG, "frames must be 16-byte aligned");
    if (W < 1 || nw < 1) return fail(LHR_ERR_INVALID_ARG, "W and nw must be >= 1");
    DeviceGuard g(db->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    Scratch scr;
    cudaError_t e = scr.alloc(scan_weighted_scratch_bytes(db, W, k), s);
    if (e != cudaSuccess) return cuda_fail(e, "scratch allocation");
    if ((e = launch_scan_weighted(db, frames, W, k, w, idx, dist, scr.ptr, s)) != cudaSuccess)
        return cuda_fail(e, "weighted scan launch");
    if ((e = launch_soft_forward(db, frames, offsets, W, nw, k, w, tau, idx, dist, p, yhat, s)) != cudaSuccess)
        return cuda_fail(e, "soft forward launch");
    return LHR_OK;
}

lhr_status lhr_soft_backward(const lhr_db* db, const float* frames, const int32_t* offsets, int32_t W, int32_t nw,
                             int32_t k, const float* w, const float* tau, const int64_t* idx, const float* dist,
                             const double* p, const double* yhat, const double* g_yhat, float* dq, float* dw,
                             float* dtau, void* cuda_stream) {
    lhr_status st = check_soft(db, k, w, tau);
    if (st != LHR_OK) return st;
    if (!frames || !offsets || !idx || !dist || !p || !yhat || !g_yhat || !dq || !dw || !dtau)
        return fail(LHR_ERR_INVALID_ARG, "every array argument must be non-NULL");
    if (W < 1 || nw < 1) return fail(LHR_ERR_INVALID_ARG, "W and nw must be >= 1");
    DeviceGuard g(db->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    Scratch scr;
    cudaError_t e = scr.alloc(soft_backward_scratch_bytes(db, nw), s);
    if (e != cudaSuccess) return cuda_fail(e, "scratch allocation");
    e = launch_soft_backward(db, frames, offsets, W, nw, k, w, tau, idx, dist, p, yhat, g_yhat, dq, dw, dtau, scr.ptr,
                             s);
    if (e != cudaSuccess) return cuda_fail(e, "soft backward launch");
    return LHR_OK;
}

lhr_status lhr_loc_mse(const double* yhat, const double* y, int32_t nw, const double* scale, double* loss,
                       double* grad, void* cuda_stream) {
    if (!yhat || !y) return fail(LHR_ERR_INVALID_ARG, "yhat and y must be non-NULL");
    if (!loss && !grad) return fail(LHR_ERR_INVALID_ARG, "ask for the loss, the gradient or both");
    if (nw < 1) return fail(LHR_ERR_INVALID_ARG, "nw must be >= 1");
    cudaError_t e = launch_loc_mse(yhat, y, nw, scale, loss, grad, reinterpret_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return cuda_fail(e, "location loss launch");
    return LHR_OK;
}

lhr_status lhr_profile_enable(int32_t on) {
    g_prof.store(on != 0);
    return LHR_OK;
}

lhr_status lhr_profile_read(const char* kernel, int64_t* launches, double* total_ms, int32_t reset) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    int64_t cnt = 0;
    double tot = 0.0;
    std::vector<ProfRec> keep;
    for (ProfRec& r : g_prof_recs) {
        const bool match = kernel == nullptr || r.name.find(kernel) != std::string::npos;
        if (match) {
            float ms = 0.f;
            if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
                ++cnt;
                tot += ms;
            } else {
                cudaGetLastError();
            }
        }
        if (match && reset) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        } else {
            keep.push_back(r);
        }
    }
    if (reset) g_prof_recs.swap(keep);
    if (launches) *launches = cnt;
    if (total_ms) *total_ms = tot;
    return LHR_OK;
}

lhr_status lhr_db_error(const lhr_db* db, int32_t* err, void* cuda_stream) {
    if (!db || !err) return fail(LHR_ERR_INVALID_ARG, "db and err must be non-NULL");
    DeviceGuard g(db->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    int32_t h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, db->err, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(db->err, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "read error word");
    *err = h;
    return LHR_OK;
}

}  // extern "C"
