// Host-side internals shared by the library's translation units: the
// database handle, scratch allocation, and the launchers each kernel file
// exports to the C ABI layer.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/lhr.h"

constexpr int kSnPad = 256;
constexpr int kSampleStride = 64;     // pilot sample: every 64th row
constexpr int kSampleMinRows = 4096;  // sample only databases of at least 64 x 4096 rows
constexpr int64_t kPilotMinRows = 65536;  // exhaustive-scan pilot sample for databases of at least this many rows
constexpr int kHierWsBlocks = 8;          // streams that get a persistent control block of the fused kernel

// Which stream holds which control block of the fused coarse-to-fine kernel
// (the first kHierWsBlocks streams that call it, for the handle's lifetime).
struct HierWsMap {
    std::mutex mu;
    cudaStream_t owner[kHierWsBlocks] = {};
    bool used[kHierWsBlocks] = {};
};

struct lhr_db {
    int device = 0;
    int64_t n = 0;
    int dim = 0;
    int coarse_dim = 0;
    uint32_t lowp = 0;
    double tile_m = 0.3;
    int n_sub = 1;
    int sms = 1;  // multiprocessors of `device`

    // Rows in internal order: grouped by subspace (stable), so each subspace is
    // one contiguous range. perm[i] is the caller's row of internal row i
    // (nullptr when the order is the caller's).
    float* X = nullptr;         // n x dim
    float* xnorm = nullptr;     // n + kSnPad: FP32 ||x||^2 per row (internal order), zero padded
    float xnorm_max = 0.f;      // max over rows of ||x||^2
    float* Xc = nullptr;        // n x coarse_dim (coarse prefix slab), or nullptr
    int32_t* perm = nullptr;    // n, or nullptr
    int32_t* iperm = nullptr;   // n: internal row of each caller row, or nullptr (with perm)
    // Caller's order.
    double* xy = nullptr;       // n x 2
    int32_t* tile = nullptr;    // n x 2 (tx, ty) = floor(xy / tile_m)

    // Scan partition: chunk c covers internal rows [chunks[c].x, chunks[c].y) of
    // subspace chunks[c].z; chunks of subspace s are [chunk_off[s], chunk_off[s+1]).
    int nchunks = 0;
    int chunk_rows = 0;
    int4* chunks = nullptr;
    int32_t* chunk_off = nullptr;
    std::vector<int32_t> chunk_off_h;
    std::vector<int64_t> sub_rows_h;  // rows per subspace

    // Low-precision copies (internal order) and, per row, (FP32 scale s,
    // FP32 norm s^2 ||x^||^2 of the quantised row); the (s, norm) arrays carry
    // kSnPad rows of zero padding so whole-tile bulk copies stay in bounds.
    void* Xb = nullptr;   float2* snb = nullptr;   // BF16
    void* X8 = nullptr;   float2* sn8 = nullptr;   // FP8 e4m3
    // Every sample_stride-th row of each copy (rows 0, stride, 2 stride, ...),
    // n_sample rows, with its (s, norm) pairs: the pilot pass that sets the
    // low-precision path's per-query score threshold runs over these.
    int sample_stride = 1;
    int64_t n_sample = 0;
    void* Xb_s = nullptr; float2* snb_s = nullptr;
    void* X8_s = nullptr; float2* sn8_s = nullptr;

    // FP16 copy (internal order) of X * xh_scale, xh_scale = 2^(15 - e) for
    // max |x| = f 2^e, f in [0.5, 1) (so every scaled value is below 2^15 in
    // magnitude): the operand of the many-frame path's tensor-core filter.
    // Present when half_copy_wanted(n, dim).
    void* Xh = nullptr;
    float xh_scale = 1.f;

    // FP32 pilot sample of the exhaustive scan: internal rows 0, 64, 128, ...
    // (n_pilot rows) and the subspace of each. A frame's k-th distance over the
    // sample bounds its k-th over the whole database from above, so the full
    // scan starts with (a bound close to) it instead of +inf. Absent below
    // kPilotMinRows.
    int64_t n_pilot = 0;
    float* Xp = nullptr;
    int32_t* sub_p = nullptr;  // n_pilot: subspace of each sample row

    int32_t* err = nullptr;  // device error word (lhr_db_error)

    // Control blocks of the fused coarse-to-fine kernel (hier.cu): words that
    // must be zero when it starts. A block belongs to one stream (hws_map); the
    // kernel leaves it zeroed, so a call on that stream needs no memset.
    // kHierWsBlocks x hier_ws_block_bytes(), zeroed at build; nullptr without a
    // coarse slab. Views of the handle (subspaces) share both pointers.
    unsigned char* hws = nullptr;
    HierWsMap* hws_map = nullptr;
};

namespace lhr {

// The many-frame path's FP16 operand copy serves whole 128-byte K slices of at
// most 256 dimensions and row indices that fit its 32-bit candidate keys.
inline bool half_copy_wanted(int64_t n, int dim) {
    return dim % 64 == 0 && dim <= 256 && n >= kPilotMinRows && n < ((int64_t)1 << 31);
}

// Thread-local error message plumbing.
lhr_status fail(lhr_status st, const std::string& msg);
lhr_status cuda_fail(cudaError_t e, const char* what);

// Stream-ordered scratch from a library-owned memory pool of the current
// device. Freed (stream-ordered) by release().
struct Scratch {
    void* ptr = nullptr;
    cudaStream_t stream = nullptr;
    cudaError_t alloc(size_t bytes, cudaStream_t s);
    void release();
    ~Scratch() { release(); }
};

// Opt-in per-kernel event timing (lhr_profile_enable). A scope records an
// event pair around the launches it encloses when profiling is on.
struct ProfScope {
    int slot = -1;
    bool capturing = false;
    cudaStream_t stream = nullptr;
    ProfScope(const char* kernel, cudaStream_t s);
    ~ProfScope();
};

// Exhaustive FP32 scan + fused top-k (scan.cu).
// `pilot`: seed the scan's thresholds from the pilot sample when the database
// has one (same results, fewer exact recomputes; more scratch).
size_t scan_scratch_bytes(const lhr_db* db, int nq, int k, bool pilot);
// many.cu: exhaustive top k for many frames at once: a tensor-core filter over
// the FP16 copy (its own pilot, then the full pass) keeps every row that can be
// in a frame's top k; those are re-scored exactly in FP32.
bool many_eligible(const lhr_db* db, int nq, int k);
size_t many_scratch_bytes(const lhr_db* db, int nq);
cudaError_t launch_many(const lhr_db* db, const float* q, int nq, int k, const float* w, const float* xn,
                        const float* xmax_w, float margin_scale, int64_t* idx, float* dist, void* scratch,
                        cudaStream_t stream);

cudaError_t launch_scan(const lhr_db* db, const float* q, int nq, int k, int64_t* idx, float* dist,
                        void* scratch, bool pilot, cudaStream_t stream);
// Weighted exhaustive scan: d_w = sum_j w_j (q_j - x_j)^2, w device (D), >= 0.
size_t scan_weighted_scratch_bytes(const lhr_db* db, int nq, int k);
cudaError_t launch_scan_weighted(const lhr_db* db, const float* q, int nq, int k, const float* w, int64_t* idx,
                                 float* dist, void* scratch, cudaStream_t stream);

struct AggArgs;

// Fused coarse-to-fine (+ optional Algorithm 2) for requests of at most 8
// frames: one cooperative launch (hier.cu).
bool hier_fused_eligible(const lhr_db* db, int nq, int shortlist);
size_t hier_scratch_bytes(const lhr_db* db, int nq);
size_t hier_ws_block_bytes();
cudaError_t launch_hier_fused(const lhr_db* db, const float* q, int nq, int shortlist, int k, int64_t* idx,
                              float* dist, const AggArgs* agg_args, void* scratch, cudaStream_t stream);

// Sorts the keys key[0, nq) ascending (ties by index) and writes, for sorted
// position i < n_sorted (a multiple of 256): perm[i] = the index there (-1 past
// nq), its row_bytes of `codes` (a zero row past nq) into codes_s, and per 32
// positions the largest key among their valid indices (-inf if none) into
// gmax. Batches above 16,384 keep their order (lowp.cu).
cudaError_t launch_sort_queries(const float* key, int nq, int n_sorted, const void* codes, int row_bytes,
                                void* codes_s, int* perm, float* gmax, cudaStream_t stream);

// Low-precision tensor-core scores + FP32 re-rank (lowp.cu).
size_t lowp_scratch_bytes(const lhr_db* db, int nq, bool fp8, int W);
cudaError_t launch_lowp(const lhr_db* db, const float* q, int nq, bool fp8, int W, int k, int64_t* idx, float* dist,
                        void* scratch, cudaStream_t stream);

// Coarse-to-fine (coarse.cu).
size_t coarse_scratch_bytes(const lhr_db* db, int nq, int shortlist);
cudaError_t launch_coarse(const lhr_db* db, const float* q, int nq, int shortlist, int k, int64_t* idx,
                          float* dist, void* scratch, cudaStream_t stream);
// One subspace's [nq][k] result into slot s of [nq][n_sub][k], rows mapped to the caller's.
cudaError_t launch_subspace_remap(const int64_t* tidx, const float* tdist, int nq, int k, int n_sub, int s, int64_t off,
                                  const int32_t* perm, int64_t* idx, float* dist, cudaStream_t stream);

// Algorithm 2 (aggregate.cu). Candidates of window w: rows idx[c] for c in
// [cand_begin(w), cand_end(w)) where the range is cand_offsets[w]..[w+1]
// scaled by `per_frame` (frame offsets times candidates per frame) when
// per_frame > 0.
struct AggArgs {
    const int64_t* idx;
    const float* dist;
    const int32_t* offsets;
    int per_frame;  // > 0: offsets are frame offsets, each frame owns per_frame candidates
    long long limit;  // candidates available in idx / dist; a window reaching past it is an error
    int nw;
    int mode;
    int top_c;
    int toler_pct;
    long long r2max;
    float tau;
    double tile_m;
    double* xy_out;
    int32_t* status;
};
cudaError_t launch_aggregate(const lhr_db* db, const AggArgs& a, cudaStream_t stream);

// Request plumbing of the C ABI (api.cu), shared with the serving runtime.
lhr_status check_query_params(const lhr_db* db, const lhr_query_params* p);
lhr_status check_agg_params(const lhr_agg_params* a);
AggArgs make_agg(const lhr_db* db, const lhr_agg_params* a);
// Retrieval for nq frames with the path p selects (fused, coarse-to-fine,
// exhaustive or low-precision); scratch from the stream-ordered pool.
lhr_status run_retrieval(const lhr_db* db, const float* q, int nq, const lhr_query_params* p, int64_t* idx,
                         float* dist, cudaStream_t s);
long long circle_r2_limit(double radius_m, double tile_m);

// Soft retrieval forward / backward and the location loss (soft.cu).
size_t soft_backward_scratch_bytes(const lhr_db* db, int nw);
cudaError_t launch_soft_forward(const lhr_db* db, const float* frames, const int32_t* offsets, int W, int nw, int k,
                                const float* w, const float* tau, const int64_t* idx, const float* dist, double* p,
                                double* yhat, cudaStream_t stream);
cudaError_t launch_soft_backward(const lhr_db* db, const float* frames, const int32_t* offsets, int W, int nw, int k,
                                 const float* w, const float* tau, const int64_t* idx, const float* dist,
                                 const double* p, const double* yhat, const double* g, float* dq, float* dw,
                                 float* dtau, void* scratch, cudaStream_t stream);
cudaError_t launch_loc_mse(const double* yhat, const double* y, int nw, const double* scale, double* loss,
                           double* grad, cudaStream_t stream);

// Database construction helpers (build.cu).
cudaError_t launch_build_derived(lhr_db* db, cudaStream_t stream);
cudaError_t launch_check_finite(const float* x, int64_t count, int32_t* flag, cudaStream_t stream);
cudaError_t launch_gather_rows(const float* src, const int32_t* perm, int64_t n, int dim, float* dst,
                               cudaStream_t stream);
cudaError_t launch_tiles(const double* xy, int64_t n, double t, int32_t* tile, int32_t* flag, cudaStream_t stream);
cudaError_t launch_norms(const lhr_db* db, unsigned* max_bits, cudaStream_t stream);
cudaError_t launch_pilot_sample(const lhr_db* db, cudaStream_t stream);
// db->Xh from db->X: max |x| into *absmax_bits (zeroed by the caller), then the scaled copy.
cudaError_t launch_half_copy(const lhr_db* db, unsigned* absmax_bits, cudaStream_t stream);

}  // namespace lhr
