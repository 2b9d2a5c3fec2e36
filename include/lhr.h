/*
 * lhr.h -- C ABI of the GB300 library for hierarchical panoramic-feature
 * retrieval and 2-D multi-frame candidate aggregation (indoor localization,
 * arXiv 2006.08861).
 *
 * The paper states the problem this interface follows:
 *   - a server-side database of landmark features, each tied to floor-plan
 *     coordinates by a geo-referenced table made while modelling (§3, §3.2);
 *     the database may be divided into n_s subspaces, e.g. one per floor,
 *     searched independently (§3.1);
 *   - a localization request of M frames: q_m plus (M-1)/2 frames before and
 *     after it (§3.1, Algorithm 1 "selectNearbyFrames");
 *   - each frame is compared with every database frame by Euclidean distance
 *     and its top N candidates are kept, per subspace (§3.1, Algorithm 1
 *     "calculateDistance", "selectTopCandidates"; §4);
 *   - the candidates of all M frames are fused into one floor-plan position by
 *     tile-density aggregation (§3.2, Algorithm 2).
 *
 * Conventions (every entry point):
 *   - Array arguments are DEVICE pointers owned by the caller unless the
 *     argument says otherwise; the library never frees caller memory.
 *   - Calls are asynchronous on `cuda_stream` (a cudaStream_t; NULL = the
 *     legacy default stream) unless stated otherwise. Output arrays are valid
 *     once that stream reaches the end of the call's work.
 *   - Distances are SQUARED Euclidean distances (same order as Euclidean).
 *   - Top-N lists are ascending by (distance, database row): ties go to the
 *     lower row. A list longer than its subspace is padded with row -1 and
 *     distance +inf.
 *   - Argument errors are found on the host before any launch and return
 *     LHR_ERR_INVALID_ARG (nothing is launched, outputs are untouched).
 *     CUDA launch / allocation failures return LHR_ERR_CUDA / LHR_ERR_OOM.
 *     No C++ exception crosses this interface. lhr_last_error() returns a
 *     thread-local description of the last non-OK return.
 *   - Device-side waits are bounded; a wait that gives up records
 *     LHR_ERR_TIMEOUT in the database's error word (see lhr_db_error).
 */
#ifndef LHR_H
#define LHR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lhr_db lhr_db; /* opaque; owns every device buffer it allocates */

typedef enum {
    LHR_OK = 0,
    LHR_WARN_LOW_CONFIDENCE = 1, /* per-window status: no TopC tile passed the threshold */
    LHR_ERR_INVALID_ARG = -1,
    LHR_ERR_CUDA = -2,
    LHR_ERR_OOM = -3,
    LHR_ERR_TIMEOUT = -4,
    LHR_ERR_UNSUPPORTED = -5
} lhr_status;

typedef enum { LHR_F32 = 0, LHR_BF16 = 1, LHR_FP8_E4M3 = 2 } lhr_dtype;

typedef enum {
    LHR_AGG_TILE = 0,          /* Algorithm 2: centre of the winning 2-D tile */
    LHR_AGG_TILE_CENTROID = 1, /* mean position of the candidates in the winning tile's circle */
    LHR_AGG_SOFTMAX = 2        /* sum_i p_i xy_i, p = softmax(-d_i / tau) over the window */
} lhr_agg_mode;

/* Low-precision copies to build (bit mask for lhr_db_config.lowp). */
#define LHR_LOWP_BF16 1u
#define LHR_LOWP_FP8 2u

typedef struct {
    int32_t dim;        /* D: feature length, 4 <= D <= 512, D % 4 == 0 */
    int32_t coarse_dim; /* Dc: prefix length of the coarse level; 0 = none; else 4 <= Dc <= D, Dc % 4 == 0 */
    uint32_t lowp;      /* LHR_LOWP_* copies to build (need D % 32 == 0, D <= 512) */
    int32_t reserved;   /* must be 0 */
    double tile_m;      /* floor-plan tile edge in metres (paper: 0.30); > 0 */
} lhr_db_config;

typedef struct {
    int32_t k;            /* N of "top N" per frame and subspace: 1 <= k <= 32 */
    int32_t shortlist;    /* 0: exhaustive scan; S > 0: coarse-to-fine with an S-row shortlist (k <= S <= 4096) */
    lhr_dtype score;      /* LHR_F32: direct FP32 distances; LHR_BF16 / LHR_FP8_E4M3: tensor-core scores */
    int32_t rerank_width; /* low-precision scores only: W rows kept per query and re-ranked in FP32 (k <= W <= 128) */
} lhr_query_params;

typedef struct {
    lhr_agg_mode mode;
    int32_t top_c;     /* TopC tiles tested (paper: 10); >= 1 */
    double radius_m;   /* tolerance-circle radius in metres (paper: 3.0); >= 0 */
    int32_t toler_pct; /* tolerPer in percent (paper: 20); 0..100 */
    float tau;         /* softmax temperature (LHR_AGG_SOFTMAX only); > 0 */
} lhr_agg_params;

/*
 * lhr_build_db -- environment modelling (§3: every landmark is one feature,
 * stored server-side; §3.2: the geo-referenced index -> floor-plan table).
 *
 *   feats    n x D float32, row-major; host or device memory (detected).
 *            Every value must be finite.
 *   xy       n x 2 float64 floor-plan coordinates (x west->east, y
 *            south->north, metres); host or device memory.
 *   subspace n int32 subspace ids in [0, n_s) (§3.1 "subspaces"), host or
 *            device; NULL = one subspace.
 *   n        number of rows, 1 <= n < 2^31.
 *   cfg      dimensions, coarse prefix, low-precision copies, tile edge.
 *   out      receives the new handle; unchanged on error.
 * The library copies everything it needs; the caller keeps ownership of its
 * inputs. Besides the FP32 rows it keeps, for n >= 65,536 rows with D a
 * multiple of 64 up to 256, an FP16 copy of the rows scaled by a power of two
 * (n x D x 2 bytes): the operand of the exhaustive form's tensor-core filter
 * for many frames at once (lhr_query). Synchronizes `cuda_stream` before
 * returning.
 */
lhr_status lhr_build_db(const float* feats, const double* xy, const int32_t* subspace, int64_t n,
                        const lhr_db_config* cfg, void* cuda_stream, lhr_db** out);

/* Frees every device buffer of `db` (after synchronizing the device). NULL is a no-op. */
lhr_status lhr_free_db(lhr_db* db);

/* Shape of a database: rows, D, Dc, number of subspaces (any pointer may be NULL). */
lhr_status lhr_db_info(const lhr_db* db, int64_t* n, int32_t* dim, int32_t* coarse_dim,
                       int32_t* n_subspaces);

/*
 * lhr_query -- per-frame top-N retrieval (§3.1, Algorithm 1 steps
 * "calculateDistance" and "selectTopCandidates"; §4 "smallest Euclidean
 * distance", "top N").
 *
 *   q     nq x D float32 query frames (device), row-major, 16-byte aligned.
 *   nq    number of frames, >= 1.
 *   p     k, and the form: exhaustive FP32 (shortlist 0, score F32),
 *         coarse-to-fine (shortlist S > 0, needs a database built with
 *         coarse_dim > 0 and one subspace), or low-precision tensor-core
 *         scores + FP32 re-rank (score BF16/FP8, needs that copy, one
 *         subspace).
 *   idx   nq x n_s x k int64 (device): database rows (caller's numbering).
 *   dist  nq x n_s x k float32 (device): squared distances, FP32 direct form.
 * The exhaustive form over one subspace with 64 to 8,192 frames and k <= 32,
 * on a database with the FP16 copy, filters on the tensor cores (FP16
 * operands, a margin that bounds their rounding) and re-scores every row
 * that can be in a frame's top k with the FP32 direct form: the exact FP32
 * top k, as the streaming FP32 scan (which serves the other cases) returns.
 */
lhr_status lhr_query(const lhr_db* db, const float* q, int32_t nq, const lhr_query_params* p,
                     int64_t* idx, float* dist, void* cuda_stream);

/*
 * lhr_query_window -- the whole localization request: Algorithm 1 over every
 * frame of every window, then Algorithm 2 per window (§3.1, §3.2).
 *
 *   frames   W x D float32 (device): the frames of all windows back to back.
 *   offsets  nw + 1 int32 (device): window w holds frames
 *            [offsets[w], offsets[w+1]); offsets[0] = 0, offsets[nw] = W,
 *            non-decreasing. Window lengths may differ. A window that is
 *            empty, reaches outside [0, W], or holds more than 8192
 *            candidates (frames x n_s x k) gets status LHR_ERR_INVALID_ARG.
 *   W        total number of frames (= offsets[nw]), >= 1.
 *   nw       number of windows, >= 1.
 *   p, a     retrieval and aggregation parameters.
 *   idx/dist W x n_s x k (device): every frame's candidates, as lhr_query.
 *   xy       nw x 2 float64 (device): the final position of each window.
 *   status   nw int32 (device): LHR_OK, LHR_WARN_LOW_CONFIDENCE or an error.
 *
 * Requests of at most 8 frames on the coarse-to-fine FP32 path (this call or
 * lhr_query) run as one fused launch whose zero-initialised control words
 * live in the handle, one block per calling stream (the first 8 streams; the
 * others get a memset of scratch): each launch leaves its block zeroed for
 * the next. Calls on one stream are ordered, so they never share a block at
 * the same time. A CUDA graph captured on a stream keeps that stream's block:
 * two such graphs, or such a graph and direct calls on its capture stream,
 * must not run concurrently.
 */
lhr_status lhr_query_window(const lhr_db* db, const float* frames, const int32_t* offsets, int32_t W,
                            int32_t nw, const lhr_query_params* p, const lhr_agg_params* a,
                            int64_t* idx, float* dist, double* xy, int32_t* status, void* cuda_stream);

/*
 * lhr_aggregate_2d -- Algorithm 2 alone (§3.2) on caller-supplied candidates.
 *
 *   idx           n_cand candidate rows (device int64); row -1 is padding and
 *                 is skipped; any other row must be in [0, n) (a row outside
 *                 is skipped and recorded as LHR_ERR_INVALID_ARG in the
 *                 database's error word).
 *   dist          n_cand candidate squared distances (device float32), read
 *                 only in LHR_AGG_SOFTMAX mode (may be NULL otherwise).
 *   n_cand        length of idx / dist, >= 1.
 *   cand_offsets  nw + 1 int32 (device): window w owns candidates
 *                 [cand_offsets[w], cand_offsets[w+1]); 1..8192 per window and
 *                 inside [0, n_cand], else that window's status is
 *                 LHR_ERR_INVALID_ARG.
 *   xy, status    as lhr_query_window.
 */
lhr_status lhr_aggregate_2d(const lhr_db* db, const int64_t* idx, const float* dist, int64_t n_cand,
                            const int32_t* cand_offsets, int32_t nw, const lhr_agg_params* a,
                            double* xy, int32_t* status, void* cuda_stream);

/*
 * lhr_db_error -- reads and clears the database's device error word, which
 * kernels set when a bounded device-side wait gives up (LHR_ERR_TIMEOUT) or a
 * candidate row is out of range (LHR_ERR_INVALID_ARG). Synchronizes the stream.
 * *err receives LHR_OK when nothing was recorded.
 */
lhr_status lhr_db_error(const lhr_db* db, int32_t* err, void* cuda_stream);

/*
 * lhr_query_static -- the exhaustive FP32 lhr_query (shortlist 0, score F32)
 * for callers that cannot allocate device memory. The paper has no
 * counterpart; this entry point exists for the caller, not for the method.
 *
 * Who needs it: code that must not call cudaMalloc / cudaMallocAsync or any
 * allocating routine, for instance a host thread working under a memory
 * budget that another allocator already owns in full (a framework's caching
 * allocator), or a real-time loop in which an allocation's implicit
 * synchronization or failure is not acceptable. lhr_query instead takes its
 * per-call scratch from a stream-ordered memory pool.
 *
 * How: the scratch (per-chunk candidate lists and per-query-block counters)
 * is a fixed 4 MiB array in the library's device code. Every GPU that loads
 * the library holds that array until the process exits. A request whose
 * scratch would exceed 4 MiB (it grows with nq, k and the database's chunk
 * count, about nq x k x 8 x 152 bytes on a 152-SM GPU) is rejected with
 * LHR_ERR_INVALID_ARG before anything is launched; use fewer frames per call.
 * The call allocates nothing: no cudaMalloc, cudaFree or allocating library
 * routine (keep lhr_profile_enable off, which creates CUDA events).
 *
 * The first call on a device looks up the array's device address (once per
 * device, that device current); make that first call before any stream
 * capture. All calls share the one array and each call clears the parts that
 * must start at zero, so calls whose work overlaps on the GPU (other streams,
 * other threads) race and corrupt each other's results: serialize them.
 *
 * Arguments, outputs and errors as lhr_query with p = {k, 0, LHR_F32, 0}.
 */
lhr_status lhr_query_static(const lhr_db* db, const float* q, int32_t nq, int32_t k, int64_t* idx, float* dist,
                            void* cuda_stream);

/*
 * Soft retrieval -- a differentiable relaxation of Algorithm 1's selection
 * (§3.1) and of the window aggregation (§3.2) with learnable per-dimension
 * feature weights w and a temperature tau. The paper defines no gradient; the
 * form below is this library's, stated here in full.
 *
 *   d_w(q, x) = sum_j w_j (q_j - x_j)^2            (w_j >= 0; w = 1: §4's distance squared)
 *   per frame f: the top k rows of each subspace by d_w (ties: lower row),
 *                held fixed when differentiating
 *   per window b: l_i = -d_i / tau over the window's m n_s k candidates,
 *                 p = softmax(l), y^_b = sum_i p_i xy_i        (FP64 sums)
 *   lhr_loc_mse:  L = (1/B) sum_b ||y^_b - y_b||^2
 *
 * lhr_query_weighted -- the selection alone: lhr_query's exhaustive FP32 scan
 * with d_w. q nq x D float32 (device, 16-byte aligned); w D float32 (device,
 * 16-byte aligned, every w_j finite and >= 0: a negative or non-finite weight
 * records LHR_ERR_INVALID_ARG in the error word and the results are
 * meaningless); 1 <= k <= 32; idx / dist nq x n_s x k as lhr_query, dist = d_w.
 *
 * lhr_soft_forward -- selection, then the window softmax. frames W x D and
 * offsets nw + 1 as lhr_query_window (windows disjoint and in order); tau one
 * float32 on the device (> 0, else the window's y^ is NaN and
 * LHR_ERR_INVALID_ARG is recorded). Outputs (device): idx, dist W x n_s x k;
 * p W x n_s x k float64 softmax weights (0 for padding slots); yhat nw x 2
 * float64. Needs D <= 1024 and n_s k <= 1024 (else LHR_ERR_UNSUPPORTED).
 *
 * lhr_soft_backward -- given g_yhat = dL/dy^ (nw x 2 float64, device) and the
 * forward's idx, dist, p, yhat, writes
 *   dq   W x D float32:  dL/dq_fj = sum_{i in f} dL/dd_i 2 w_j (q_fj - x_ij)
 *   dw   D float32:      dL/dw_j  = sum_i dL/dd_i (q_f(i)j - x_ij)^2
 *   dtau 1 float32:      dL/dtau  = sum_i dL/dl_i d_i / tau^2
 * with dL/dl_i = p_i g_b . (xy_i - y^_b) and dL/dd_i = -dL/dl_i / tau. The
 * rows are re-read (no distance tile is kept); sums over windows run in a
 * fixed order, so the result is deterministic.
 *
 * lhr_loc_mse -- loss = L (one float64) and/or grad = scale * dL/dy^
 * (nw x 2 float64); scale is one float64 on the device, NULL = 1. Either
 * output may be NULL, not both. Runs on the current device.
 */
lhr_status lhr_query_weighted(const lhr_db* db, const float* q, int32_t nq, int32_t k, const float* w,
                              int64_t* idx, float* dist, void* cuda_stream);
lhr_status lhr_soft_forward(const lhr_db* db, const float* frames, const int32_t* offsets, int32_t W, int32_t nw,
                            int32_t k, const float* w, const float* tau, int64_t* idx, float* dist, double* p,
                            double* yhat, void* cuda_stream);
lhr_status lhr_soft_backward(const lhr_db* db, const float* frames, const int32_t* offsets, int32_t W, int32_t nw,
                             int32_t k, const float* w, const float* tau, const int64_t* idx, const float* dist,
                             const double* p, const double* yhat, const double* g_yhat, float* dq, float* dw,
                             float* dtau, void* cuda_stream);
lhr_status lhr_loc_mse(const double* yhat, const double* y, int32_t nw, const double* scale, double* loss,
                       double* grad, void* cuda_stream);

/*
 * Serving runtime (no counterpart in the paper's own system, which localizes
 * one user at a time): continuous batching of requests from many concurrent
 * user streams. Each submitted frame is retrieved once (lhr_query's path for
 * `shortlist` / `score`) and its top k is cached in the stream's device ring;
 * a request for the stream's last m frames (Algorithm 2, §3.2) gathers the
 * cached candidates. A scheduler thread forms ticks of up to max_batch_frames
 * queued frames, oldest first, and launches each on one of n_lanes CUDA
 * streams when a lane is free and the tick's scratch fits mem_budget_bytes
 * beside the ticks in flight, so ticks overlap on the device. Results equal
 * lhr_query / lhr_aggregate_2d on the same frames: batching changes the
 * schedule only.
 *
 * Streams are admitted by memory: with ring_mem_bytes > 0 the server holds
 * floor(ring_mem_bytes / ring bytes) device rings (ring bytes = ring_frames x
 * (D x 4 + n_s x k x 12)); a stream must be opened (lhr_server_open_stream),
 * which fails with LHR_ERR_OOM while every ring is held, and closing a stream
 * (lhr_server_close_stream) returns its ring once its frames are done. With
 * ring_mem_bytes = 0 every stream id is open from the start.
 */
typedef struct lhr_server lhr_server;
typedef struct {
    int32_t n_streams;        /* user stream ids 0 .. n_streams - 1 */
    int32_t max_window;       /* longest window m a request may ask for (>= 1) */
    int32_t ring_frames;      /* frames (and top-k lists) kept per stream on the device, > max_window */
    int32_t max_batch_frames; /* frames per tick, i.e. per retrieval launch (>= 1) */
    int32_t n_lanes;          /* CUDA streams the ticks rotate over (>= 2) */
    int32_t k;                /* top k per frame and subspace (1 .. 32) */
    int32_t shortlist;        /* 0: exhaustive scan (or low-precision scores); S: coarse-to-fine (needs a coarse level) */
    lhr_dtype score;          /* LHR_F32; LHR_BF16 / LHR_FP8_E4M3: tensor-core scores + FP32 re-rank (shortlist 0) */
    int64_t mem_budget_bytes; /* device scratch the ticks in flight may hold together (> 0) */
    lhr_agg_params agg;       /* Algorithm 2 parameters of every window */
    int32_t rerank_width;     /* low-precision scores: rows re-ranked in FP32 per frame (k .. 128); else ignored */
    int32_t reserved;         /* 0 */
    int64_t ring_mem_bytes;   /* 0: every stream open, one ring each; > 0: device memory for rings, streams opened on demand */
} lhr_server_config;

typedef struct {
    int64_t request_id; /* as submitted */
    int32_t stream_id;
    int32_t m;          /* frames in the window (fewer than asked when the stream had fewer) */
    int32_t status;     /* LHR_OK, LHR_WARN_LOW_CONFIDENCE or an error */
    int32_t reserved;
    double xy[2];       /* the window's position, metres */
    double latency_us;  /* submission of the window's last frame -> result on the host */
} lhr_server_result;

/* Allocates the rings and lanes and starts the scheduler thread. db must
 * outlive the server. */
lhr_status lhr_server_create(const lhr_db* db, const lhr_server_config* cfg, lhr_server** out);
/* Queues one frame (D float32, host memory, copied before return) of a stream;
 * window_m > 0 also requests the position of the stream's last window_m frames
 * (this one included). Thread-safe; never blocks on the GPU. */
lhr_status lhr_server_submit(lhr_server* s, int32_t stream_id, const float* frame, int32_t window_m,
                             int64_t request_id);
/* Moves up to max_results finished windows into out (waiting up to wait_ms
 * for the first); *n_out receives the count. LHR_ERR_CUDA once a tick failed. */
lhr_status lhr_server_poll(lhr_server* s, lhr_server_result* out, int32_t max_results, int32_t* n_out,
                           int32_t wait_ms);
/* Admits a new stream when a ring is free: *stream_id receives its id (its frames
 * start from none). LHR_ERR_OOM when every ring is held by an open stream;
 * LHR_ERR_INVALID_ARG when the server opened every stream at creation. */
lhr_status lhr_server_open_stream(lhr_server* s, int32_t* stream_id);
/* Closes an open stream: no more submissions are accepted for it, and its ring
 * returns to the server once its queued and in-flight frames are done. Waits up
 * to timeout_ms for that; LHR_ERR_TIMEOUT means the frames are still running
 * and the ring returns by itself when they finish. Results of its windows stay
 * available to lhr_server_poll. */
lhr_status lhr_server_close_stream(lhr_server* s, int32_t stream_id, int32_t timeout_ms);
/* Waits until every submitted frame is processed (LHR_ERR_TIMEOUT after timeout_ms). */
lhr_status lhr_server_drain(lhr_server* s, int32_t timeout_ms);
/* Finishes queued work, stops the scheduler and frees everything. */
lhr_status lhr_server_destroy(lhr_server* s);

/*
 * Instrumentation (no counterpart in the paper): per-kernel CUDA-event timing.
 * lhr_profile_enable(1) makes every later launch record an event pair on its
 * stream around each kernel; lhr_profile_read synchronizes those events and
 * returns, for kernels whose name contains `kernel` (NULL = all), the number
 * of launches and their summed device time in milliseconds, then forgets them
 * when `reset` is non-zero. Off by default; costs two event records per
 * kernel when on. Process-wide. A launch made while its stream is being
 * captured into a CUDA graph records the pair as event-record nodes of the
 * graph: every replay re-records them, so read such records with reset = 0
 * after each replay, and reset them only once the graph is destroyed.
 */
lhr_status lhr_profile_enable(int32_t on);
lhr_status lhr_profile_read(const char* kernel, int64_t* launches, double* total_ms, int32_t reset);

/* Thread-local message describing the last non-OK return on this thread. */
const char* lhr_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LHR_H */
