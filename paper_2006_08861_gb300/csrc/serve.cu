// Serving runtime: continuous batching of localization requests from many
// concurrent user streams (§3: a user's camera sends panoramic frames; each
// frame's top-N candidates feed Algorithm 2 over the user's last M frames).
//
// Host side (one scheduler thread per server):
//   * lhr_server_submit appends a frame of one user stream and, optionally,
//     asks for the position of the stream's last m frames; the call only
//     queues (host copy of the frame) and returns.
//   * The scheduler forms a tick from the queued frames, oldest first, up to
//     max_batch_frames, admits it when a lane (CUDA stream with its own
//     buffers) is free and the tick's scratch fits the device-memory budget
//     next to the ticks in flight, and launches it: H2D copy of the frames,
//     one retrieval for all of them (coarse-to-fine or exhaustive, the
//     library's kernels), a scatter into the streams' device rings (frame and
//     its top-k, cached: each frame is retrieved once however many windows
//     use it), a gather of every requested window's candidates from the
//     cached top-k, Algorithm 2 over all those windows in one launch, and a
//     D2H copy of the positions. Frames that arrive while ticks run join the
//     next tick on another lane, so the work of several ticks overlaps on the
//     device; a window whose earlier frames belong to a tick still in flight
//     waits for that tick's retrieval event on the device, not on the host.
//   * Completed windows go to a result queue read by lhr_server_poll, with
//     their latency from submission to completion.
// A frame is retrieved and a window aggregated exactly as by lhr_query /
// lhr_aggregate_2d on the same inputs: batching changes the schedule, never
// a result.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace lhr {
namespace {

using Clock = std::chrono::steady_clock;

// Ring slot (stream st, slot j) -> frame + its top-k, and window gathers.
__global__ void scatter_kernel(const float* frames, const int64_t* idx, const float* dist, const int32_t* map, int nb,
                               int D, int kc, float* ring_frames, int64_t* cache_idx, float* cache_dist) {
    const int b = blockIdx.x;
    if (b >= nb) return;
    const int64_t slot = map[b];
    for (int j = threadIdx.x; j < D; j += blockDim.x) ring_frames[slot * D + j] = frames[(size_t)b * D + j];
    for (int j = threadIdx.x; j < kc; j += blockDim.x) {
        cache_idx[slot * kc + j] = idx[(size_t)b * kc + j];
        cache_dist[slot * kc + j] = dist[(size_t)b * kc + j];
    }
}

// Window w's frames are the ring slots wslots[woff[w] .. woff[w+1]); its
// candidates land at cidx[woff[w] * kc ...] in frame order.
__global__ void gather_kernel(const int32_t* wslots, int n_frames, int kc, const int64_t* cache_idx,
                              const float* cache_dist, int64_t* cidx, float* cdist) {
    const int i = blockIdx.x;
    if (i >= n_frames) return;
    const int64_t slot = wslots[i];
    for (int j = threadIdx.x; j < kc; j += blockDim.x) {
        cidx[(size_t)i * kc + j] = cache_idx[slot * kc + j];
        cdist[(size_t)i * kc + j] = cache_dist[slot * kc + j];
    }
}

struct Submission {
    int32_t stream;
    int32_t m;
    int64_t request_id;
    std::vector<float> frame;
    Clock::time_point t;
};

struct WindowReq {
    int64_t request_id;
    int32_t stream;
    int32_t m;
    Clock::time_point t;
};

struct SlotInfo {
    int64_t seq = -1;   // frame number of the stream held by the slot
    int lane = -1;      // lane and tick that computed its top-k
    int64_t tick = -1;
};

struct Lane {
    cudaStream_t s = nullptr;
    cudaEvent_t retr_done = nullptr, all_done = nullptr;
    bool busy = false;
    int64_t tick = -1;
    size_t reserved = 0;
    // frames of the tick
    float* h_frames = nullptr;  // pinned, max_batch x D
    int32_t* h_map = nullptr;   // pinned, max_batch: ring slot of each frame
    float* d_frames = nullptr;
    int32_t* d_map = nullptr;
    int64_t* d_idx = nullptr;   // max_batch x kc
    float* d_dist = nullptr;
    // windows of the tick
    int32_t* h_wslots = nullptr;  // pinned, max_batch x R
    int32_t* h_woff = nullptr;    // pinned, candidate offsets (max_batch + 1)
    int32_t* d_wslots = nullptr;
    int32_t* d_woff = nullptr;
    int64_t* d_cidx = nullptr;    // max_batch x R x kc
    float* d_cdist = nullptr;
    double* d_xy = nullptr;
    int32_t* d_status = nullptr;
    double* h_xy = nullptr;       // pinned
    int32_t* h_status = nullptr;  // pinned
    std::vector<WindowReq> windows;
    std::vector<int32_t> frame_streams;  // stream of each frame (in-flight accounting)
};

}  // namespace
}  // namespace lhr

struct lhr_server {
    const lhr_db* db = nullptr;
    lhr_server_config cfg{};
    lhr_query_params qp{};
    int D = 0, kc = 0, R = 0;
    int n_rings = 0;          // device rings (frames + cached top-k lists), one per open stream
    bool on_demand = false;   // streams are opened and closed by the caller (rings admitted by memory)
    float* ring_frames = nullptr;
    int64_t* cache_idx = nullptr;
    float* cache_dist = nullptr;
    std::vector<std::vector<lhr::SlotInfo>> slots;  // [ring][R]
    std::vector<int32_t> ring_of;                   // ring of each stream id, -1 = none
    std::vector<int32_t> state;                     // per stream id: 0 closed, 1 open, 2 closing
    std::vector<int32_t> free_rings;
    std::vector<int64_t> queued;                    // frames per stream waiting in the submission queue
    std::vector<int64_t> next_seq;                  // frames submitted per stream
    std::vector<int32_t> in_flight;                 // frames per stream in busy lanes
    std::vector<lhr::Lane> lanes;
    int64_t ticks = 0;
    size_t reserved = 0;

    std::thread sched;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<lhr::Submission> subq;
    std::deque<lhr_server_result> doneq;
    int64_t submitted = 0, completed = 0;  // frames
    bool stop = false;
    std::string error;  // first failure of the scheduler thread
};

namespace lhr {
namespace {

size_t tick_scratch(const lhr_server* S, int nb) {
    const lhr_db* db = S->db;
    if (S->qp.score != LHR_F32) return lowp_scratch_bytes(db, nb, S->qp.score == LHR_FP8_E4M3, S->qp.rerank_width);
    if (S->qp.shortlist > 0)
        return hier_fused_eligible(db, nb, S->qp.shortlist) ? hier_scratch_bytes(db, nb)
                                                            : coarse_scratch_bytes(db, nb, S->qp.shortlist);
    return scan_scratch_bytes(db, nb, S->qp.k, true);
}

// A closing stream's ring goes back to the free list once none of its frames is
// queued or in flight (caller holds S->mu).
void maybe_release(lhr_server* S, int st) {
    if (S->state[st] == 2 && S->queued[st] == 0 && S->in_flight[st] == 0) {
        S->free_rings.push_back(S->ring_of[st]);
        S->ring_of[st] = -1;
        S->state[st] = 0;
    }
}

// Lanes whose tick finished: their windows become results.
void finish_lanes(lhr_server* S, bool block) {
    for (size_t li = 0; li < S->lanes.size(); ++li) {
        Lane& L = S->lanes[li];
        if (!L.busy) continue;
        cudaError_t e = block ? cudaEventSynchronize(L.all_done) : cudaEventQuery(L.all_done);
        if (e == cudaErrorNotReady) continue;
        if (e != cudaSuccess) {
            std::lock_guard<std::mutex> lk(S->mu);
            if (S->error.empty()) S->error = std::string("tick failed: ") + cudaGetErrorString(e);
        }
        const auto now = Clock::now();
        std::lock_guard<std::mutex> lk(S->mu);
        for (size_t w = 0; w < L.windows.size(); ++w) {
            lhr_server_result r{};
            r.request_id = L.windows[w].request_id;
            r.stream_id = L.windows[w].stream;
            r.m = L.windows[w].m;
            r.status = e == cudaSuccess ? L.h_status[w] : LHR_ERR_CUDA;
            r.xy[0] = L.h_xy[2 * w];
            r.xy[1] = L.h_xy[2 * w + 1];
            r.latency_us = std::chrono::duration<double, std::micro>(now - L.windows[w].t).count();
            S->doneq.push_back(r);
        }
        for (int32_t st : L.frame_streams) S->in_flight[st]--;
        for (int32_t st : L.frame_streams) maybe_release(S, st);
        S->completed += (int64_t)L.frame_streams.size();
        S->reserved -= L.reserved;
        L.busy = false;
        L.windows.clear();
        L.frame_streams.clear();
        S->cv_done.notify_all();
    }
}

void fail_sched(lhr_server* S, const std::string& msg) {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->error.empty()) S->error = msg;
    S->cv_done.notify_all();
}

// Takes queued frames (oldest first) into a tick on lane `li` and launches it.
// Returns false when nothing could be taken.
bool launch_tick(lhr_server* S, int li) {
    Lane& L = S->lanes[li];
    const int D = S->D, kc = S->kc, R = S->R;
    const int maxm = S->cfg.max_window;
    std::vector<Submission> take;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        // a stream may not hold more frames in flight than its ring can keep
        // beside the max_window frames its windows read; a taken frame counts
        // as in flight at once, so its stream's ring stays while it is used
        while (!S->subq.empty() && (int)take.size() < S->cfg.max_batch_frames) {
            const Submission& sb = S->subq.front();
            if (S->in_flight[sb.stream] + 1 > R - maxm) break;
            S->in_flight[sb.stream]++;
            S->queued[sb.stream]--;
            take.push_back(std::move(S->subq.front()));
            S->subq.pop_front();
        }
    }
    const int nb = (int)take.size();
    if (nb == 0) return false;
    const int64_t tick = S->ticks++;
    L.tick = tick;
    L.windows.clear();
    L.frame_streams.clear();
    std::vector<std::pair<int, int64_t>> deps;  // (lane, tick) computing earlier frames of this tick's windows
    int nwin = 0, wframes = 0;
    L.h_woff[0] = 0;
    for (int b = 0; b < nb; ++b) {
        Submission& sb = take[b];
        const int st = sb.stream;
        const int rg = S->ring_of[st];  // open or closing: the ring stays until its frames are done
        const int64_t seq = S->next_seq[st]++;
        const int slot = (int)(seq % R);
        std::memcpy(L.h_frames + (size_t)b * D, sb.frame.data(), (size_t)D * sizeof(float));
        L.h_map[b] = rg * R + slot;
        S->slots[rg][slot] = SlotInfo{seq, li, tick};
        L.frame_streams.push_back(st);
        if (sb.m > 0) {
            const int m = (int)std::min<int64_t>(sb.m, seq + 1);
            for (int64_t f = seq - m + 1; f <= seq; ++f) {
                const int fs = (int)(f % R);
                const SlotInfo& si = S->slots[rg][fs];
                L.h_wslots[wframes++] = rg * R + fs;
                if (si.tick != tick) deps.emplace_back(si.lane, si.tick);
            }
            L.windows.push_back(WindowReq{sb.request_id, st, m, sb.t});
            ++nwin;
            L.h_woff[nwin] = wframes * kc;
        }
    }
    L.reserved = tick_scratch(S, nb);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->reserved += L.reserved;
    }
    // device-side waits on earlier ticks still running on other lanes
    for (auto& dp : deps) {
        const Lane& o = S->lanes[dp.first];
        if (dp.first != li && o.busy && o.tick == dp.second) cudaStreamWaitEvent(L.s, o.retr_done, 0);
    }
    cudaError_t e = cudaMemcpyAsync(L.d_frames, L.h_frames, (size_t)nb * D * sizeof(float), cudaMemcpyHostToDevice, L.s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(L.d_map, L.h_map, nb * sizeof(int32_t), cudaMemcpyHostToDevice, L.s);
    if (e != cudaSuccess) {
        fail_sched(S, std::string("tick copy: ") + cudaGetErrorString(e));
        return false;
    }
    if (run_retrieval(S->db, L.d_frames, nb, &S->qp, L.d_idx, L.d_dist, L.s) != LHR_OK) {
        fail_sched(S, "tick retrieval: " + std::string(lhr_last_error()));
        return false;
    }
    scatter_kernel<<<nb, 128, 0, L.s>>>(L.d_frames, L.d_idx, L.d_dist, L.d_map, nb, D, kc, S->ring_frames,
                                        S->cache_idx, S->cache_dist);
    cudaEventRecord(L.retr_done, L.s);
    if (nwin > 0) {
        cudaMemcpyAsync(L.d_wslots, L.h_wslots, wframes * sizeof(int32_t), cudaMemcpyHostToDevice, L.s);
        cudaMemcpyAsync(L.d_woff, L.h_woff, (nwin + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, L.s);
        gather_kernel<<<wframes, 128, 0, L.s>>>(L.d_wslots, wframes, kc, S->cache_idx, S->cache_dist, L.d_cidx,
                                                L.d_cdist);
        AggArgs ag = make_agg(S->db, &S->cfg.agg);
        ag.idx = L.d_cidx;
        ag.dist = L.d_cdist;
        ag.offsets = L.d_woff;
        ag.per_frame = 0;
        ag.limit = (long long)wframes * kc;
        ag.nw = nwin;
        ag.xy_out = L.d_xy;
        ag.status = L.d_status;
        if ((e = launch_aggregate(S->db, ag, L.s)) != cudaSuccess) {
            fail_sched(S, std::string("tick aggregation: ") + cudaGetErrorString(e));
            return false;
        }
        cudaMemcpyAsync(L.h_xy, L.d_xy, (size_t)nwin * 2 * sizeof(double), cudaMemcpyDeviceToHost, L.s);
        cudaMemcpyAsync(L.h_status, L.d_status, nwin * sizeof(int32_t), cudaMemcpyDeviceToHost, L.s);
    }
    if ((e = cudaEventRecord(L.all_done, L.s)) != cudaSuccess || (e = cudaGetLastError()) != cudaSuccess) {
        fail_sched(S, std::string("tick launch: ") + cudaGetErrorString(e));
        return false;
    }
    L.busy = true;
    return true;
}

void scheduler(lhr_server* S) {
    cudaSetDevice(S->db->device);
    for (;;) {
        finish_lanes(S, false);
        bool stop, have;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            stop = S->stop;
            have = !S->subq.empty();
            if (!S->error.empty()) have = false;
        }
        int free_lane = -1, busy = 0;
        for (size_t i = 0; i < S->lanes.size(); ++i) {
            if (S->lanes[i].busy) ++busy;
            else if (free_lane < 0) free_lane = (int)i;
        }
        if (stop && !have && busy == 0) return;
        bool launched = false;
        if (have && free_lane >= 0) {
            // memory admission: the next tick's scratch must fit beside the ticks in flight
            int nb;
            {
                std::lock_guard<std::mutex> lk(S->mu);
                nb = (int)std::min<size_t>(S->subq.size(), (size_t)S->cfg.max_batch_frames);
            }
            const size_t need = tick_scratch(S, nb);
            if (busy == 0 || S->reserved + need <= (size_t)S->cfg.mem_budget_bytes) launched = launch_tick(S, free_lane);
        }
        if (!launched) {
            if (busy > 0) {
                std::this_thread::sleep_for(std::chrono::microseconds(20));
            } else {
                std::unique_lock<std::mutex> lk(S->mu);
                S->cv_work.wait_for(lk, std::chrono::milliseconds(2),
                                    [&] { return S->stop || !S->subq.empty(); });
            }
        }
    }
}

void free_server(lhr_server* S) {
    for (Lane& L : S->lanes) {
        if (L.s) cudaStreamSynchronize(L.s);
        void* dev[] = {L.d_frames, L.d_map, L.d_idx, L.d_dist, L.d_wslots, L.d_woff, L.d_cidx, L.d_cdist, L.d_xy,
                       L.d_status};
        for (void* p : dev)
            if (p) cudaFree(p);
        void* host[] = {L.h_frames, L.h_map, L.h_wslots, L.h_woff, L.h_xy, L.h_status};
        for (void* p : host)
            if (p) cudaFreeHost(p);
        if (L.retr_done) cudaEventDestroy(L.retr_done);
        if (L.all_done) cudaEventDestroy(L.all_done);
        if (L.s) cudaStreamDestroy(L.s);
    }
    if (S->ring_frames) cudaFree(S->ring_frames);
    if (S->cache_idx) cudaFree(S->cache_idx);
    if (S->cache_dist) cudaFree(S->cache_dist);
    delete S;
}

}  // namespace
}  // namespace lhr

using namespace lhr;

extern "C" {

lhr_status lhr_server_create(const lhr_db* db, const lhr_server_config* cfg, lhr_server** out) {
    if (!db || !cfg || !out) return fail(LHR_ERR_INVALID_ARG, "db, cfg and out must be non-NULL");
    if (cfg->n_streams < 1 || cfg->max_window < 1 || cfg->max_batch_frames < 1 || cfg->n_lanes < 2)
        return fail(LHR_ERR_INVALID_ARG, "n_streams, max_window, max_batch_frames >= 1 and n_lanes >= 2 required");
    if (cfg->ring_frames < cfg->max_window + 1)
        return fail(LHR_ERR_INVALID_ARG, "ring_frames must exceed max_window");
    if (cfg->mem_budget_bytes <= 0) return fail(LHR_ERR_INVALID_ARG, "mem_budget_bytes must be > 0");
    if (cfg->reserved != 0 || cfg->ring_mem_bytes < 0)
        return fail(LHR_ERR_INVALID_ARG, "reserved must be 0 and ring_mem_bytes >= 0");
    lhr_query_params qp{cfg->k, cfg->shortlist, cfg->score, cfg->score == LHR_F32 ? 0 : cfg->rerank_width};
    lhr_status st = check_query_params(db, &qp);
    if (st != LHR_OK) return st;
    if ((st = check_agg_params(&cfg->agg)) != LHR_OK) return st;
    if ((int64_t)cfg->max_window * db->n_sub * cfg->k > 8192)
        return fail(LHR_ERR_INVALID_ARG, "max_window x n_s x k exceeds 8192 candidates per window");
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(db->device);
    lhr_server* S = new lhr_server();
    S->db = db;
    S->cfg = *cfg;
    S->qp = qp;
    S->D = db->dim;
    S->kc = db->n_sub * cfg->k;
    S->R = cfg->ring_frames;
    const int D = S->D, kc = S->kc, R = S->R, NB = cfg->max_batch_frames;
    const size_t ring_bytes = (size_t)R * ((size_t)D * sizeof(float) + (size_t)kc * (sizeof(int64_t) + sizeof(float)));
    S->on_demand = cfg->ring_mem_bytes > 0;
    S->n_rings = S->on_demand ? (int)std::min<int64_t>(cfg->n_streams, cfg->ring_mem_bytes / (int64_t)ring_bytes)
                              : cfg->n_streams;
    if (S->n_rings < 1) {
        delete S;
        if (prev >= 0) cudaSetDevice(prev);
        return fail(LHR_ERR_INVALID_ARG, "ring_mem_bytes holds no ring (ring_frames x (D x 4 + n_s x k x 12) bytes)");
    }
    const size_t nslot = (size_t)S->n_rings * R;
    cudaError_t e = cudaMalloc(&S->ring_frames, nslot * D * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&S->cache_idx, nslot * kc * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc(&S->cache_dist, nslot * kc * sizeof(float));
    S->slots.assign(S->n_rings, std::vector<SlotInfo>(R));
    S->next_seq.assign(cfg->n_streams, 0);
    S->in_flight.assign(cfg->n_streams, 0);
    S->queued.assign(cfg->n_streams, 0);
    S->ring_of.assign(cfg->n_streams, -1);
    S->state.assign(cfg->n_streams, 0);
    if (S->on_demand) {
        for (int r = S->n_rings - 1; r >= 0; --r) S->free_rings.push_back(r);
    } else {
        for (int st = 0; st < cfg->n_streams; ++st) {
            S->ring_of[st] = st;
            S->state[st] = 1;
        }
    }
    S->lanes.resize(cfg->n_lanes);
    for (Lane& L : S->lanes) {
        if (e != cudaSuccess) break;
        e = cudaStreamCreateWithFlags(&L.s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L.retr_done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L.all_done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost(&L.h_frames, (size_t)NB * D * sizeof(float));
        if (e == cudaSuccess) e = cudaMallocHost(&L.h_map, NB * sizeof(int32_t));
        if (e == cudaSuccess) e = cudaMallocHost(&L.h_wslots, (size_t)NB * R * sizeof(int32_t));
        if (e == cudaSuccess) e = cudaMallocHost(&L.h_woff, (NB + 1) * sizeof(int32_t));
        if (e == cudaSuccess) e = cudaMallocHost(&L.h_xy, (size_t)NB * 2 * sizeof(double));
        if (e == cudaSuccess) e = cudaMallocHost(&L.h_status, NB * sizeof(int32_t));
        if (e == cudaSuccess) e = cudaMalloc(&L.d_frames, (size_t)NB * D * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&L.d_map, NB * sizeof(int32_t));
        if (e == cudaSuccess) e = cudaMalloc(&L.d_idx, (size_t)NB * kc * sizeof(int64_t));
        if (e == cudaSuccess) e = cudaMalloc(&L.d_dist, (size_t)NB * kc * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&L.d_wslots, (size_t)NB * R * sizeof(int32_t));
        if (e == cudaSuccess) e = cudaMalloc(&L.d_woff, (NB + 1) * sizeof(int32_t));
        if (e == cudaSuccess) e = cudaMalloc(&L.d_cidx, (size_t)NB * R * kc * sizeof(int64_t));
        if (e == cudaSuccess) e = cudaMalloc(&L.d_cdist, (size_t)NB * R * kc * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&L.d_xy, (size_t)NB * 2 * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&L.d_status, NB * sizeof(int32_t));
    }
    if (e != cudaSuccess) {
        free_server(S);
        if (prev >= 0) cudaSetDevice(prev);
        return cuda_fail(e, "server allocation");
    }
    S->sched = std::thread(scheduler, S);
    if (prev >= 0) cudaSetDevice(prev);
    *out = S;
    return LHR_OK;
}

lhr_status lhr_server_submit(lhr_server* S, int32_t stream_id, const float* frame, int32_t window_m,
                             int64_t request_id) {
    if (!S || !frame) return fail(LHR_ERR_INVALID_ARG, "server and frame must be non-NULL");
    if (stream_id < 0 || stream_id >= S->cfg.n_streams) return fail(LHR_ERR_INVALID_ARG, "stream_id out of range");
    if (window_m < 0 || window_m > S->cfg.max_window) return fail(LHR_ERR_INVALID_ARG, "window_m out of range");
    Submission sb;
    sb.stream = stream_id;
    sb.m = window_m;
    sb.request_id = request_id;
    sb.frame.assign(frame, frame + S->D);
    sb.t = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (!S->error.empty()) return fail(LHR_ERR_CUDA, S->error);
        if (S->stop) return fail(LHR_ERR_INVALID_ARG, "server is stopping");
        if (S->state[stream_id] != 1) return fail(LHR_ERR_INVALID_ARG, "stream is not open");
        S->queued[stream_id]++;
        S->subq.push_back(std::move(sb));
        S->submitted++;
    }
    S->cv_work.notify_one();
    return LHR_OK;
}

lhr_status lhr_server_poll(lhr_server* S, lhr_server_result* out, int32_t max_results, int32_t* n_out,
                           int32_t wait_ms) {
    if (!S || !n_out || (max_results > 0 && !out)) return fail(LHR_ERR_INVALID_ARG, "bad poll arguments");
    std::unique_lock<std::mutex> lk(S->mu);
    if (wait_ms > 0)
        S->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms),
                            [&] { return !S->doneq.empty() || !S->error.empty(); });
    int n = 0;
    while (n < max_results && !S->doneq.empty()) {
        out[n++] = S->doneq.front();
        S->doneq.pop_front();
    }
    *n_out = n;
    if (!S->error.empty()) return fail(LHR_ERR_CUDA, S->error);
    return LHR_OK;
}

lhr_status lhr_server_open_stream(lhr_server* S, int32_t* stream_id) {
    if (!S || !stream_id) return fail(LHR_ERR_INVALID_ARG, "server and stream_id must be non-NULL");
    std::lock_guard<std::mutex> lk(S->mu);
    if (!S->on_demand) return fail(LHR_ERR_INVALID_ARG, "every stream was opened at creation (ring_mem_bytes = 0)");
    if (!S->error.empty()) return fail(LHR_ERR_CUDA, S->error);
    if (S->free_rings.empty()) return fail(LHR_ERR_OOM, "admission refused: every ring is held by an open stream");
    int id = -1;
    for (int st = 0; st < S->cfg.n_streams && id < 0; ++st)
        if (S->state[st] == 0) id = st;
    if (id < 0) return fail(LHR_ERR_OOM, "admission refused: every stream id is in use");
    const int rg = S->free_rings.back();
    S->free_rings.pop_back();
    S->ring_of[id] = rg;
    S->state[id] = 1;
    S->next_seq[id] = 0;
    for (SlotInfo& si : S->slots[rg]) si = SlotInfo{};
    *stream_id = id;
    return LHR_OK;
}

lhr_status lhr_server_close_stream(lhr_server* S, int32_t stream_id, int32_t timeout_ms) {
    if (!S) return fail(LHR_ERR_INVALID_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(S->mu);
    if (stream_id < 0 || stream_id >= S->cfg.n_streams || S->state[stream_id] == 0)
        return fail(LHR_ERR_INVALID_ARG, "stream is not open");
    if (!S->on_demand) return fail(LHR_ERR_INVALID_ARG, "every stream was opened at creation (ring_mem_bytes = 0)");
    S->state[stream_id] = 2;  // closing: no more submissions; the ring returns when its frames are done
    maybe_release(S, stream_id);
    const bool done = S->cv_done.wait_for(lk, std::chrono::milliseconds(std::max(timeout_ms, 0)),
                                          [&] { return S->state[stream_id] == 0 || !S->error.empty(); });
    if (!S->error.empty()) return fail(LHR_ERR_CUDA, S->error);
    if (!done) return fail(LHR_ERR_TIMEOUT, "stream still has frames in flight (its ring returns when they finish)");
    return LHR_OK;
}

lhr_status lhr_server_drain(lhr_server* S, int32_t timeout_ms) {
    if (!S) return fail(LHR_ERR_INVALID_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(S->mu);
    const bool ok = S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] {
        return (S->subq.empty() && S->completed == S->submitted) || !S->error.empty();
    });
    if (!S->error.empty()) return fail(LHR_ERR_CUDA, S->error);
    if (!ok) return fail(LHR_ERR_TIMEOUT, "lhr_server_drain: work still in flight");
    return LHR_OK;
}

lhr_status lhr_server_destroy(lhr_server* S) {
    if (!S) return LHR_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->sched.joinable()) S->sched.join();
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(S->db->device);
    free_server(S);
    if (prev >= 0) cudaSetDevice(prev);
    return LHR_OK;
}

}  // extern "C"
