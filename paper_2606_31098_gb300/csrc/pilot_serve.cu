// Serving: a persistent request loop with continuous batching at pyramid-level granularity.
//
// Clients submit frames from many concurrent streams (uneven crops, hypothesis counts).
// A worker thread owns the GPU:
//   admission  a pending frame is admitted when a slot is free, its hypotheses fit in the
//              hypothesis state array and its data fit in the device arena (the HBM budget
//              given at create); admission copies the frame into the arena, where its
//              pyramid and LM state stay until it completes.
//   round      every active frame advances by one pyramid level: one graph replay uploads
//              the round's descriptors, sets up newly admitted frames, runs one persistent
//              launch in which each frame's hypotheses run that frame's current level
//              (frames at different levels share the launch), applies per-frame top-K,
//              finalises frames that finished the finest level and downloads results.
//   retire     finished frames free their slot, hypotheses and arena space; frames that
//              arrived meanwhile are admitted before the next round.
// Each frame's arithmetic is exactly that of pilot_align_solve (same kernels, same
// reduction order), so a frame's result does not depend on what else is being served.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pilot_internal.cuh"

using namespace pilot;

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

pilot_status sfail(pilot_status st, const std::string& m) {
    record_error(m.c_str());
    return st;
}

// First-fit allocator over [0, capacity) with coalescing free ranges.
class RangeAllocator {
  public:
    void reset(size_t capacity) {
        free_.clear();
        if (capacity) free_[0] = capacity;
        in_use_ = peak_ = 0;
    }
    bool alloc(size_t n, size_t* off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n, start = it->first + n;
                free_.erase(it);
                if (rest) free_[start] = rest;
                in_use_ += n;
                peak_ = std::max(peak_, in_use_);
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n) {
        if (!n) return;
        in_use_ -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t in_use() const { return in_use_; }
    size_t peak() const { return peak_; }

  private:
    std::map<size_t, size_t> free_;
    size_t in_use_ = 0, peak_ = 0;
};

size_t a256(size_t b) { return (b + 255) / 256 * 256; }

// Device bytes a frame occupies in the arena (every array rounded to 256 bytes).
size_t frame_bytes(const pilot_frame& f) {
    const size_t es = dtype_bytes(f.feat_dtype), N = f.N, C = f.C;
    size_t b = a256(sizeof(float) * 3 * N);
    if (f.point_weight) b += a256(sizeof(float) * N);
    if (f.point_valid) b += a256(N);
    for (int l = 0; l < f.L; ++l) {
        b += a256(es * N * C) + a256(es * (size_t)f.H[l] * f.W[l] * C);
        if (f.ref_scale[l]) b += a256(sizeof(float) * C);
        if (f.qry_scale[l]) b += a256(sizeof(float) * C);
        if (f.qry_conf[l]) b += a256(sizeof(float) * (size_t)f.H[l] * f.W[l]);
    }
    b += a256(sizeof(double) * 12 * (size_t)f.M);
    if (f.use_range) b += a256(sizeof(float) * (size_t)f.dsm_H * f.dsm_W);
    return b;
}

enum ReqState { kPending = 0, kActive = 1, kDone = 2, kFailed = 3 };

// levels_per_round = 0: a frame whose level work (anchors x active hypotheses) is at most this
// runs all its remaining levels in one round
constexpr long long kSmallLevelWork = 1ll << 21;

struct Request {
    uint64_t ticket = 0;
    pilot_frame src{};           // the caller's frame (pointers valid until done)
    pilot_frame dev{};           // the arena copy
    double t_submit = 0, t_admit = 0, t_done = 0;
    size_t arena_off = 0, arena_bytes = 0, hyp_off = 0;
    int slot = -1, level = 0, n_active = 0, quota = 1;
    bool initialized = false;
    long long hyp_iters = 0;
    int state = kPending;
    std::vector<double> T, cost;
    std::vector<int> n_valid, status;
    int best = -1;
};

}  // namespace

struct pilot_server {
    pilot_align_config cfg{};
    int device = 0;
    size_t budget = 0;
    int max_slots = 0, max_pending = 0;
    unsigned char* arena = nullptr;
    RangeAllocator arena_alloc, hyp_alloc;
    std::vector<int> free_slots;
    HypState* state = nullptr;
    int* active = nullptr;
    double* min_valid = nullptr;
    unsigned long long* sync = nullptr;   // level kernel: item claims, barrier arrivals, generations
    float* pose32 = nullptr;              // [job][12] FP32 poses to evaluate
    unsigned* job_meta = nullptr;         // [job] hypothesis | evaluate bit
    unsigned* flags = nullptr;            // level kernel's per-job-tile flags: completed items, then published iterations
    size_t flag_words = 0;                // words of each of the two flag arrays
    float* partial = nullptr;             // [work item][kAcc] tile records
    unsigned char* desc_dev = nullptr;
    unsigned char* desc_host = nullptr;
    size_t desc_bytes = 0, off_frames = 0, off_fr_list = 0, off_fr_item = 0, off_fr_job = 0;
    unsigned char* res_dev = nullptr;
    unsigned char* res_host = nullptr;
    size_t res_bytes = 0;
    cudaStream_t stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;
    int grid = 0;
    bool key_set = false;
    pilot_dtype dt = PILOT_F32;
    int C = 0, L = 0;
    int variant = 0;           // kVariantScaled | kVariantConf, shared by every served frame
    int levels_per_round = 1;  // pyramid levels each admitted frame advances per round; 0: by size
    int reserved_sms = 0;      // SMs' worth of CTA slots the round's persistent launch leaves free
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    pilot_status failure = PILOT_OK;
    std::string failure_msg;
    std::deque<Request*> pending;
    std::vector<Request*> running;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
    uint64_t next_ticket = 1;
    long long rounds = 0, admitted = 0, completed = 0, peak_active = 0;
    cudaEvent_t ev_begin = nullptr, ev_end = nullptr;  // bracket each round on the stream
    double round_device_ms = 0, round_wall_ms = 0;
};

namespace {

void release_buffers(pilot_server* s) {
    if (s->gexec) cudaGraphExecDestroy(s->gexec);
    if (s->graph) cudaGraphDestroy(s->graph);
    cudaFree(s->arena);
    cudaFree(s->state);
    cudaFree(s->active);
    cudaFree(s->min_valid);
    cudaFree(s->sync);
    cudaFree(s->pose32);
    cudaFree(s->job_meta);
    cudaFree(s->flags);
    cudaFree(s->partial);
    cudaFree(s->desc_dev);
    if (s->desc_host) cudaFreeHost(s->desc_host);
    cudaFree(s->res_dev);
    if (s->res_host) cudaFreeHost(s->res_host);
    if (s->ev_begin) cudaEventDestroy(s->ev_begin);
    if (s->ev_end) cudaEventDestroy(s->ev_end);
    if (s->stream) cudaStreamDestroy(s->stream);
}

// Copy one array into the arena (H2D for host frames, D2D for device frames).
template <typename T>
cudaError_t place(pilot_server* s, const Request& r, size_t* cursor, const T* src, size_t bytes,
                  const T** dst) {
    if (!src || bytes == 0) {
        *dst = nullptr;
        return cudaSuccess;
    }
    unsigned char* d = s->arena + r.arena_off + *cursor;
    *cursor += a256(bytes);
    *dst = reinterpret_cast<const T*>(d);
    return cudaMemcpyAsync(d, src, bytes, r.src.is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           s->stream);
}

cudaError_t stage_frame(pilot_server* s, Request& r) {
    const pilot_frame& f = r.src;
    pilot_frame& d = r.dev;
    d = f;
    d.is_device = 1;
    const size_t es = dtype_bytes(f.feat_dtype), N = f.N, C = f.C;
    size_t cur = 0;
    cudaError_t e = place(s, r, &cur, f.points, sizeof(float) * 3 * N, &d.points);
    if (e == cudaSuccess) e = place(s, r, &cur, f.point_weight, sizeof(float) * N, &d.point_weight);
    if (e == cudaSuccess) e = place(s, r, &cur, f.point_valid, N, &d.point_valid);
    for (int l = 0; l < f.L && e == cudaSuccess; ++l) {
        const void* p = nullptr;
        e = place(s, r, &cur, static_cast<const unsigned char*>(f.ref_feat[l]), es * N * C,
                  reinterpret_cast<const unsigned char**>(&p));
        d.ref_feat[l] = p;
        if (e == cudaSuccess)
            e = place(s, r, &cur, static_cast<const unsigned char*>(f.qry_feat[l]), es * (size_t)f.H[l] * f.W[l] * C,
                      reinterpret_cast<const unsigned char**>(&p));
        d.qry_feat[l] = p;
        if (e == cudaSuccess) e = place(s, r, &cur, f.ref_scale[l], sizeof(float) * C, &d.ref_scale[l]);
        if (e == cudaSuccess) e = place(s, r, &cur, f.qry_scale[l], sizeof(float) * C, &d.qry_scale[l]);
        if (e == cudaSuccess)
            e = place(s, r, &cur, f.qry_conf[l], sizeof(float) * (size_t)f.H[l] * f.W[l], &d.qry_conf[l]);
    }
    if (e == cudaSuccess) e = place(s, r, &cur, f.T_cw, sizeof(double) * 12 * (size_t)f.M, &d.T_cw);
    if (e == cudaSuccess && f.use_range)
        e = place(s, r, &cur, f.dsm, sizeof(float) * (size_t)f.dsm_H * f.dsm_W, &d.dsm);
    return e;
}

cudaError_t capture_round(pilot_server* s) {
    if (s->gexec) cudaGraphExecDestroy(s->gexec);
    if (s->graph) cudaGraphDestroy(s->graph);
    s->gexec = nullptr;
    s->graph = nullptr;
    int sms = 0, per_sm = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
    if (e == cudaSuccess) e = level_occupancy_query(s->dt, s->C, s->variant, &per_sm);
    if (e != cudaSuccess) return e;
    // the round's persistent launch takes every CTA slot but those of reserved_sms SMs, so
    // that the clients' work on other streams (crops, feature extraction, seeding) runs
    // beside a round instead of waiting for it; the results do not depend on the grid
    s->grid = std::max(1, sms - s->reserved_sms) * (per_sm > 0 ? per_sm : 1);
    const BatchHeader* hdr = reinterpret_cast<const BatchHeader*>(s->desc_dev);
    const FrameDesc* frames = reinterpret_cast<const FrameDesc*>(s->desc_dev + s->off_frames);
    if ((e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
    e = cudaMemcpyAsync(s->desc_dev, s->desc_host, s->desc_bytes, cudaMemcpyHostToDevice, s->stream);
    unsigned* error = reinterpret_cast<unsigned*>(s->res_dev + ResultLayout::make(s->cfg.max_hyps).bytes +
                                                  sizeof(int) * (size_t)s->max_slots);
    if (e == cudaSuccess) e = cudaMemsetAsync(error, 0, sizeof(unsigned), s->stream);
    if (e == cudaSuccess)
        e = launch_round_prepare(hdr, frames, s->state, s->active, s->cfg.min_valid_frac, s->min_valid,
                                 s->max_slots, s->stream);
    LevelArgs a{};
    a.header = hdr;
    a.frames = frames;
    a.fr_list = reinterpret_cast<const int*>(s->desc_dev + s->off_fr_list);
    a.fr_item = reinterpret_cast<const int*>(s->desc_dev + s->off_fr_item);
    a.fr_job = reinterpret_cast<const int*>(s->desc_dev + s->off_fr_job);
    a.active = s->active;
    a.state = s->state;
    a.min_valid = s->min_valid;
    a.pose32 = s->pose32;
    a.job_meta = s->job_meta;
    a.partial = s->partial;
    a.sync = s->sync;
    a.tile_done = s->flags;
    a.tile_ready = s->flags + s->flag_words;
    a.error = error;
    a.barrier_timeout_ns = kBarrierTimeoutNs;
    a.barrier_extra = 0;
    a.level = -1;
    a.list_index = 0;
    a.k_max = 0;
    LevelKeep keep{};
    for (int l = 0; l < PILOT_MAX_LEVELS; ++l) {
        a.iters[l] = s->cfg.iters_per_level[l];
        a.k_max = std::max(a.k_max, a.iters[l]);
        keep.k[l] = s->cfg.keep_top_k[l];
    }
    a.tile = kPlainTile;
    a.tiles_per_item = tiles_per_item(kPlainTile);
    a.damping_mode = s->cfg.damping_mode;
    a.huber = (float)s->cfg.huber_photo;
    a.lambda0 = s->cfg.lambda0;
    // levels_per_round sub-rounds: each advances every listed frame by one level (a frame that
    // finishes level 0 is finalised and has no jobs in the later sub-rounds)
    const int subs = s->levels_per_round > 0 ? s->levels_per_round : s->L;
    for (int sub = 0; sub < subs && e == cudaSuccess; ++sub) {
        if (sub > 0)
            e = launch_round_advance(hdr, const_cast<FrameDesc*>(frames), a.fr_list, const_cast<int*>(a.fr_item),
                                     const_cast<int*>(a.fr_job), keep, a.tile, a.tiles_per_item, s->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(s->sync, 0, sizeof(unsigned long long) * kSyncWords, s->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(s->flags, 0, sizeof(unsigned) * 2 * s->flag_words, s->stream);
        if (e == cudaSuccess) e = level_launch(s->dt, s->C, s->variant, a, s->grid, s->stream);
        if (e == cudaSuccess)
            e = launch_round_finish(hdr, frames, s->state, s->active, s->min_valid, s->res_dev, s->cfg.max_hyps,
                                    s->max_slots, std::min(s->cfg.max_hyps, kMaxFrameHyps), s->stream);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->res_host, s->res_dev, s->res_bytes, cudaMemcpyDeviceToHost, s->stream);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(s->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return e != cudaSuccess ? e : e2;
    }
    s->graph = g;
    return cudaGraphInstantiate(&s->gexec, g, 0);
}

// Admit pending frames in arrival order while a slot, hypothesis room and arena space are
// free (head-of-line: a frame that does not fit yet blocks the ones behind it).
cudaError_t admit(pilot_server* s) {
    while (!s->pending.empty() && !s->free_slots.empty()) {
        Request* r = s->pending.front();
        size_t aoff = 0, hoff = 0;
        if (!s->hyp_alloc.alloc((size_t)r->src.M, &hoff)) break;
        if (!s->arena_alloc.alloc(r->arena_bytes, &aoff)) {
            s->hyp_alloc.release(hoff, (size_t)r->src.M);
            break;
        }
        s->pending.pop_front();
        r->arena_off = aoff;
        r->hyp_off = hoff;
        r->slot = s->free_slots.back();
        s->free_slots.pop_back();
        r->level = r->src.L - 1;
        r->n_active = r->src.M;
        r->state = kActive;
        r->t_admit = now_ms();
        s->running.push_back(r);
        ++s->admitted;
        const cudaError_t e = stage_frame(s, *r);
        if (e != cudaSuccess) return e;
    }
    s->peak_active = std::max<long long>(s->peak_active, (long long)s->running.size());
    return cudaSuccess;
}

// Descriptors of one round: every slot gets a FrameDesc (idle slots do nothing); jobs are
// the active hypotheses of every running frame, frames with more anchors first.
void write_round(pilot_server* s) {
    const pilot_align_config& c = s->cfg;
    BatchHeader* hdr = reinterpret_cast<BatchHeader*>(s->desc_host);
    FrameDesc* fds = reinterpret_cast<FrameDesc*>(s->desc_host + s->off_frames);
    int* list = reinterpret_cast<int*>(s->desc_host + s->off_fr_list);
    int* items = reinterpret_cast<int*>(s->desc_host + s->off_fr_item);
    int* jobs = reinterpret_cast<int*>(s->desc_host + s->off_fr_job);
    memset(hdr, 0, sizeof(BatchHeader));
    hdr->n_frames = s->max_slots;
    memset(fds, 0, sizeof(FrameDesc) * (size_t)s->max_slots);
    std::vector<Request*> order = s->running;
    std::stable_sort(order.begin(), order.end(), [](Request* a, Request* b) { return a->src.N > b->src.N; });
    // work items of one tile when the round's items of the default size would not give every
    // CTA two (a light round: more, smaller items spread its gathers over the device); the
    // records and their sums do not depend on it
    int tpi = tiles_per_item(kPlainTile);
    long long total_items = 0;
    for (Request* r : order) total_items += frame_items(r->n_active, r->dev.N, kPlainTile, tpi);
    if (total_items < 2ll * s->grid) tpi = 1;
    hdr->tiles_per_item = tpi;
    int nl = 0;
    items[0] = jobs[0] = 0;
    for (Request* r : order) {
        const pilot_frame& f = r->dev;
        FrameDesc& d = fds[r->slot];
        const size_t N = (size_t)f.N;
        d.px = f.points;
        d.py = f.points ? f.points + N : nullptr;
        d.pz = f.points ? f.points + 2 * N : nullptr;
        d.weight = f.point_weight;
        d.valid = f.point_valid;
        d.N = f.N;
        d.M = f.M;
        for (int l = 0; l < f.L; ++l) {
            d.ref[l] = f.ref_feat[l];
            d.qry[l] = f.qry_feat[l];
            d.rscale[l] = f.ref_scale[l];
            d.qscale[l] = f.qry_scale[l];
            d.conf[l] = f.qry_conf[l];
            d.H[l] = f.H[l];
            d.W[l] = f.W[l];
            const double sc = ldexp(1.0, -l);
            d.fx[l] = (float)(f.fx * sc);
            d.fy[l] = (float)(f.fy * sc);
            d.cx[l] = (float)(f.cx * sc);
            d.cy[l] = (float)(f.cy * sc);
        }
        d.T_cw = f.T_cw;
        d.hyp_offset = (int)r->hyp_off;
        d.level = r->level;
        d.n_active = r->n_active;
        const int K = c.keep_top_k[r->level];
        d.keep = K;
        d.flags = (r->initialized ? 0 : kFlagInit) | ((r->level > 0 && K > 0 && K < r->n_active) ? kFlagPrune : 0) |
                  (r->level == 0 ? kFlagFinalize : 0);
        d.prior = frame_prior(c, &f, f.dsm);
        // levels this round: fixed, or (0) all remaining ones for a frame whose level work
        // (anchors x active hypotheses) is small and one level otherwise
        r->quota = s->levels_per_round > 0
                       ? s->levels_per_round
                       : ((long long)f.N * r->n_active <= kSmallLevelWork ? r->level + 1 : 1);
        d.quota = r->quota;
        list[nl] = r->slot;
        jobs[nl + 1] = jobs[nl] + r->n_active;
        items[nl + 1] = items[nl] + frame_items(r->n_active, f.N, kPlainTile, tpi);
        ++nl;
    }
    hdr->n_listed[0] = nl;
}

// After a round: advance levels, collect finished frames.
void after_round(pilot_server* s) {
    const pilot_align_config& c = s->cfg;
    const ResultLayout rl = ResultLayout::make(c.max_hyps);
    const unsigned char* res = s->res_host;
    const int* best = reinterpret_cast<const int*>(res + rl.bytes);
    std::vector<Request*> still;
    const double t = now_ms();
    for (Request* r : s->running) {
        // the round advanced every listed frame by up to levels_per_round levels
        r->initialized = true;
        bool finished = false;
        for (int sub = 0; sub < r->quota; ++sub) {
            r->hyp_iters += (long long)r->n_active * c.iters_per_level[r->level];
            const int K = c.keep_top_k[r->level];
            if (r->level > 0 && K > 0 && K < r->n_active) r->n_active = K;
            if (r->level == 0) {
                finished = true;
                break;
            }
            --r->level;
        }
        if (!finished) {
            still.push_back(r);
            continue;
        }
        const int M = r->src.M;
        const size_t o = r->hyp_off;
        r->T.assign(reinterpret_cast<const double*>(res + rl.off_T) + 12 * o,
                    reinterpret_cast<const double*>(res + rl.off_T) + 12 * (o + M));
        r->cost.assign(reinterpret_cast<const double*>(res + rl.off_cost) + o,
                       reinterpret_cast<const double*>(res + rl.off_cost) + o + M);
        r->n_valid.assign(reinterpret_cast<const int*>(res + rl.off_nvalid) + o,
                          reinterpret_cast<const int*>(res + rl.off_nvalid) + o + M);
        r->status.assign(reinterpret_cast<const int*>(res + rl.off_status) + o,
                         reinterpret_cast<const int*>(res + rl.off_status) + o + M);
        r->best = best[r->slot];
        r->state = kDone;
        r->t_done = t;
        s->arena_alloc.release(r->arena_off, r->arena_bytes);
        s->hyp_alloc.release(r->hyp_off, (size_t)M);
        s->free_slots.push_back(r->slot);
        ++s->completed;
    }
    s->running.swap(still);
}

void fail_all(pilot_server* s, cudaError_t e, const char* what) {
    s->failure = PILOT_ECUDA;
    s->failure_msg = std::string(what) + ": " + cudaGetErrorString(e);
    for (Request* r : s->running) r->state = kFailed;
    for (Request* r : s->pending) r->state = kFailed;
    s->running.clear();
    s->pending.clear();
}

void worker_main(pilot_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lock(s->mu);
    while (!s->stop) {
        if (s->failure == PILOT_OK) {
            const cudaError_t e = admit(s);
            if (e != cudaSuccess) {
                fail_all(s, e, "frame staging");
                s->cv_done.notify_all();
                continue;
            }
        }
        if (s->running.empty()) {
            s->cv_work.wait_for(lock, std::chrono::milliseconds(2));
            continue;
        }
        write_round(s);
        lock.unlock();
        const double t0 = now_ms();
        cudaError_t e = cudaEventRecord(s->ev_begin, s->stream);
        if (e == cudaSuccess) e = cudaGraphLaunch(s->gexec, s->stream);
        if (e == cudaSuccess) e = cudaEventRecord(s->ev_end, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        float dev_ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&dev_ms, s->ev_begin, s->ev_end);
        const double t1 = now_ms();
        lock.lock();
        ++s->rounds;
        s->round_device_ms += dev_ms;
        s->round_wall_ms += t1 - t0;
        const unsigned* barrier_error = reinterpret_cast<const unsigned*>(
            s->res_host + ResultLayout::make(s->cfg.max_hyps).bytes + sizeof(int) * (size_t)s->max_slots);
        if (e != cudaSuccess) {
            fail_all(s, e, "serving round");
        } else if (*barrier_error != 0) {
            fail_all(s, cudaErrorTimeout, "serving round (level kernel grid barrier timed out)");
        } else {
            after_round(s);
        }
        s->cv_done.notify_all();
    }
}

}  // namespace

extern "C" {

pilot_status pilot_serve_create(const pilot_align_config* cfg_in, size_t hbm_budget, int max_slots,
                                pilot_server** out) {
    if (!cfg_in || !out) return sfail(PILOT_EINVAL, "config or out is NULL");
    *out = nullptr;
    pilot_align_config cfg = config_with_defaults(*cfg_in);
    pilot_status st = check_config(cfg);
    if (st != PILOT_OK) return st;
    if (max_slots < 1 || max_slots > 4096) return sfail(PILOT_EINVAL, "max_slots must be in [1, 4096]");
    if (hbm_budget < (1u << 20)) return sfail(PILOT_EINVAL, "hbm_budget below 1 MiB");
    std::unique_ptr<pilot_server> s(new pilot_server());
    s->cfg = cfg;
    s->budget = hbm_budget;
    s->max_slots = max_slots;
    s->max_pending = 4 * max_slots + 64;
    cudaError_t e = cudaGetDevice(&s->device);
    auto bad = [&](const char* what) {
        std::string m = std::string(what) + ": " + cudaGetErrorString(e);
        release_buffers(s.get());
        return sfail(e == cudaErrorMemoryAllocation ? PILOT_ENOMEM : PILOT_ECUDA, m);
    };
    if (e != cudaSuccess) return bad("cudaGetDevice");
    const size_t H = (size_t)cfg.max_hyps;
    s->off_frames = a256(sizeof(BatchHeader));
    s->off_fr_list = a256(s->off_frames + sizeof(FrameDesc) * (size_t)max_slots);
    s->off_fr_item = a256(s->off_fr_list + sizeof(int) * (size_t)max_slots);
    s->off_fr_job = a256(s->off_fr_item + sizeof(int) * ((size_t)max_slots + 1));
    s->desc_bytes = a256(s->off_fr_job + sizeof(int) * ((size_t)max_slots + 1));
    // result block, the best index per slot, then the barrier error word
    s->res_bytes = ResultLayout::make(cfg.max_hyps).bytes + sizeof(int) * ((size_t)max_slots + 1);
    const size_t max_tiles = cfg.max_points > 0 ? ((size_t)cfg.max_points + kPlainTile - 1) / kPlainTile : 1;
    if ((e = cudaMalloc((void**)&s->arena, hbm_budget)) != cudaSuccess) return bad("arena allocation");
    if ((e = cudaMalloc((void**)&s->state, sizeof(HypState) * H)) != cudaSuccess) return bad("state allocation");
    if ((e = cudaMalloc((void**)&s->active, sizeof(int) * H)) != cudaSuccess) return bad("active lists");
    if ((e = cudaMalloc((void**)&s->min_valid, sizeof(double) * (size_t)max_slots)) != cudaSuccess) return bad("thresholds");
    if ((e = cudaMalloc((void**)&s->sync, sizeof(unsigned long long) * kSyncWords)) != cudaSuccess)
        return bad("level counters");
    if ((e = cudaMalloc((void**)&s->pose32, sizeof(float) * 12 * H)) != cudaSuccess) return bad("candidates");
    if ((e = cudaMalloc((void**)&s->job_meta, sizeof(unsigned) * H)) != cudaSuccess) return bad("job table");
    s->flag_words = level_flag_words(cfg.max_hyps, max_slots, (int)max_tiles);
    if ((e = cudaMalloc((void**)&s->flags, sizeof(unsigned) * 2 * s->flag_words)) != cudaSuccess)
        return bad("job tile flags");
    if ((e = cudaMalloc((void**)&s->partial, sizeof(float) * kAcc * (H + (size_t)(kHypTile - 1) * max_slots) *
                                                 (max_tiles + tiles_per_item(kPlainTile)))) != cudaSuccess)
        return bad("tile records");
    if ((e = cudaMalloc((void**)&s->desc_dev, s->desc_bytes)) != cudaSuccess) return bad("descriptors");
    if ((e = cudaMallocHost((void**)&s->desc_host, s->desc_bytes)) != cudaSuccess) return bad("descriptor staging");
    if ((e = cudaMalloc((void**)&s->res_dev, s->res_bytes)) != cudaSuccess) return bad("results");
    if ((e = cudaMallocHost((void**)&s->res_host, s->res_bytes)) != cudaSuccess) return bad("result staging");
    if ((e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking)) != cudaSuccess) return bad("stream");
    if ((e = cudaEventCreate(&s->ev_begin)) != cudaSuccess) return bad("round events");
    if ((e = cudaEventCreate(&s->ev_end)) != cudaSuccess) return bad("round events");
    s->arena_alloc.reset(hbm_budget);
    s->hyp_alloc.reset(H);
    for (int i = max_slots - 1; i >= 0; --i) s->free_slots.push_back(i);
    pilot_server* raw = s.release();
    raw->worker = std::thread(worker_main, raw);
    *out = raw;
    return PILOT_OK;
}

pilot_status pilot_serve_submit(pilot_server* s, const pilot_frame* f, uint64_t* ticket) {
    if (!s || !f || !ticket) return sfail(PILOT_EINVAL, "server, frame or ticket is NULL");
    pilot_status st = check_frame(s->cfg, f);
    if (st != PILOT_OK) return st;
    if (f->M == 0) return sfail(PILOT_EINVAL, "a served frame needs at least one hypothesis");
    if (f->M > kMaxFrameHyps) return sfail(PILOT_EINVAL, "M above 8192");
    const int variant = frame_variant(f);
    if (variant == -1) return sfail(PILOT_EINVAL, "give both scale arrays on every level, or none");
    if (variant == -2) return sfail(PILOT_EINVAL, "give a confidence map on every level, or none");
    const size_t bytes = frame_bytes(*f);
    if (bytes > s->budget) return sfail(PILOT_EINVAL, "the frame needs more device memory than the whole budget");
    std::unique_lock<std::mutex> lock(s->mu);
    if (s->failure != PILOT_OK) return sfail(s->failure, s->failure_msg);
    if (!s->key_set) {
        int prev = -1;
        cudaGetDevice(&prev);
        if (prev != s->device) cudaSetDevice(s->device);
        s->dt = f->feat_dtype;
        s->C = f->C;
        s->L = f->L;
        s->variant = variant;
        const cudaError_t e = capture_round(s);
        if (prev >= 0 && prev != s->device) cudaSetDevice(prev);
        if (e != cudaSuccess) return sfail(PILOT_ECUDA, std::string("round graph: ") + cudaGetErrorString(e));
        s->key_set = true;
    } else if (f->feat_dtype != s->dt || f->C != s->C || f->L != s->L || variant != s->variant) {
        return sfail(PILOT_EINVAL, "every served frame must share C, L, feat_dtype, scale and confidence presence");
    }
    if ((int)s->pending.size() >= s->max_pending) return sfail(PILOT_EBUSY, "pending queue full");
    std::unique_ptr<Request> r(new Request());
    r->ticket = s->next_ticket++;
    r->src = *f;
    r->arena_bytes = bytes;
    r->t_submit = now_ms();
    *ticket = r->ticket;
    s->pending.push_back(r.get());
    s->reqs.emplace(r->ticket, std::move(r));
    s->cv_work.notify_one();
    return PILOT_OK;
}

pilot_status pilot_serve_poll(pilot_server* s, uint64_t ticket, pilot_result* res, int* done,
                              double* latency_ms) {
    if (!s || !done) return sfail(PILOT_EINVAL, "server or done is NULL");
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return sfail(PILOT_EINVAL, "unknown ticket");
    Request* r = it->second.get();
    *done = 0;
    if (r->state == kFailed) {
        s->reqs.erase(it);
        return sfail(PILOT_ECUDA, s->failure_msg);
    }
    if (r->state != kDone) return PILOT_OK;
    *done = 1;
    if (res) {
        const int M = r->src.M;
        if (res->T_cw) memcpy(res->T_cw, r->T.data(), sizeof(double) * 12 * M);
        if (res->cost) memcpy(res->cost, r->cost.data(), sizeof(double) * M);
        if (res->n_valid) memcpy(res->n_valid, r->n_valid.data(), sizeof(int) * M);
        if (res->hyp_status) memcpy(res->hyp_status, r->status.data(), sizeof(int) * M);
        if (res->best) *res->best = r->best;
        if (res->hyp_iters) *res->hyp_iters = r->hyp_iters;
    }
    if (latency_ms) *latency_ms = r->t_done - r->t_submit;
    s->reqs.erase(it);
    return PILOT_OK;
}

pilot_status pilot_serve_wait(pilot_server* s, uint64_t ticket, pilot_result* res, double* latency_ms,
                              int timeout_ms) {
    if (!s) return sfail(PILOT_EINVAL, "server is NULL");
    const double deadline = now_ms() + timeout_ms;
    for (;;) {
        int done = 0;
        pilot_status st = pilot_serve_poll(s, ticket, res, &done, latency_ms);
        if (st != PILOT_OK || done) return st;
        std::unique_lock<std::mutex> lock(s->mu);
        if (now_ms() >= deadline) return sfail(PILOT_ETIMEOUT, "wait timed out");
        s->cv_done.wait_for(lock, std::chrono::milliseconds(1));
    }
}

pilot_status pilot_serve_set_levels_per_round(pilot_server* s, int levels) {
    if (!s) return sfail(PILOT_EINVAL, "server is NULL");
    if (levels < 0 || levels > PILOT_MAX_LEVELS) return sfail(PILOT_EINVAL, "levels_per_round must be in [0, 4]");
    std::unique_lock<std::mutex> lock(s->mu);
    if (s->key_set) return sfail(PILOT_EINVAL, "set levels_per_round before the first frame is submitted");
    s->levels_per_round = levels;
    return PILOT_OK;
}

pilot_status pilot_serve_set_reserved_sms(pilot_server* s, int n_sms) {
    if (!s) return sfail(PILOT_EINVAL, "server is NULL");
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess)
        return sfail(PILOT_ECUDA, "SM count query failed");
    if (n_sms < 0 || n_sms >= sms) return sfail(PILOT_EINVAL, "reserved SMs must be in [0, SM count)");
    std::unique_lock<std::mutex> lock(s->mu);
    if (s->key_set) return sfail(PILOT_EINVAL, "set reserved SMs before the first frame is submitted");
    s->reserved_sms = n_sms;
    return PILOT_OK;
}

pilot_status pilot_serve_get_stats(pilot_server* s, pilot_serve_stats* out) {
    if (!s || !out) return sfail(PILOT_EINVAL, "server or stats is NULL");
    std::unique_lock<std::mutex> lock(s->mu);
    out->rounds = s->rounds;
    out->admitted = s->admitted;
    out->completed = s->completed;
    out->pending = (long long)s->pending.size();
    out->active = (long long)s->running.size();
    out->peak_active = s->peak_active;
    out->arena_bytes_in_use = (long long)s->arena_alloc.in_use();
    out->arena_bytes_peak = (long long)s->arena_alloc.peak();
    out->round_device_ms = s->round_device_ms;
    out->round_wall_ms = s->round_wall_ms;
    return PILOT_OK;
}

void pilot_serve_destroy(pilot_server* s) {
    if (!s) return;
    {
        std::unique_lock<std::mutex> lock(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->device);
    cudaStreamSynchronize(s->stream);
    release_buffers(s);
    delete s;
}

}  // extern "C"
