// Host runtime of the C-ABI declared in include/pilot_align.h: validation, workspace,
// input staging, and the per-level launch sequence of the LM solve.
//
// One solve of one frame (Sec. IV-E, Eq. 7-9), all on the caller's stream:
//   count_valid  (min_valid = frac x valid anchors)    hyp_init (FP64 state from T_cw)
//   for l = L-1 .. 0:
//     level_init (lambda = lambda0, candidate = T)
//     build(l) with the FP64 step fused (init: store E(T), solve the first candidate)
//     repeat iters[l] times: build(l) at the candidates, fused step (accept or reject,
//       solve the next candidate)
//     optional prune (keep_top_k[l])
//   finalize (statuses, argmin) -> one device-to-host copy of the result block
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <string>
#include <vector>

#include "pilot_internal.cuh"

using namespace pilot;

namespace {

thread_local std::string g_last_error;

pilot_status fail(pilot_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

pilot_status cuda_fail(cudaError_t e, const char* what) {
    return fail(e == cudaErrorMemoryAllocation ? PILOT_ENOMEM : PILOT_ECUDA, "%s: %s (%s)", what,
                cudaGetErrorString(e), cudaGetErrorName(e));
}

#define PILOT_CUDA(expr, what)                              \
    do {                                                    \
        cudaError_t e_ = (expr);                            \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);  \
    } while (0)

constexpr int kTile = 1024;          // default anchors per build-pass tile
constexpr int kMaxStreams = 4;       // plain form: most concurrent hypothesis parts
constexpr int kDefaultStreams = 2;   // plain form: parts when the schedule says 0
constexpr int kMinTile = 512;        // smallest tile the autotuner tries (sizes the workspace)

bool channels_supported(int C) { return C == 4 || C == 8 || C == 16 || C == 32 || C == 64; }

size_t dtype_size(pilot_dtype dt) {
    switch (dt) {
        case PILOT_F32: return 4;
        case PILOT_BF16:
        case PILOT_F16: return 2;
        case PILOT_FP8E4M3: return 1;
    }
    return 0;
}

pilot_align_config with_defaults(const pilot_align_config& in) {
    pilot_align_config c = in;
    if (c.lambda0 == 0.0) c.lambda0 = 1e-3;
    if (c.huber_photo == 0.0) c.huber_photo = 0.1;
    if (c.huber_grav == 0.0) c.huber_grav = 0.1;
    if (c.huber_range == 0.0) c.huber_range = 1.0;
    if (c.max_points == 0) c.max_points = 1 << 18;
    if (c.max_hyps == 0) c.max_hyps = 256;
    if (c.max_channels == 0) c.max_channels = 32;
    if (c.max_frames == 0) c.max_frames = 64;
    return c;
}

pilot_status validate_config(const pilot_align_config& c) {
    for (int l = 0; l < PILOT_MAX_LEVELS; ++l) {
        if (c.iters_per_level[l] < 0 || c.iters_per_level[l] > 100000)
            return fail(PILOT_EINVAL, "iters_per_level[%d] = %d out of [0, 100000]", l, c.iters_per_level[l]);
        if (c.keep_top_k[l] < 0) return fail(PILOT_EINVAL, "keep_top_k[%d] < 0", l);
    }
    if (!(c.lambda0 > 0.0) || !isfinite(c.lambda0)) return fail(PILOT_EINVAL, "lambda0 must be > 0");
    if (c.damping_mode != 0 && c.damping_mode != 1) return fail(PILOT_EINVAL, "damping_mode must be 0 or 1");
    if (!(c.huber_photo > 0.0) || !(c.huber_grav > 0.0) || !(c.huber_range > 0.0))
        return fail(PILOT_EINVAL, "Huber thresholds must be > 0");
    if (!(c.min_valid_frac >= 0.0 && c.min_valid_frac <= 1.0))
        return fail(PILOT_EINVAL, "min_valid_frac must be in [0, 1]");
    if (!(c.gate_grav >= 0.0 && isfinite(c.gate_grav)) || !(c.gate_range >= 0.0 && isfinite(c.gate_range)))
        return fail(PILOT_EINVAL, "prior gates must be finite and >= 0");
    if (c.max_points < 0 || c.max_hyps < 1) return fail(PILOT_EINVAL, "max_points >= 0 and max_hyps >= 1 required");
    if (!channels_supported(c.max_channels))
        return fail(PILOT_EINVAL, "max_channels must be one of 4, 8, 16, 32, 64");
    if (c.max_frames < 1 || c.max_frames > 65536) return fail(PILOT_EINVAL, "max_frames must be in [1, 65536]");
    return PILOT_OK;
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

pilot_status validate_frame(const pilot_align_config& c, const pilot_frame* f) {
    if (!f) return fail(PILOT_EINVAL, "frame is NULL");
    if (f->N < 0 || f->N > c.max_points)
        return fail(PILOT_EINVAL, "N = %d outside [0, max_points = %d]", f->N, c.max_points);
    if (f->M < 0 || f->M > c.max_hyps) return fail(PILOT_EINVAL, "M = %d outside [0, max_hyps = %d]", f->M, c.max_hyps);
    if (!channels_supported(f->C)) return fail(PILOT_EINVAL, "C = %d unsupported (4, 8, 16, 32, 64)", f->C);
    if (f->C > c.max_channels) return fail(PILOT_EINVAL, "C = %d above max_channels = %d", f->C, c.max_channels);
    if (f->L < 1 || f->L > PILOT_MAX_LEVELS) return fail(PILOT_EINVAL, "L = %d outside [1, %d]", f->L, PILOT_MAX_LEVELS);
    const size_t es = dtype_size(f->feat_dtype);
    if (es == 0) return fail(PILOT_EINVAL, "feat_dtype %d unknown", (int)f->feat_dtype);
    if (f->N > 0 && !f->points) return fail(PILOT_EINVAL, "points is NULL");
    if (f->M > 0 && !f->T_cw) return fail(PILOT_EINVAL, "T_cw is NULL");
    if (!(f->fx > 0.0 && f->fy > 0.0 && isfinite(f->fx) && isfinite(f->fy) && isfinite(f->cx) && isfinite(f->cy)))
        return fail(PILOT_EINVAL, "intrinsics must be finite with fx, fy > 0");
    for (int l = 0; l < f->L; ++l) {
        if (f->H[l] < 2 || f->W[l] < 2) return fail(PILOT_EINVAL, "level %d map %dx%d: both sides must be >= 2", l, f->H[l], f->W[l]);
        if ((double)f->H[l] * f->W[l] * f->C >= 2147483647.0)
            return fail(PILOT_EINVAL, "level %d map has 2^31 or more elements", l);
        if (!f->qry_feat[l]) return fail(PILOT_EINVAL, "qry_feat[%d] is NULL", l);
        if (f->N > 0 && !f->ref_feat[l]) return fail(PILOT_EINVAL, "ref_feat[%d] is NULL", l);
        // device maps are read with loads of up to 32 bytes; host frames are staged into
        // the solver's own (aligned) buffers
        const size_t fa = f->is_device ? 32 : 16;
        if (!aligned(f->qry_feat[l], fa) || (f->ref_feat[l] && !aligned(f->ref_feat[l], fa)))
            return fail(PILOT_EINVAL, "level %d feature pointers must be %d-byte aligned", l, (int)fa);
        if ((f->qry_scale[l] && !aligned(f->qry_scale[l], 16)) || (f->ref_scale[l] && !aligned(f->ref_scale[l], 16)))
            return fail(PILOT_EINVAL, "level %d scale pointers must be 16-byte aligned", l);
        if (f->qry_conf[l] && !aligned(f->qry_conf[l], 4))
            return fail(PILOT_EINVAL, "level %d confidence map must be 4-byte aligned", l);
    }
    if (f->use_gravity) {
        for (int i = 0; i < 3; ++i)
            if (!isfinite(f->gravity_cam[i]) || !isfinite(f->gravity_world[i]))
                return fail(PILOT_EINVAL, "gravity vectors must be finite");
        if (!(f->w_grav >= 0.0)) return fail(PILOT_EINVAL, "w_grav must be >= 0");
    }
    if (f->use_range) {
        if (!f->dsm || f->dsm_H < 2 || f->dsm_W < 2) return fail(PILOT_EINVAL, "range prior needs a DSM of at least 2x2");
        if (!(f->dsm_gsd > 0.0) || !isfinite(f->dsm_x0) || !isfinite(f->dsm_y0))
            return fail(PILOT_EINVAL, "DSM geometry must be finite with gsd > 0");
        if (!isfinite(f->range_m) || !(f->w_range >= 0.0)) return fail(PILOT_EINVAL, "range_m finite and w_range >= 0 required");
    }
    return PILOT_OK;
}

struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
};

enum StageSlot { kStPoints, kStWeight, kStValid, kStT, kStDsm, kStRef0, kStQry0 = kStRef0 + PILOT_MAX_LEVELS,
                 kStRs0 = kStQry0 + PILOT_MAX_LEVELS, kStQs0 = kStRs0 + PILOT_MAX_LEVELS,
                 kStConf0 = kStQs0 + PILOT_MAX_LEVELS, kStCount = kStConf0 + PILOT_MAX_LEVELS };

}  // namespace

struct pilot_align_handle {
    pilot_align_config cfg{};
    int device = 0;
    int max_tiles = 0;
    HypState* state = nullptr;
    float* pose32 = nullptr;
    float* partial = nullptr;
    int* active[2] = {nullptr, nullptr};
    double* Tin = nullptr;
    double* eval_out = nullptr;
    double* min_valid = nullptr;
    unsigned* tickets = nullptr;
    float* ones = nullptr;
    unsigned char* res_dev = nullptr;
    unsigned char* res_host = nullptr;
    DevBuf stage[kStCount];
    std::vector<cudaEvent_t> events;
    // batched form
    unsigned char* bdesc_dev = nullptr;
    unsigned char* bdesc_host = nullptr;
    size_t bdesc_bytes = 0;
    unsigned char* bres_dev = nullptr;
    unsigned char* bres_host = nullptr;
    size_t bres_bytes = 0;
    int* bactive = nullptr;
    double* bmin_valid = nullptr;
    unsigned long long* bsync = nullptr;   // per level: item claims, barrier arrivals, generations
    unsigned* bjob_meta = nullptr;         // per job of a level launch: hypothesis | evaluate bit
    unsigned* bflags = nullptr;            // level kernel's per-job-tile flags: completed items, then published iterations
    size_t bflag_words = 0;                // words of each of the two flag arrays
    double flag_selftest_ms = 0;           // > 0 during pilot_align_selftest_flag_timeout: unpublishable flags
    cudaStream_t bstream = nullptr;
    // plain form, multi-stream schedule: extra streams, a fork event and their join events
    cudaStream_t pstream[kMaxStreams - 1] = {};
    // host frames: stream for the finer levels' copies and one event per level
    cudaStream_t cstream = nullptr;
    cudaEvent_t level_ready[PILOT_MAX_LEVELS] = {};
    cudaEvent_t pfork = nullptr;
    cudaEvent_t pjoin[kMaxStreams - 1] = {};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    long long graph_key = -1;
    int level_grid = 0;
    // autotuned schedules by frame-shape key; a forced schedule while tuning
    std::map<long long, pilot_schedule> tuned;
    bool forcing = false;
    pilot_schedule forced{};
    int build_launches = 0;
    int total_launches = 0;
    double build_ms = 0.0;
};

namespace {

// Device view of a frame: caller pointers (is_device) or staged copies.
struct DevFrame {
    const float* points = nullptr;
    const float* weight = nullptr;
    const uint8_t* valid = nullptr;
    const double* T = nullptr;
    const float* dsm = nullptr;
    const void* ref[PILOT_MAX_LEVELS] = {};
    const void* qry[PILOT_MAX_LEVELS] = {};
    const float* rs[PILOT_MAX_LEVELS] = {};
    const float* qs[PILOT_MAX_LEVELS] = {};
    const float* conf[PILOT_MAX_LEVELS] = {};
};

pilot_status stage_copy(pilot_align_handle* h, int slot, const void* src, size_t bytes,
                        cudaStream_t s, const void** out) {
    if (!src || bytes == 0) {
        *out = nullptr;
        return PILOT_OK;
    }
    DevBuf& b = h->stage[slot];
    if (b.bytes < bytes) {
        if (b.ptr) cudaFree(b.ptr);
        b.ptr = nullptr;
        b.bytes = 0;
        PILOT_CUDA(cudaMalloc(&b.ptr, bytes), "staging allocation");
        b.bytes = bytes;
    }
    PILOT_CUDA(cudaMemcpyAsync(b.ptr, src, bytes, cudaMemcpyHostToDevice, s), "host-to-device copy");
    *out = b.ptr;
    return PILOT_OK;
}

// Device view of frame f.  A host frame is staged into the handle's buffers with
// asynchronous copies on s; when `fine` is given, the maps and references of every level but
// the coarsest go on that second stream instead, finest last, and level_ready[l] is recorded
// there after level l, so that the coarse levels' solve overlaps the finer levels' copies.
pilot_status bind_frame(pilot_align_handle* h, const pilot_frame* f, cudaStream_t s, DevFrame* d,
                        bool copy_T, cudaStream_t fine = nullptr, cudaEvent_t* level_ready = nullptr) {
    const size_t es = dtype_size(f->feat_dtype);
    const size_t N = (size_t)f->N, C = (size_t)f->C;
    if (f->is_device) {
        d->points = f->points;
        d->weight = f->point_weight;
        d->valid = f->point_valid;
        d->T = f->T_cw;
        d->dsm = f->use_range ? f->dsm : nullptr;
        for (int l = 0; l < f->L; ++l) {
            d->ref[l] = f->ref_feat[l];
            d->qry[l] = f->qry_feat[l];
            d->rs[l] = f->ref_scale[l];
            d->qs[l] = f->qry_scale[l];
            d->conf[l] = f->qry_conf[l];
        }
        return PILOT_OK;
    }
    pilot_status st;
    const void* p;
#define STAGE(slot, src, bytes, dst, type)                                  \
    if ((st = stage_copy(h, slot, src, bytes, s, &p)) != PILOT_OK) return st; \
    dst = static_cast<type>(p);
    STAGE(kStPoints, f->points, sizeof(float) * 3 * N, d->points, const float*);
    STAGE(kStWeight, f->point_weight, sizeof(float) * N, d->weight, const float*);
    STAGE(kStValid, f->point_valid, N, d->valid, const uint8_t*);
    if (copy_T) {
        STAGE(kStT, f->T_cw, sizeof(double) * 12 * (size_t)f->M, d->T, const double*);
    }
    if (f->use_range) {
        STAGE(kStDsm, f->dsm, sizeof(float) * (size_t)f->dsm_H * f->dsm_W, d->dsm, const float*);
    }
    for (int l = f->L - 1; l >= 0; --l) {
        const cudaStream_t sl = (fine && l < f->L - 1) ? fine : s;
        if ((st = stage_copy(h, kStRef0 + l, f->ref_feat[l], es * N * C, sl, &p)) != PILOT_OK) return st;
        d->ref[l] = p;
        if ((st = stage_copy(h, kStQry0 + l, f->qry_feat[l], es * (size_t)f->H[l] * f->W[l] * C, sl, &p)) != PILOT_OK)
            return st;
        d->qry[l] = p;
        if ((st = stage_copy(h, kStRs0 + l, f->ref_scale[l], sizeof(float) * C, sl, &p)) != PILOT_OK) return st;
        d->rs[l] = static_cast<const float*>(p);
        if ((st = stage_copy(h, kStQs0 + l, f->qry_scale[l], sizeof(float) * C, sl, &p)) != PILOT_OK) return st;
        d->qs[l] = static_cast<const float*>(p);
        if ((st = stage_copy(h, kStConf0 + l, f->qry_conf[l], sizeof(float) * (size_t)f->H[l] * f->W[l], sl, &p)) !=
            PILOT_OK)
            return st;
        d->conf[l] = static_cast<const float*>(p);
        if (sl == fine) PILOT_CUDA(cudaEventRecord(level_ready[l], fine), "level copy event");
    }
#undef STAGE
    return PILOT_OK;
}

BuildParams build_params(pilot_align_handle* h, const pilot_frame* f, const DevFrame& d, int level,
                         int n_active, const int* active, int tile = kTile) {
    BuildParams b{};
    const size_t N = (size_t)f->N;
    b.px = d.points;
    b.py = d.points ? d.points + N : nullptr;
    b.pz = d.points ? d.points + 2 * N : nullptr;
    b.weight = d.weight;
    b.valid = d.valid;
    b.qry = d.qry[level];
    b.ref = d.ref[level];
    // scales: both or neither (a missing one reads as ones)
    if (d.qs[level] || d.rs[level]) {
        b.qscale = d.qs[level] ? d.qs[level] : h->ones;
        b.rscale = d.rs[level] ? d.rs[level] : h->ones;
    }
    b.conf = d.conf[level];
    b.N = f->N;
    b.C = f->C;
    b.H = f->H[level];
    b.W = f->W[level];
    const double s = ldexp(1.0, -level);      // K_l = diag(2^-l, 2^-l, 1) K_0
    b.fx = (float)(f->fx * s);
    b.fy = (float)(f->fy * s);
    b.cx = (float)(f->cx * s);
    b.cy = (float)(f->cy * s);
    b.huber = (float)h->cfg.huber_photo;
    b.pose32 = h->pose32;
    b.active_idx = active;
    b.state = h->state;
    b.partial = h->partial;
    b.n_active = n_active;
    b.tile = tile;
    b.n_tiles = f->N > 0 ? (f->N + tile - 1) / tile : 1;
    return b;
}

PriorParams prior_params(const pilot_align_config& c, const pilot_frame* f, const DevFrame& d) {
    PriorParams pp{};
    pp.use_gravity = f->use_gravity;
    for (int i = 0; i < 3; ++i) {
        pp.g_cam[i] = f->gravity_cam[i];
        pp.g_world[i] = f->gravity_world[i];
    }
    pp.w_grav = f->w_grav;
    pp.huber_grav = c.huber_grav;
    pp.use_range = f->use_range;
    if (f->use_range) {
        // Eq. 4: v = K^-1 p_c / ||K^-1 p_c||, p_c the level-0 image centre
        const double k[3] = {(0.5 * f->W[0] - f->cx) / f->fx, (0.5 * f->H[0] - f->cy) / f->fy, 1.0};
        const double nk = sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
        for (int i = 0; i < 3; ++i) pp.q[i] = f->range_m * k[i] / nk;
    }
    pp.w_range = f->w_range;
    pp.huber_range = c.huber_range;
    pp.gate_grav = c.gate_grav;
    pp.gate_range = c.gate_range;
    pp.dsm = d.dsm;
    pp.dsm_H = f->dsm_H;
    pp.dsm_W = f->dsm_W;
    pp.dsm_x0 = f->dsm_x0;
    pp.dsm_y0 = f->dsm_y0;
    pp.dsm_gsd = f->dsm_gsd;
    pp.dsm_inv_gsd = 1.0 / f->dsm_gsd;
    return pp;
}

cudaError_t dispatch_build(pilot_dtype dt, const BuildParams& b, cudaStream_t s) {
    switch (dt) {
        case PILOT_F32: return launch_build_dtype<PILOT_F32>(b, s);
        case PILOT_BF16: return launch_build_dtype<PILOT_BF16>(b, s);
        case PILOT_F16: return launch_build_dtype<PILOT_F16>(b, s);
        case PILOT_FP8E4M3: return launch_build_dtype<PILOT_FP8E4M3>(b, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t dispatch_build_fused(pilot_dtype dt, const FusedBuildParams& b, cudaStream_t s) {
    switch (dt) {
        case PILOT_F32: return launch_build_fused_dtype<PILOT_F32>(b, s);
        case PILOT_BF16: return launch_build_fused_dtype<PILOT_BF16>(b, s);
        case PILOT_F16: return launch_build_fused_dtype<PILOT_F16>(b, s);
        case PILOT_FP8E4M3: return launch_build_fused_dtype<PILOT_FP8E4M3>(b, s);
    }
    return cudaErrorInvalidValue;
}

// One build launch, plain (ep == nullptr) or with the FP64 step fused in.
pilot_status run_build(pilot_align_handle* h, pilot_dtype dt, const BuildParams& b, cudaStream_t s,
                       const EpilogueParams* ep = nullptr, int slot_offset = 0) {
    const bool prof = h->cfg.profile != 0;
    size_t k = 2 * (size_t)h->build_launches;
    if (prof) {
        while (h->events.size() < k + 2) {
            cudaEvent_t e;
            PILOT_CUDA(cudaEventCreate(&e), "event create");
            h->events.push_back(e);
        }
        PILOT_CUDA(cudaEventRecord(h->events[k], s), "event record");
    }
    if (ep) {
        FusedBuildParams fb{b, *ep, h->tickets + slot_offset, h->min_valid};
        PILOT_CUDA(dispatch_build_fused(dt, fb, s), "fused build-pass launch");
    } else {
        PILOT_CUDA(dispatch_build(dt, b, s), "build-pass launch");
    }
    if (prof) PILOT_CUDA(cudaEventRecord(h->events[k + 1], s), "event record");
    ++h->build_launches;
    ++h->total_launches;
    return PILOT_OK;
}

long long schedule_key(int batched, pilot_dtype dt, int C, double mean_n, double mean_m) {
    const int nb = (int)floor(log2(mean_n > 1.0 ? mean_n : 1.0));
    const int mb = (int)floor(log2(mean_m > 1.0 ? mean_m : 1.0));
    return ((long long)batched << 40) | ((long long)dt << 32) | ((long long)C << 16) | ((long long)nb << 8) |
           (long long)mb;
}

long long frames_key(const pilot_frame* frames, int n, int batched) {
    double sn = 0, sm = 0;
    for (int i = 0; i < n; ++i) {
        sn += frames[i].N;
        sm += frames[i].M;
    }
    return schedule_key(batched, frames[0].feat_dtype, frames[0].C, sn / n, sm / n);
}

pilot_schedule default_schedule() { return pilot_schedule{kTile, 0, 0, 0}; }

pilot_schedule schedule_for(const pilot_align_handle* h, const pilot_frame* frames, int n, int batched) {
    if (h->forcing) return h->forced;
    auto it = h->tuned.find(frames_key(frames, n, batched));
    return it != h->tuned.end() ? it->second : default_schedule();
}

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

void release(pilot_align_handle* h) {
    if (!h) return;
    cudaFree(h->state);
    cudaFree(h->pose32);
    cudaFree(h->partial);
    cudaFree(h->active[0]);
    cudaFree(h->active[1]);
    cudaFree(h->Tin);
    cudaFree(h->eval_out);
    cudaFree(h->min_valid);
    cudaFree(h->tickets);
    cudaFree(h->ones);
    cudaFree(h->res_dev);
    if (h->res_host) cudaFreeHost(h->res_host);
    for (auto& b : h->stage)
        if (b.ptr) cudaFree(b.ptr);
    for (auto e : h->events) cudaEventDestroy(e);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->graph) cudaGraphDestroy(h->graph);
    cudaFree(h->bdesc_dev);
    if (h->bdesc_host) cudaFreeHost(h->bdesc_host);
    cudaFree(h->bres_dev);
    if (h->bres_host) cudaFreeHost(h->bres_host);
    cudaFree(h->bactive);
    cudaFree(h->bmin_valid);
    cudaFree(h->bsync);
    cudaFree(h->bjob_meta);
    cudaFree(h->bflags);
    if (h->bstream) cudaStreamDestroy(h->bstream);
    for (int i = 0; i < kMaxStreams - 1; ++i) {
        if (h->pstream[i]) cudaStreamDestroy(h->pstream[i]);
        if (h->pjoin[i]) cudaEventDestroy(h->pjoin[i]);
    }
    if (h->pfork) cudaEventDestroy(h->pfork);
    if (h->cstream) cudaStreamDestroy(h->cstream);
    for (int i = 0; i < PILOT_MAX_LEVELS; ++i)
        if (h->level_ready[i]) cudaEventDestroy(h->level_ready[i]);
    delete h;
}

}  // namespace

namespace pilot {
void record_error(const char* msg) { g_last_error = msg; }
const char* last_error_message() { return g_last_error.c_str(); }
pilot_align_config config_with_defaults(const pilot_align_config& c) { return with_defaults(c); }
pilot_status check_config(const pilot_align_config& c) { return validate_config(c); }
pilot_status check_frame(const pilot_align_config& c, const pilot_frame* f) { return validate_frame(c, f); }
size_t dtype_bytes(pilot_dtype dt) { return dtype_size(dt); }
int frame_variant(const pilot_frame* f) {
    int v = 0;
    for (int l = 0; l < f->L; ++l) {
        const bool sl = f->qry_scale[l] || f->ref_scale[l];
        const int vl = (sl ? kVariantScaled : 0) | (f->qry_conf[l] ? kVariantConf : 0);
        if (sl && (!f->qry_scale[l] || !f->ref_scale[l])) return -1;
        if (l == 0) v = vl;
        if ((vl ^ v) & kVariantScaled) return -1;
        if ((vl ^ v) & kVariantConf) return -2;
    }
    return v;
}
PriorParams frame_prior(const pilot_align_config& c, const pilot_frame* f, const float* dsm_dev) {
    DevFrame d;
    d.dsm = f->use_range ? dsm_dev : nullptr;
    return prior_params(c, f, d);
}
}  // namespace pilot

namespace {

// Layout of the batch descriptor block (device copy and pinned host staging).
struct BatchLayout {
    size_t off_hdr, off_frames, off_nactive, off_fr_list, off_fr_item, off_fr_job, bytes;
    int max_frames, max_jobs;
    static BatchLayout make(int max_frames, int max_hyps) {
        auto a256 = [](size_t b) { return (b + 255) / 256 * 256; };
        BatchLayout l;
        l.max_frames = max_frames;
        l.max_jobs = max_hyps;
        l.off_hdr = 0;
        l.off_frames = a256(sizeof(BatchHeader));
        l.off_nactive = a256(l.off_frames + sizeof(FrameDesc) * (size_t)max_frames);
        l.off_fr_list = a256(l.off_nactive + sizeof(int) * PILOT_MAX_LEVELS * (size_t)max_frames);
        l.off_fr_item = a256(l.off_fr_list + sizeof(int) * PILOT_MAX_LEVELS * (size_t)max_frames);
        l.off_fr_job = a256(l.off_fr_item + sizeof(int) * PILOT_MAX_LEVELS * (size_t)(max_frames + 1));
        l.bytes = a256(l.off_fr_job + sizeof(int) * PILOT_MAX_LEVELS * (size_t)(max_frames + 1));
        return l;
    }
};

pilot_status batch_alloc(pilot_align_handle* h) {
    if (h->bdesc_dev) return PILOT_OK;
    const pilot_align_config& c = h->cfg;
    const BatchLayout lay = BatchLayout::make(c.max_frames, c.max_hyps);
    h->bdesc_bytes = lay.bytes;
    // result block, then the best index per frame, then the barrier error word
    h->bres_bytes = ResultLayout::make(c.max_hyps).bytes + sizeof(int) * ((size_t)c.max_frames + 1);
    PILOT_CUDA(cudaMalloc((void**)&h->bdesc_dev, h->bdesc_bytes), "batch descriptor allocation");
    PILOT_CUDA(cudaMallocHost((void**)&h->bdesc_host, h->bdesc_bytes), "batch descriptor staging");
    PILOT_CUDA(cudaMalloc((void**)&h->bres_dev, h->bres_bytes), "batch result allocation");
    PILOT_CUDA(cudaMallocHost((void**)&h->bres_host, h->bres_bytes), "batch result staging");
    PILOT_CUDA(cudaMalloc((void**)&h->bactive, sizeof(int) * (size_t)c.max_hyps), "batch active lists");
    PILOT_CUDA(cudaMalloc((void**)&h->bmin_valid, sizeof(double) * (size_t)c.max_frames), "batch thresholds");
    PILOT_CUDA(cudaMalloc((void**)&h->bsync, sizeof(unsigned long long) * kSyncWords * PILOT_MAX_LEVELS),
               "batch level counters");
    PILOT_CUDA(cudaMalloc((void**)&h->bjob_meta, sizeof(unsigned) * (size_t)c.max_hyps), "batch job table");
    h->bflag_words = level_flag_words(c.max_hyps, c.max_frames, h->max_tiles);
    PILOT_CUDA(cudaMalloc((void**)&h->bflags, sizeof(unsigned) * 2 * h->bflag_words), "batch job tile flags");
    PILOT_CUDA(cudaStreamCreateWithFlags(&h->bstream, cudaStreamNonBlocking), "batch stream");
    return PILOT_OK;
}

cudaError_t launch_level(pilot_dtype dt, int C, int variant, const LevelArgs& a, int grid, cudaStream_t s) {
    switch (dt) {
        case PILOT_F32: return launch_level_persistent_dtype<PILOT_F32>(C, variant, a, grid, s);
        case PILOT_BF16: return launch_level_persistent_dtype<PILOT_BF16>(C, variant, a, grid, s);
        case PILOT_F16: return launch_level_persistent_dtype<PILOT_F16>(C, variant, a, grid, s);
        case PILOT_FP8E4M3: return launch_level_persistent_dtype<PILOT_FP8E4M3>(C, variant, a, grid, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t level_occupancy(pilot_dtype dt, int C, int variant, int* n) {
    switch (dt) {
        case PILOT_F32: return level_persistent_occupancy<PILOT_F32>(C, variant, n);
        case PILOT_BF16: return level_persistent_occupancy<PILOT_BF16>(C, variant, n);
        case PILOT_F16: return level_persistent_occupancy<PILOT_F16>(C, variant, n);
        case PILOT_FP8E4M3: return level_persistent_occupancy<PILOT_FP8E4M3>(C, variant, n);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

namespace pilot {
cudaError_t level_launch(pilot_dtype dt, int C, int variant, const LevelArgs& a, int grid, cudaStream_t s) {
    return launch_level(dt, C, variant, a, grid, s);
}
cudaError_t level_occupancy_query(pilot_dtype dt, int C, int variant, int* n) {
    return level_occupancy(dt, C, variant, n);
}
}  // namespace pilot

namespace {

// flow_mask bit l: level l runs the level kernel's schedule without grid barriers; selftest:
// the graph of the flag self-test
long long graph_key(pilot_dtype dt, int C, int variant, int L, const pilot_schedule& sc, int flow_mask,
                    bool selftest) {
    return ((long long)selftest << 62) | ((long long)dt << 44) | ((long long)C << 36) | ((long long)variant << 32) |
           ((long long)L << 28) | ((long long)flow_mask << 22) | ((long long)sc.tile << 8) | (long long)sc.ctas_per_sm;
}

// Records the whole batched solve on h->bstream: descriptor upload, per-frame set-up,
// one persistent launch per level (+ per-frame top-K), selection, result download.
pilot_status capture_batch_graph(pilot_align_handle* h, pilot_dtype dt, int C, int variant, int L,
                                 const pilot_schedule& sc, int flow_mask) {
    const pilot_align_config& c = h->cfg;
    const BatchLayout lay = BatchLayout::make(c.max_frames, c.max_hyps);
    int dev = 0, sms = 0, per_sm = 0;
    PILOT_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    PILOT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    PILOT_CUDA(level_occupancy(dt, C, variant, &per_sm), "occupancy query");
    if (per_sm < 1) per_sm = 1;
    if (sc.ctas_per_sm > 0 && sc.ctas_per_sm < per_sm) per_sm = sc.ctas_per_sm;
    h->level_grid = sms * per_sm;
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->gexec = nullptr;
    h->graph = nullptr;
    cudaStream_t s = h->bstream;
    const BatchHeader* hdr = reinterpret_cast<const BatchHeader*>(h->bdesc_dev + lay.off_hdr);
    const FrameDesc* frames = reinterpret_cast<const FrameDesc*>(h->bdesc_dev + lay.off_frames);
    const int* nactive = reinterpret_cast<const int*>(h->bdesc_dev + lay.off_nactive);
    const int* fr_list = reinterpret_cast<const int*>(h->bdesc_dev + lay.off_fr_list);
    const int* fr_item = reinterpret_cast<const int*>(h->bdesc_dev + lay.off_fr_item);
    const int* fr_job = reinterpret_cast<const int*>(h->bdesc_dev + lay.off_fr_job);
    unsigned* error = reinterpret_cast<unsigned*>(h->bres_dev + ResultLayout::make(c.max_hyps).bytes +
                                                  sizeof(int) * (size_t)c.max_frames);
    PILOT_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "graph capture begin");
    cudaError_t e = cudaMemcpyAsync(h->bdesc_dev, h->bdesc_host, h->bdesc_bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(h->bsync, 0, sizeof(unsigned long long) * kSyncWords * PILOT_MAX_LEVELS, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(error, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) e = launch_batch_init(hdr, frames, h->state, h->bactive, c.max_frames, s);
    if (e == cudaSuccess)
        e = launch_batch_count_valid(hdr, frames, c.min_valid_frac, h->bmin_valid, c.max_frames, s);
    for (int level = L - 1; level >= 0 && e == cudaSuccess; --level) {
        LevelArgs a{};
        a.header = hdr;
        a.frames = frames;
        a.fr_list = fr_list + (size_t)level * lay.max_frames;
        a.fr_item = fr_item + (size_t)level * (lay.max_frames + 1);
        a.fr_job = fr_job + (size_t)level * (lay.max_frames + 1);
        a.active = h->bactive;
        a.state = h->state;
        a.min_valid = h->bmin_valid;
        a.pose32 = h->pose32;
        a.job_meta = h->bjob_meta;
        a.partial = h->partial;
        a.sync = h->bsync + (size_t)level * kSyncWords;
        // gather-heavy levels: the schedule without grid barriers (its per-job-tile flags)
        const bool flow = (flow_mask >> level) & 1;
        a.tile_done = flow ? h->bflags : nullptr;
        a.tile_ready = flow ? h->bflags + h->bflag_words : nullptr;
        a.error = error;
        a.barrier_timeout_ns = kBarrierTimeoutNs;
        a.barrier_extra = 0;
        if (flow && h->flag_selftest_ms > 0) {
            // the flag self-test: every wait for a job tile's flag asks for one iteration more
            // than will ever be published, and gives up after the test's timeout
            a.barrier_extra = 1;
            a.barrier_timeout_ns = (unsigned long long)(h->flag_selftest_ms * 1e6);
        }
        a.level = level;
        a.list_index = level;
        for (int l = 0; l < PILOT_MAX_LEVELS; ++l) a.iters[l] = c.iters_per_level[l];
        a.k_max = c.iters_per_level[level];
        a.tile = sc.tile;
        a.tiles_per_item = tiles_per_item(sc.tile);
        a.damping_mode = c.damping_mode;
        a.huber = (float)c.huber_photo;
        a.lambda0 = c.lambda0;
        if (flow) e = cudaMemsetAsync(h->bflags, 0, sizeof(unsigned) * 2 * h->bflag_words, s);
        if (e == cudaSuccess) e = launch_level(dt, C, variant, a, h->level_grid, s);
        const int K = c.keep_top_k[level];
        if (e == cudaSuccess && level > 0 && K > 0)
            e = launch_batch_prune(hdr, frames, h->state, h->bactive, nactive + (size_t)level * lay.max_frames, K,
                                   h->bmin_valid, c.max_frames, std::min(c.max_hyps, kMaxFrameHyps), s);
    }
    if (e == cudaSuccess)
        e = launch_batch_finalize(hdr, frames, h->state, h->bmin_valid, h->bres_dev, c.max_hyps, c.max_frames, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->bres_host, h->bres_dev, h->bres_bytes, cudaMemcpyDeviceToHost, s);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(s, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(e, "batch graph capture");
    }
    if (e2 != cudaSuccess) return cuda_fail(e2, "graph capture end");
    h->graph = g;
    PILOT_CUDA(cudaGraphInstantiate(&h->gexec, g, 0), "graph instantiate");
    h->graph_key = graph_key(dt, C, variant, L, sc, flow_mask, h->flag_selftest_ms > 0);
    return PILOT_OK;
}

}  // namespace

extern "C" {

const char* pilot_align_last_error(void) { return g_last_error.c_str(); }

pilot_status pilot_align_validate(const pilot_align_config* cfg_in, const pilot_frame* frame) {
    if (!cfg_in) return fail(PILOT_EINVAL, "config is NULL");
    const pilot_align_config cfg = with_defaults(*cfg_in);
    pilot_status st = validate_config(cfg);
    if (st != PILOT_OK) return st;
    return validate_frame(cfg, frame);
}

pilot_status pilot_align_create(const pilot_align_config* cfg_in, pilot_align_handle** out) {
    if (!cfg_in || !out) return fail(PILOT_EINVAL, "config or out is NULL");
    *out = nullptr;
    const pilot_align_config cfg = with_defaults(*cfg_in);
    pilot_status st = validate_config(cfg);
    if (st != PILOT_OK) return st;
    pilot_align_handle* h = new pilot_align_handle();
    h->cfg = cfg;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(e, "cudaGetDevice");
    }
    const size_t M = (size_t)cfg.max_hyps;
    h->max_tiles = cfg.max_points > 0 ? (cfg.max_points + kMinTile - 1) / kMinTile : 1;
    const ResultLayout lay = ResultLayout::make(cfg.max_hyps);
    std::vector<float> ones(cfg.max_channels, 1.0f);
#define ALLOC(ptr, bytes)                                      \
    if ((e = cudaMalloc((void**)&(ptr), (bytes))) != cudaSuccess) { \
        release(h);                                            \
        return cuda_fail(e, "workspace allocation");           \
    }
    ALLOC(h->state, sizeof(HypState) * M);
    ALLOC(h->pose32, sizeof(float) * 12 * M);
    // tile records: plain form [slot][tile]; batched form [(tile_item * tiles_per_item + tile)
    // * kHypTile + h], which rounds each job tile's anchor tiles up to whole work items and a
    // frame's jobs up to whole job tiles
    ALLOC(h->partial, sizeof(float) * kAcc * (M + (size_t)(kHypTile - 1) * cfg.max_frames) *
                          ((size_t)h->max_tiles + kItemAnchors / kMinTile));
    ALLOC(h->active[0], sizeof(int) * M);
    ALLOC(h->active[1], sizeof(int) * M);
    ALLOC(h->Tin, sizeof(double) * 12 * M);
    ALLOC(h->eval_out, sizeof(double) * kNumSums * M);
    ALLOC(h->min_valid, sizeof(double));
    ALLOC(h->tickets, sizeof(unsigned) * M);
    ALLOC(h->ones, sizeof(float) * cfg.max_channels);
    ALLOC(h->res_dev, lay.bytes);
#undef ALLOC
    if ((e = cudaMallocHost((void**)&h->res_host, lay.bytes)) != cudaSuccess) {
        release(h);
        return cuda_fail(e, "pinned result buffer");
    }
    if ((e = cudaMemcpy(h->ones, ones.data(), sizeof(float) * cfg.max_channels, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(h->tickets, 0, sizeof(unsigned) * M)) != cudaSuccess) {
        release(h);
        return cuda_fail(e, "workspace init");
    }
    *out = h;
    return PILOT_OK;
}

void pilot_align_destroy(pilot_align_handle* h) {
    if (!h) return;
    DeviceGuard g(h->device);
    cudaDeviceSynchronize();
    release(h);
}

pilot_status pilot_align_solve(pilot_align_handle* h, const pilot_frame* f, pilot_result* res,
                               void* stream) {
    if (!h || !res) return fail(PILOT_EINVAL, "handle or result is NULL");
    pilot_status st = validate_frame(h->cfg, f);
    if (st != PILOT_OK) return st;
    h->build_launches = 0;
    h->total_launches = 0;
    h->build_ms = 0.0;
    long long hyp_iters = 0;
    if (f->M == 0) {
        if (res->best) *res->best = -1;
        if (res->hyp_iters) *res->hyp_iters = 0;
        return PILOT_OK;
    }
    DeviceGuard guard(h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const pilot_align_config& c = h->cfg;
    DevFrame d;
    const bool overlap = !f->is_device && f->L > 1;     // finer levels copied while coarse ones solve
    if (overlap && !h->cstream) {
        PILOT_CUDA(cudaStreamCreateWithFlags(&h->cstream, cudaStreamNonBlocking), "copy stream");
        for (int i = 0; i < PILOT_MAX_LEVELS; ++i)
            PILOT_CUDA(cudaEventCreateWithFlags(&h->level_ready[i], cudaEventDisableTiming), "level event");
    }
    if ((st = bind_frame(h, f, s, &d, true, overlap ? h->cstream : nullptr, h->level_ready)) != PILOT_OK) return st;
    const int M = f->M;

    PILOT_CUDA(cudaMemsetAsync(h->tickets, 0, sizeof(unsigned) * M, s), "ticket reset");
    PILOT_CUDA(launch_count_valid(d.valid, f->N, c.min_valid_frac, h->min_valid, s), "count_valid launch");
    PILOT_CUDA(launch_hyp_init(h->state, d.T, h->active[0], M, s), "hyp_init launch");
    h->total_launches += 2;
    int cur = 0, n_active = M;
    const PriorParams prior = prior_params(c, f, d);

    const pilot_schedule sched = schedule_for(h, f, 1, 0);
    const int tile = sched.tile;
    const int n_streams = sched.streams > 0 ? sched.streams : kDefaultStreams;
    if (n_streams > 1 && !h->pfork) {
        PILOT_CUDA(cudaEventCreateWithFlags(&h->pfork, cudaEventDisableTiming), "fork event");
        for (int i = 0; i < kMaxStreams - 1; ++i) {
            PILOT_CUDA(cudaStreamCreateWithFlags(&h->pstream[i], cudaStreamNonBlocking), "extra stream");
            PILOT_CUDA(cudaEventCreateWithFlags(&h->pjoin[i], cudaEventDisableTiming), "join event");
        }
    }
    for (int level = f->L - 1; level >= 0; --level) {
        const int iters = c.iters_per_level[level];
        BuildParams b = build_params(h, f, d, level, n_active, h->active[cur], tile);
        EpilogueParams ep{};
        ep.state = h->state;
        ep.pose32 = h->pose32;
        ep.partial = h->partial;
        ep.active_idx = h->active[cur];
        ep.n_active = n_active;
        ep.n_tiles = b.n_tiles;
        ep.lambda0 = c.lambda0;
        ep.damping_mode = c.damping_mode;
        ep.prior = prior;
        if (overlap && level < f->L - 1) PILOT_CUDA(cudaStreamWaitEvent(s, h->level_ready[level], 0), "level copy wait");
        PILOT_CUDA(launch_level_init(h->state, h->pose32, h->active[cur], n_active, c.lambda0, s), "level_init launch");
        ++h->total_launches;
        // parts of the active list, part p = slots [off[p], off[p + 1]) on stream p (s for
        // p = 0), each with its own slice of the partial records and tickets
        const int parts = n_streams < n_active ? n_streams : n_active;
        int off[kMaxStreams + 1];
        BuildParams bp[kMaxStreams];
        EpilogueParams epp[kMaxStreams];
        cudaStream_t sp[kMaxStreams];
        for (int p = 0; p <= parts; ++p) off[p] = (int)(((long long)n_active * p) / parts);
        for (int p = 0; p < parts; ++p) {
            bp[p] = b;
            epp[p] = ep;
            bp[p].n_active = epp[p].n_active = off[p + 1] - off[p];
            bp[p].active_idx = epp[p].active_idx = b.active_idx + off[p];
            bp[p].partial = b.partial + (size_t)off[p] * b.n_tiles * kAcc;
            epp[p].partial = bp[p].partial;
            sp[p] = p ? h->pstream[p - 1] : s;
        }
        if (parts > 1) {
            PILOT_CUDA(cudaEventRecord(h->pfork, s), "fork record");
            for (int p = 1; p < parts; ++p) PILOT_CUDA(cudaStreamWaitEvent(sp[p], h->pfork, 0), "fork wait");
        }
        for (int k = 0; k <= iters; ++k) {
            for (int p = 0; p < parts; ++p) {
                epp[p].mode = (k == 0) ? kEpiInit : kEpiStep;
                epp[p].solve_next = k < iters;
                if ((st = run_build(h, f->feat_dtype, bp[p], sp[p], &epp[p], off[p])) != PILOT_OK) return st;
            }
        }
        for (int p = 1; p < parts; ++p) {
            PILOT_CUDA(cudaEventRecord(h->pjoin[p - 1], sp[p]), "join record");
            PILOT_CUDA(cudaStreamWaitEvent(s, h->pjoin[p - 1], 0), "join wait");
        }
        hyp_iters += (long long)n_active * iters;
        const int K = c.keep_top_k[level];
        if (level > 0 && K > 0 && K < n_active) {
            PILOT_CUDA(launch_prune(h->state, h->active[cur], h->active[cur ^ 1], n_active, K, h->min_valid, s),
                       "prune launch");
            ++h->total_launches;
            cur ^= 1;
            n_active = K;
        }
    }
    const ResultLayout lay = ResultLayout::make(M);
    PILOT_CUDA(launch_finalize(h->state, M, h->min_valid, h->res_dev, lay, s), "finalize launch");
    ++h->total_launches;
    PILOT_CUDA(cudaMemcpyAsync(h->res_host, h->res_dev, lay.bytes, cudaMemcpyDeviceToHost, s), "result copy");
    PILOT_CUDA(cudaStreamSynchronize(s), "solve");
    if (c.profile) {
        double total = 0.0;
        for (int i = 0; i < h->build_launches; ++i) {
            float ms = 0.f;
            PILOT_CUDA(cudaEventElapsedTime(&ms, h->events[2 * i], h->events[2 * i + 1]), "event timing");
            total += ms;
        }
        h->build_ms = total;
    }
    const unsigned char* r = h->res_host;
    if (res->T_cw) memcpy(res->T_cw, r + lay.off_T, sizeof(double) * 12 * M);
    if (res->cost) memcpy(res->cost, r + lay.off_cost, sizeof(double) * M);
    if (res->n_valid) memcpy(res->n_valid, r + lay.off_nvalid, sizeof(int) * M);
    if (res->hyp_status) memcpy(res->hyp_status, r + lay.off_status, sizeof(int) * M);
    if (res->best) memcpy(res->best, r + lay.off_best, sizeof(int));
    if (res->hyp_iters) *res->hyp_iters = hyp_iters;
    return PILOT_OK;
}

pilot_status pilot_align_debug_normal_eq(pilot_align_handle* h, const pilot_frame* f, int level,
                                         const double* T_cw, double* out29, void* stream) {
    if (!h || !out29 || !T_cw) return fail(PILOT_EINVAL, "handle, T_cw or out29 is NULL");
    pilot_status st = validate_frame(h->cfg, f);
    if (st != PILOT_OK) return st;
    if (level < 0 || level >= f->L) return fail(PILOT_EINVAL, "level %d outside [0, %d)", level, f->L);
    const int M = f->M;
    if (M == 0) return PILOT_OK;
    DeviceGuard guard(h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    h->build_launches = 0;
    h->total_launches = 0;
    DevFrame d;
    if ((st = bind_frame(h, f, s, &d, false)) != PILOT_OK) return st;
    PILOT_CUDA(cudaMemcpyAsync(h->Tin, T_cw, sizeof(double) * 12 * M, cudaMemcpyHostToDevice, s), "pose copy");
    PILOT_CUDA(launch_set_poses(h->state, h->pose32, h->Tin, h->active[0], M, s), "set_poses launch");
    BuildParams b = build_params(h, f, d, level, M, h->active[0]);
    if ((st = run_build(h, f->feat_dtype, b, s)) != PILOT_OK) return st;
    EpilogueParams ep{};
    ep.state = h->state;
    ep.pose32 = h->pose32;
    ep.partial = h->partial;
    ep.active_idx = h->active[0];
    ep.n_active = M;
    ep.n_tiles = b.n_tiles;
    ep.mode = kEpiEval;
    ep.prior = prior_params(h->cfg, f, d);
    ep.eval_out = h->eval_out;
    PILOT_CUDA(launch_epilogue(ep, h->min_valid, s), "epilogue launch");
    h->total_launches += 2;
    PILOT_CUDA(cudaMemcpyAsync(out29, h->eval_out, sizeof(double) * kNumSums * M, cudaMemcpyDeviceToHost, s),
               "normal-equation copy");
    PILOT_CUDA(cudaStreamSynchronize(s), "debug_normal_eq");
    return PILOT_OK;
}

pilot_status pilot_align_selftest_barrier_timeout(pilot_align_handle* h, double timeout_ms, double* elapsed_ms,
                                                  void* stream) {
    if (!h) return fail(PILOT_EINVAL, "handle is NULL");
    if (!(timeout_ms >= 1.0 && timeout_ms <= 10000.0)) return fail(PILOT_EINVAL, "timeout_ms must be in [1, 10000]");
    DeviceGuard guard(h->device);
    pilot_status st;
    if ((st = batch_alloc(h)) != PILOT_OK) return st;
    const pilot_align_config& c = h->cfg;
    const BatchLayout lay = BatchLayout::make(c.max_frames, c.max_hyps);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0, per_sm = 0;
    PILOT_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    PILOT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    PILOT_CUDA(level_occupancy(PILOT_F32, 32, false, &per_sm), "occupancy query");
    unsigned* error = reinterpret_cast<unsigned*>(h->bres_dev + ResultLayout::make(c.max_hyps).bytes +
                                                  sizeof(int) * (size_t)c.max_frames);
    // an empty frame list: the kernel's level-start pass has no jobs, and its first barrier
    // waits for one CTA more than the grid holds
    PILOT_CUDA(cudaMemsetAsync(h->bdesc_dev, 0, h->bdesc_bytes, s), "descriptor reset");
    PILOT_CUDA(cudaMemsetAsync(h->bsync, 0, sizeof(unsigned long long) * kSyncWords, s), "counter reset");
    PILOT_CUDA(cudaMemsetAsync(error, 0, sizeof(unsigned), s), "error reset");
    LevelArgs a{};
    a.header = reinterpret_cast<const BatchHeader*>(h->bdesc_dev + lay.off_hdr);
    a.frames = reinterpret_cast<const FrameDesc*>(h->bdesc_dev + lay.off_frames);
    a.fr_list = reinterpret_cast<const int*>(h->bdesc_dev + lay.off_fr_list);
    a.fr_item = reinterpret_cast<const int*>(h->bdesc_dev + lay.off_fr_item);
    a.fr_job = reinterpret_cast<const int*>(h->bdesc_dev + lay.off_fr_job);
    a.active = h->bactive;
    a.state = h->state;
    a.min_valid = h->bmin_valid;
    a.pose32 = h->pose32;
    a.job_meta = h->bjob_meta;
    a.partial = h->partial;
    a.sync = h->bsync;
    a.error = error;
    a.barrier_timeout_ns = (unsigned long long)(timeout_ms * 1e6);
    a.barrier_extra = 1;
    a.level = 0;
    a.list_index = 0;
    a.k_max = 0;
    a.tile = kTile;
    a.tiles_per_item = tiles_per_item(kTile);
    cudaEvent_t e0, e1;
    PILOT_CUDA(cudaEventCreate(&e0), "event create");
    PILOT_CUDA(cudaEventCreate(&e1), "event create");
    cudaError_t e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = launch_level(PILOT_F32, 32, false, a, sms * (per_sm > 0 ? per_sm : 1), s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    unsigned flag = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, error, sizeof flag, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "barrier self-test");
    if (elapsed_ms) *elapsed_ms = ms;
    if (flag != 1u) return fail(PILOT_ECUDA, "barrier self-test: the impossible barrier did not report its timeout");
    return PILOT_OK;
}

pilot_status pilot_align_selftest_flag_timeout(pilot_align_handle* h, const pilot_frame* frames, int n,
                                               double timeout_ms, double* elapsed_ms, void* stream) {
    if (!h || !frames || n < 1) return fail(PILOT_EINVAL, "handle or frames missing");
    if (!(timeout_ms >= 1.0 && timeout_ms <= 10000.0)) return fail(PILOT_EINVAL, "timeout_ms must be in [1, 10000]");
    if (n > h->cfg.max_frames) return fail(PILOT_EINVAL, "more frames than max_frames");
    // results are discarded: one scratch record per hypothesis
    long long total = 0;
    for (int i = 0; i < n; ++i) total += frames[i].M > 0 ? frames[i].M : 0;
    std::vector<double> T(12 * (size_t)total + 12), cost((size_t)total + 1);
    std::vector<int> nv((size_t)total + 1), hs((size_t)total + 1), best(n);
    std::vector<long long> hi(n);
    std::vector<pilot_result> res(n);
    size_t o = 0;
    for (int i = 0; i < n; ++i) {
        res[i] = pilot_result{T.data() + 12 * o, cost.data() + o, nv.data() + o, hs.data() + o, &best[i], &hi[i]};
        o += frames[i].M > 0 ? frames[i].M : 0;
    }
    h->flag_selftest_ms = timeout_ms;
    const auto t0 = std::chrono::steady_clock::now();
    const pilot_status st = pilot_align_solve_batch(h, frames, n, res.data(), stream);
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    h->flag_selftest_ms = 0;
    if (elapsed_ms) *elapsed_ms = ms;
    if (st == PILOT_ETIMEOUT) return PILOT_OK;
    if (st != PILOT_OK) return st;
    return fail(PILOT_ECUDA, "flag self-test: the unpublishable flag did not report its timeout");
}

pilot_status pilot_align_solve_batch(pilot_align_handle* h, const pilot_frame* frames, int n,
                                     pilot_result* results, void* stream) {
    if (!h || (n > 0 && (!frames || !results))) return fail(PILOT_EINVAL, "handle, frames or results is NULL");
    const pilot_align_config& c = h->cfg;
    if (n < 0 || n > c.max_frames) return fail(PILOT_EINVAL, "n_frames = %d outside [0, max_frames = %d]", n, c.max_frames);
    if (n == 0) return PILOT_OK;
    pilot_status st;
    long long total = 0;
    const pilot_frame& f0 = frames[0];
    int variant = 0;
    for (int i = 0; i < n; ++i) {
        const pilot_frame* f = frames + i;
        if ((st = validate_frame(c, f)) != PILOT_OK) return fail(st, "frame %d: %s", i, g_last_error.c_str());
        if (!f->is_device) return fail(PILOT_EINVAL, "frame %d: the batched form needs device frames", i);
        if (f->C != f0.C || f->L != f0.L || f->feat_dtype != f0.feat_dtype)
            return fail(PILOT_EINVAL, "frame %d: C, L and feat_dtype must match frame 0", i);
        if (f->M > kMaxFrameHyps) return fail(PILOT_EINVAL, "frame %d: M = %d above %d", i, f->M, kMaxFrameHyps);
        const int vf = frame_variant(f);
        if (vf == -1) return fail(PILOT_EINVAL, "frame %d: give both scale arrays on every level, or none", i);
        if (vf == -2) return fail(PILOT_EINVAL, "frame %d: give a confidence map on every level, or none", i);
        if (i == 0) variant = vf;
        if (vf != variant)
            return fail(PILOT_EINVAL, "frame %d: scale and confidence presence must match frame 0", i);
        total += f->M;
    }
    if (total > c.max_hyps) return fail(PILOT_EINVAL, "batch has %lld hypotheses, above max_hyps = %d", total, c.max_hyps);
    DeviceGuard guard(h->device);
    if ((st = batch_alloc(h)) != PILOT_OK) return st;
    const BatchLayout lay = BatchLayout::make(c.max_frames, c.max_hyps);
    unsigned char* hb = h->bdesc_host;
    BatchHeader* hdr = reinterpret_cast<BatchHeader*>(hb + lay.off_hdr);
    FrameDesc* fds = reinterpret_cast<FrameDesc*>(hb + lay.off_frames);
    int* nactive = reinterpret_cast<int*>(hb + lay.off_nactive);
    int* fr_list = reinterpret_cast<int*>(hb + lay.off_fr_list);
    int* fr_item = reinterpret_cast<int*>(hb + lay.off_fr_item);
    int* fr_job = reinterpret_cast<int*>(hb + lay.off_fr_job);
    memset(hdr, 0, sizeof(BatchHeader));
    hdr->n_frames = n;
    hdr->total_hyps = (int)total;
    const int L = f0.L;
    int off = 0;
    for (int i = 0; i < n; ++i) {
        const pilot_frame* f = frames + i;
        FrameDesc& d = fds[i];
        memset(&d, 0, sizeof d);
        const size_t N = (size_t)f->N;
        d.px = f->points;
        d.py = f->points ? f->points + N : nullptr;
        d.pz = f->points ? f->points + 2 * N : nullptr;
        d.weight = f->point_weight;
        d.valid = f->point_valid;
        d.N = f->N;
        d.M = f->M;
        for (int l = 0; l < L; ++l) {
            d.ref[l] = f->ref_feat[l];
            d.qry[l] = f->qry_feat[l];
            d.rscale[l] = f->ref_scale[l];
            d.qscale[l] = f->qry_scale[l];
            d.conf[l] = f->qry_conf[l];
            d.H[l] = f->H[l];
            d.W[l] = f->W[l];
            const double sc = ldexp(1.0, -l);
            d.fx[l] = (float)(f->fx * sc);
            d.fy[l] = (float)(f->fy * sc);
            d.cx[l] = (float)(f->cx * sc);
            d.cy[l] = (float)(f->cy * sc);
        }
        d.T_cw = f->T_cw;
        d.hyp_offset = off;
        DevFrame dv;
        dv.dsm = f->use_range ? f->dsm : nullptr;
        d.prior = prior_params(c, f, dv);
        off += f->M;
    }
    // hypotheses per frame and level (top-K is deterministic in count), and each level's
    // frame list: frames with more anchors first (job_order 0) or in the caller's order (1);
    // jobs and work items are numbered frame after frame in list order
    const pilot_schedule sc = schedule_for(h, frames, n, 1);
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    if (sc.job_order == 0)
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return frames[a].N > frames[b].N; });
    const int tpi = tiles_per_item(sc.tile);
    std::vector<long long> hyp_iters(n, 0);
    std::vector<int> cur(n);
    int flow_mask = 0;     // levels that run without grid barriers
    for (int i = 0; i < n; ++i) cur[i] = frames[i].M;
    for (int level = L - 1; level >= 0; --level) {
        int* list = fr_list + (size_t)level * lay.max_frames;
        int* items = fr_item + (size_t)level * (lay.max_frames + 1);
        int* jobs = fr_job + (size_t)level * (lay.max_frames + 1);
        items[0] = jobs[0] = 0;
        for (int oi = 0; oi < n; ++oi) {
            const int i = order[oi];
            nactive[(size_t)level * lay.max_frames + i] = cur[i];
            list[oi] = i;
            jobs[oi + 1] = jobs[oi] + cur[i];
            items[oi + 1] = items[oi] + frame_items(cur[i], frames[i].N, sc.tile, tpi);
        }
        hdr->n_listed[level] = n;
        // the schedule without grid barriers for levels with much gather work per iteration, or
        // at least one work item of anchors per job on average (few steps per gather); the
        // lockstep schedule where the FP64 steps dominate (e.g. 500 anchors per job)
        long long units = 0, n_jobs = 0;   // anchor x hypothesis units and jobs of one iteration
        for (int i = 0; i < n; ++i) {
            units += (long long)frames[i].N * cur[i];
            n_jobs += cur[i];
        }
        if (units >= kSplitUnits || (n_jobs > 0 && units >= (long long)kItemAnchors * n_jobs))
            flow_mask |= 1 << level;
        for (int i = 0; i < n; ++i) {
            hyp_iters[i] += (long long)cur[i] * c.iters_per_level[level];
            const int K = c.keep_top_k[level];
            if (level > 0 && K > 0 && K < cur[i]) cur[i] = K;
        }
    }
    if (h->flag_selftest_ms > 0 && flow_mask == 0)
        return fail(PILOT_EINVAL, "flag self-test: no level of this batch runs without grid barriers");
    const long long key = graph_key(f0.feat_dtype, f0.C, variant, L, sc, flow_mask, h->flag_selftest_ms > 0);
    if (!h->gexec || h->graph_key != key)
        if ((st = capture_batch_graph(h, f0.feat_dtype, f0.C, variant, L, sc, flow_mask)) != PILOT_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PILOT_CUDA(cudaGraphLaunch(h->gexec, s), "batch graph launch");
    PILOT_CUDA(cudaStreamSynchronize(s), "batch solve");
    h->total_launches = 4 + 2 * L + 1;
    const ResultLayout rl = ResultLayout::make(c.max_hyps);
    const unsigned char* r = h->bres_host;
    const int* best = reinterpret_cast<const int*>(r + rl.bytes);
    if (best[c.max_frames] != 0)
        return fail(PILOT_ETIMEOUT, "batched solve: a level kernel's grid barrier or flag wait timed out (results invalid)");
    for (int i = 0; i < n; ++i) {
        const int o = fds[i].hyp_offset, M = frames[i].M;
        pilot_result& out = results[i];
        if (out.T_cw) memcpy(out.T_cw, r + rl.off_T + sizeof(double) * 12 * (size_t)o, sizeof(double) * 12 * M);
        if (out.cost) memcpy(out.cost, r + rl.off_cost + sizeof(double) * (size_t)o, sizeof(double) * M);
        if (out.n_valid) memcpy(out.n_valid, r + rl.off_nvalid + sizeof(int) * (size_t)o, sizeof(int) * M);
        if (out.hyp_status) memcpy(out.hyp_status, r + rl.off_status + sizeof(int) * (size_t)o, sizeof(int) * M);
        if (out.best) *out.best = best[i];
        if (out.hyp_iters) *out.hyp_iters = hyp_iters[i];
    }
    return PILOT_OK;
}

pilot_status pilot_align_autotune(pilot_align_handle* h, const pilot_frame* frames, int n, int batched,
                                  int reps, pilot_schedule* chosen, double* best_ms, void* stream) {
    if (!h || !frames || n < 1) return fail(PILOT_EINVAL, "handle or frames missing");
    if (batched && n > h->cfg.max_frames) return fail(PILOT_EINVAL, "more frames than max_frames");
    if (reps < 1) reps = 1;
    std::vector<pilot_schedule> cands;
    for (int tile : {512, 1024, 2048, 4096}) {
        if (!batched) {
            for (int streams : {1, 2}) cands.push_back(pilot_schedule{tile, 0, 0, streams});
            continue;
        }
        for (int per_sm : {1, 0})
            for (int order : {0, 1}) cands.push_back(pilot_schedule{tile, per_sm, order, 0});
    }
    // results are discarded: one scratch record per hypothesis
    long long total = 0;
    for (int i = 0; i < (batched ? n : 1); ++i) total += frames[i].M;
    std::vector<double> T(12 * (size_t)total), cost(total);
    std::vector<int> nv(total), hs(total), best(n);
    std::vector<long long> hi(n);
    std::vector<pilot_result> res(n);
    size_t o = 0;
    for (int i = 0; i < (batched ? n : 1); ++i) {
        res[i] = pilot_result{T.data() + 12 * o, cost.data() + o, nv.data() + o, hs.data() + o, &best[i], &hi[i]};
        o += frames[i].M;
    }
    DeviceGuard guard(h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    PILOT_CUDA(cudaEventCreate(&e0), "event create");
    PILOT_CUDA(cudaEventCreate(&e1), "event create");
    double best_t = 1e300;
    pilot_schedule win = default_schedule();
    pilot_status st = PILOT_OK;
    h->forcing = true;
    for (const pilot_schedule& sc : cands) {
        h->forced = sc;
        float total_ms = 0.f;
        for (int r = 0; r <= reps && st == PILOT_OK; ++r) {
            cudaEventRecord(e0, s);
            st = batched ? pilot_align_solve_batch(h, frames, n, res.data(), stream)
                         : pilot_align_solve(h, frames, res.data(), stream);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r > 0) total_ms += ms;          // the first run warms up (and captures the graph)
        }
        if (st != PILOT_OK) break;
        const double mean = total_ms / reps;
        if (mean < best_t) {
            best_t = mean;
            win = sc;
        }
    }
    h->forcing = false;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != PILOT_OK) return st;
    h->tuned[frames_key(frames, batched ? n : 1, batched)] = win;
    if (chosen) *chosen = win;
    if (best_ms) *best_ms = best_t;
    return PILOT_OK;
}

pilot_status pilot_align_set_schedule(pilot_align_handle* h, const pilot_frame* frames, int n, int batched,
                                      const pilot_schedule* sc) {
    if (!h || !frames || n < 1 || !sc) return fail(PILOT_EINVAL, "handle, frames or schedule missing");
    if (sc->tile != 512 && sc->tile != 1024 && sc->tile != 2048 && sc->tile != 4096)
        return fail(PILOT_EINVAL, "tile %d is not 512, 1024, 2048 or 4096", sc->tile);
    if (sc->ctas_per_sm < 0 || sc->ctas_per_sm > 2) return fail(PILOT_EINVAL, "ctas_per_sm %d outside [0, 2]", sc->ctas_per_sm);
    if (sc->job_order < 0 || sc->job_order > 1) return fail(PILOT_EINVAL, "job_order %d outside [0, 1]", sc->job_order);
    if (sc->streams < 0 || sc->streams > kMaxStreams)
        return fail(PILOT_EINVAL, "streams %d outside [0, %d]", sc->streams, kMaxStreams);
    h->tuned[frames_key(frames, batched ? n : 1, batched)] = *sc;
    return PILOT_OK;
}

pilot_status pilot_align_get_schedule(const pilot_align_handle* h, const pilot_frame* frames, int n,
                                      int batched, pilot_schedule* out) {
    if (!h || !frames || n < 1 || !out) return fail(PILOT_EINVAL, "handle, frames or out missing");
    *out = schedule_for(h, frames, batched ? n : 1, batched);
    return PILOT_OK;
}

pilot_status pilot_align_profile(const pilot_align_handle* h, double* build_ms, int* build_launches,
                                 int* total_launches) {
    if (!h) return fail(PILOT_EINVAL, "handle is NULL");
    if (build_ms) *build_ms = h->build_ms;
    if (build_launches) *build_launches = h->build_launches;
    if (total_launches) *total_launches = h->total_launches;
    return PILOT_OK;
}

}  // extern "C"
