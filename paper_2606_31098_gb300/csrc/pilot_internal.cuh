// Internal declarations shared by the CUDA library's translation units (not installed).
//
// Device data layout (one frame):
//   anchors      SoA FP32  x[N] y[N] z[N]            (coalesced per-anchor reads)
//   ref features N x C per level, storage dtype       (one contiguous row per anchor)
//   query maps   H x W x C per level (NHWC)           (one tap = C contiguous values)
//   hypotheses   HypState[M], FP64 LM state per hypothesis
//   candidates   pose32[M][12], FP32 [R | t] the build pass evaluates
//   partials     partial[slot][tile][32] FP32: 21 H + 6 g + cost + n_valid (+3 pad)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pilot_align.h"

namespace pilot {

constexpr int kAcc = 32;           // padded width of one partial-sum record
constexpr int kNumSums = 29;       // 21 H + 6 g + cost + n_valid
constexpr int kVariantScaled = 1;   // per-channel dequantisation scales given
constexpr int kVariantConf = 2;     // query confidence maps given
constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;   // level kernel: longest barrier wait
constexpr int kSyncWords = 4;      // per persistent level launch: claims, arrivals, generations, pad
constexpr int kItemAnchors = 4096; // persistent level kernel: anchors per work item (whole tiles)
constexpr int kMaxFrameHyps = 8192; // batched and served forms: hypotheses of one frame at most
constexpr int kSmemFrames = 512;   // persistent level kernel: frame tables staged in shared memory up to this
constexpr long long kSplitUnits = 8ll << 20;   // batched levels with at least this many anchor x hypothesis units per iteration (or kItemAnchors anchors per job) run without grid barriers

// Tiles per work item of the persistent level kernel for a reduction tile of `tile` anchors.
__host__ __device__ inline int tiles_per_item(int tile) { return tile >= kItemAnchors ? 1 : kItemAnchors / tile; }

// Work items per job of a frame of N anchors.
__host__ __device__ inline int items_per_job(int N, int tile, int tpi) {
    const int tiles = N > 0 ? (N + tile - 1) / tile : 1;
    return (tiles + tpi - 1) / tpi;
}

#ifndef PILOT_HYP_TILE
#define PILOT_HYP_TILE 4
#endif
// Hypotheses a build-pass CTA holds over one anchor tile (2, 4 or 8): the reference row of an
// anchor is read once for all of them.
constexpr int kHypTile = PILOT_HYP_TILE;
static_assert(kHypTile == 2 || kHypTile == 4 || kHypTile == 8, "hypothesis tile");

// Words of one of the level kernel's per-job-tile flag arrays (indexed by a job tile's first
// work item) for at most max_hyps jobs in max_frames frames of at most max_tiles anchor tiles.
inline size_t level_flag_words(int max_hyps, int max_frames, int max_tiles) {
    return ((size_t)max_hyps / kHypTile + (size_t)max_frames + 1) * ((size_t)max_tiles + 1);
}

// Work items of a frame of N anchors with n_jobs jobs: the jobs are taken kHypTile at a time
// (a work item covers all jobs of its tile, as a build-pass CTA holds kHypTile hypotheses).
__host__ __device__ inline int frame_items(int n_jobs, int N, int tile, int tpi) {
    return (n_jobs + kHypTile - 1) / kHypTile * items_per_job(N, tile, tpi);
}
constexpr int kBuildThreads = 256;
constexpr float kZNear = 0.1f;

// FP64 Levenberg-Marquardt state of one hypothesis.
struct HypState {
    double T[12];      // accepted pose [R | t], world -> camera
    double Tc[12];     // candidate pose awaiting evaluation
    double H[21];      // J^T W J at T (upper triangle, row-major)
    double g[6];       // J^T W r at T
    double cost;       // objective at T
    double lambda;     // LM damping
    int n_valid;       // visible anchors at T
    int has_cand;      // 1: Tc must be evaluated by the next build pass
    int last_fail;     // 1: the last damped solve was not positive definite
    int active;        // 0: pruned
    int status;        // pilot_hyp_status (final)
    int pad;
};

// Inputs of one build pass (one level of one frame).
struct BuildParams {
    const float* px;
    const float* py;
    const float* pz;
    const float* weight;       // N or nullptr
    const uint8_t* valid;      // N or nullptr
    const void* qry;           // H x W x C
    const void* ref;           // N x C
    const float* qscale;       // C or nullptr
    const float* rscale;       // C or nullptr
    const float* conf;         // H x W query confidence or nullptr
    int N, C, H, W;
    float fx, fy, cx, cy;      // level intrinsics
    float huber;               // photo Huber delta
    const float* pose32;       // [M][12]
    const int* active_idx;     // [n_active] hypothesis index of each slot
    const HypState* state;     // has_cand flags
    float* partial;            // [n_active][n_tiles][kAcc]
    int n_active;
    int n_tiles;
    int tile;                  // anchors per tile
};

// Prior terms (Eq. 3-6), FP64.
struct PriorParams {
    int use_gravity;
    double g_cam[3], g_world[3], w_grav, huber_grav;
    int use_range;
    double q[3];               // d^range * v (Eq. 4 ray scaled by the range), camera frame
    double w_range, huber_range;
    double gate_grav, gate_range;   // residual gates (0 = none)
    const float* dsm;
    int dsm_H, dsm_W;
    double dsm_x0, dsm_y0, dsm_gsd, dsm_inv_gsd;   // inv = 1 / gsd
};

enum EpilogueMode { kEpiInit = 0, kEpiStep = 1, kEpiEval = 2 };

struct EpilogueParams {
    HypState* state;
    float* pose32;
    const float* partial;
    const int* active_idx;
    int n_active, n_tiles;
    int mode;                  // EpilogueMode
    int solve_next;            // 1: compute the next candidate after this evaluation
    double lambda0;
    int damping_mode;
    PriorParams prior;
    double* eval_out;          // kEpiEval: [slot][29]
};

// A build pass whose last CTA per hypothesis tile runs the FP64 LM steps itself (the CTA
// that takes the last ticket of its tile sums the tile records and calls lm_step for each
// of its hypotheses).
struct FusedBuildParams {
    BuildParams b;
    EpilogueParams ep;
    unsigned* tickets;         // one per hypothesis tile of the launch, zero between launches
    const double* min_valid;
};

// ---- batched form: many frames, one persistent launch per pyramid level ----

// One frame of a batch, as the device kernels see it.
struct FrameDesc {
    const float* px;
    const float* py;
    const float* pz;
    const float* weight;
    const uint8_t* valid;
    const void* ref[PILOT_MAX_LEVELS];
    const void* qry[PILOT_MAX_LEVELS];
    const float* rscale[PILOT_MAX_LEVELS];
    const float* qscale[PILOT_MAX_LEVELS];
    const float* conf[PILOT_MAX_LEVELS];
    int N, M;
    int H[PILOT_MAX_LEVELS], W[PILOT_MAX_LEVELS];
    float fx[PILOT_MAX_LEVELS], fy[PILOT_MAX_LEVELS], cx[PILOT_MAX_LEVELS], cy[PILOT_MAX_LEVELS];
    const double* T_cw;        // M x 12 initial hypotheses
    int hyp_offset;            // first global hypothesis (state, active list, results)
    int level;                 // serving: the level this frame runs in the current round
    int n_active;              // serving: hypotheses still active at that level
    int flags;                 // serving: kFlagInit | kFlagPrune | kFlagFinalize
    int keep;                  // serving: top-K after this level (kFlagPrune)
    int quota;                 // serving: levels this frame may still run in the current round
    PriorParams prior;
};

enum FrameFlags { kFlagInit = 1, kFlagPrune = 2, kFlagFinalize = 4 };

// Batch header, rewritten before every batch (the captured graph reads it).
struct BatchHeader {
    int n_frames;
    int n_listed[PILOT_MAX_LEVELS];   // frames listed for each level's persistent launch
    int total_hyps;
    int tiles_per_item;               // > 0: work-item size of the launches over these tables; 0: LevelArgs'
};

// Persistent level kernel arguments.  A launch's jobs (one per active hypothesis of a listed
// frame) and work items are numbered frame after frame in list order: listed frame i is
// frames[fr_list[i]]; its jobs are fr_job[i] .. fr_job[i + 1] - 1 (its active slots in
// order) and its items fr_item[i] .. fr_item[i + 1] - 1, items_per_job(N) consecutive items
// per tile of kHypTile jobs (jobs kHypTile p .. kHypTile p + kHypTile - 1), each covering
// tiles_per_item anchor tiles of all of them.  Tile t of job kHypTile p + h, whose job tile's
// first item is q, keeps its record at partial[(q * tiles_per_item + t) * kHypTile + h].
struct LevelArgs {
    const BatchHeader* header;
    const FrameDesc* frames;
    const int* fr_list;
    const int* fr_item;
    const int* fr_job;
    const int* active;         // per frame: active[hyp_offset + slot] = local hypothesis
    HypState* state;           // global hypothesis index
    const double* min_valid;   // per frame
    float* pose32;             // [job][12] FP32 pose to evaluate next
    unsigned* job_meta;        // [job] hypothesis index | 0x80000000 when it has a pose to evaluate
    float* partial;            // tile records
    unsigned long long* sync;  // [0] item claims, [1] barrier arrivals, [2] barrier generations; zero before the launch
    unsigned* tile_done;       // per job tile, at its first item: items completed (all iterations); zero before the launch
    unsigned* tile_ready;      // per job tile, at its first item: iterations whose FP64 steps are published; zero before the launch
    unsigned* error;           // set to 1 when a barrier wait gives up
    unsigned long long barrier_timeout_ns;   // longest barrier wait
    int barrier_extra;         // 0; > 0 only in the failure self-tests: a grid barrier (lockstep) or a job tile's flag (barrier-free schedule) that cannot complete
    int level;                 // >= 0: every frame runs this level; -1: each its own level
    int list_index;            // which header->n_listed entry counts this launch's frames
    int iters[PILOT_MAX_LEVELS];
    int k_max;                 // iterations of the longest job of the launch
    int tile, tiles_per_item, damping_mode;
    float huber;
    double lambda0;
};

// Result block copied to the host in one transfer.
struct ResultLayout {
    size_t off_T, off_cost, off_nvalid, off_status, off_best, bytes;
    __host__ __device__ static ResultLayout make(int M) {
        ResultLayout r;
        r.off_T = 0;
        r.off_cost = r.off_T + sizeof(double) * 12 * (size_t)M;
        r.off_nvalid = r.off_cost + sizeof(double) * (size_t)M;
        r.off_status = r.off_nvalid + sizeof(int) * (size_t)M;
        r.off_best = r.off_status + sizeof(int) * (size_t)M;
        r.bytes = r.off_best + 16;
        return r;
    }
};

// ---- launchers (each returns the cudaError_t of its launch) ----
cudaError_t launch_epilogue(const EpilogueParams& p, const double* min_valid, cudaStream_t s);
cudaError_t launch_level_init(HypState* st, float* pose32, const int* active_idx, int n_active,
                              double lambda0, cudaStream_t s);
cudaError_t launch_hyp_init(HypState* st, const double* T_cw, int* active_idx, int M,
                            cudaStream_t s);
cudaError_t launch_set_poses(HypState* st, float* pose32, const double* T_cw, int* active_idx,
                             int M, cudaStream_t s);
cudaError_t launch_prune(HypState* st, const int* active_in, int* active_out, int n_active,
                         int keep, const double* min_valid, cudaStream_t s);
cudaError_t launch_count_valid(const uint8_t* valid, int N, double frac, double* min_valid,
                               cudaStream_t s);
cudaError_t launch_finalize(HypState* st, int M, const double* min_valid, unsigned char* result,
                            ResultLayout lay, cudaStream_t s);

template <pilot_dtype DT>
cudaError_t launch_build_dtype(const BuildParams& p, cudaStream_t s);
template <pilot_dtype DT>
cudaError_t launch_build_fused_dtype(const FusedBuildParams& p, cudaStream_t s);

template <pilot_dtype DT>
cudaError_t launch_level_persistent_dtype(int C, int variant, const LevelArgs& a, int grid,
                                          cudaStream_t s);
template <pilot_dtype DT>
cudaError_t level_persistent_occupancy(int C, int variant, int* ctas_per_sm);

// batch bookkeeping (one block per frame; frames beyond header->n_frames return)
cudaError_t launch_batch_init(const BatchHeader* hdr, const FrameDesc* frames, HypState* st,
                              int* active, int max_frames, cudaStream_t s);
cudaError_t launch_batch_count_valid(const BatchHeader* hdr, const FrameDesc* frames, double frac,
                                     double* min_valid, int max_frames, cudaStream_t s);
cudaError_t launch_batch_prune(const BatchHeader* hdr, const FrameDesc* frames, HypState* st,
                               int* active, const int* n_active, int keep, const double* min_valid,
                               int max_frames, int max_frame_hyps, cudaStream_t s);
cudaError_t launch_batch_finalize(const BatchHeader* hdr, const FrameDesc* frames, HypState* st,
                                  const double* min_valid, unsigned char* result, int max_hyps,
                                  int max_frames, cudaStream_t s);
// serving rounds: the same steps, each frame doing only what its flags ask for
struct LevelKeep {
    int k[PILOT_MAX_LEVELS];   // keep_top_k per level
};
cudaError_t launch_round_advance(const BatchHeader* hdr, FrameDesc* frames, const int* fr_list, int* fr_item,
                                 int* fr_job, const LevelKeep& keep, int tile, int tpi, cudaStream_t s);
cudaError_t launch_round_prepare(const BatchHeader* hdr, const FrameDesc* frames, HypState* st,
                                 int* active, double frac, double* min_valid, int max_frames,
                                 cudaStream_t s);
cudaError_t launch_round_finish(const BatchHeader* hdr, const FrameDesc* frames, HypState* st,
                                int* active, const double* min_valid, unsigned char* result,
                                int max_hyps, int max_frames, int max_frame_hyps, cudaStream_t s);

// Sets the message pilot_align_last_error() returns on the calling thread.
void record_error(const char* msg);
const char* last_error_message();

// host helpers shared by the runtime's translation units
pilot_align_config config_with_defaults(const pilot_align_config& c);
pilot_status check_config(const pilot_align_config& c);
pilot_status check_frame(const pilot_align_config& c, const pilot_frame* f);
size_t dtype_bytes(pilot_dtype dt);
PriorParams frame_prior(const pilot_align_config& c, const pilot_frame* f, const float* dsm_dev);
cudaError_t level_launch(pilot_dtype dt, int C, int variant, const LevelArgs& a, int grid, cudaStream_t s);
cudaError_t level_occupancy_query(pilot_dtype dt, int C, int variant, int* n);
// Kernel variant of a frame for the batched and served forms (every frame of one launch
// shares it): kVariantScaled when both scale arrays are given on every level,
// kVariantConf when a query confidence map is given on every level.  Returns -1 when
// the scales are given on some levels only (or one of a pair), -2 for the confidences.
int frame_variant(const pilot_frame* f);
constexpr int kPlainTile = 1024;

}  // namespace pilot
