/*
 * pilot_align.h -- C-ABI of the GB300 featuremetric multi-hypothesis LM pose solver.
 *
 * The solver estimates the world->camera pose of a query frame by aligning its feature
 * pyramid with 3D geo-anchors lifted from a TDOM/DSM crop (problem statement, Sec. IV).
 * For every anchor P_j and pose hypothesis T it projects P_j into the query pyramid,
 * bilinearly samples C channels, forms the photo residual (Eq. 1) under a Huber loss
 * (Eq. 2), adds the IMU gravity residual (Eq. 3) and the single-point laser range
 * residual (Eq. 4-6) to the total objective (Eq. 7), and takes damped Gauss-Newton
 * (Levenberg-Marquardt) steps (Eq. 8) with the left SE(3) update (Eq. 9), coarse to
 * fine over the pyramid, for many hypotheses at once (Sec. IV-E and Supp.
 * "Multi-Hypothesis Refinement"); the output is the hypothesis of lowest objective.
 *
 * Conventions shared by every entry point:
 *   - No C++ exception crosses this boundary.  Every call returns a pilot_status; the
 *     detail of the last failure on the calling thread is in pilot_align_last_error().
 *   - Inputs are never modified.  Output buffers belong to the caller.
 *   - A handle owns its device workspace (sized at create from the config's max_*
 *     fields); frames larger than that are rejected with PILOT_EINVAL.  A handle is not
 *     re-entrant: use one handle per host thread.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *     Every call that takes a stream, except pilot_align_normal_eq_noalloc (which only
 *     enqueues), has returned all results to host memory, and has finished using the
 *     caller's input buffers, when it returns.
 *   - Per-hypothesis failures (too few visible anchors, a singular damped system,
 *     non-finite values) are reported as per-hypothesis statuses, not as errors.
 *   - Readings where the paper is silent (documented at each field):
 *       pose state T_cw = [R | t] world->camera, row-major 3x4, FP64; the LM update is
 *       T <- exp(dxi) T with dxi = (nu, omega), translation first;
 *       pixel i covers [i, i+1); level l intrinsics are K_0 scaled by 2^-l;
 *       Huber acts on the squared norm: rho(s) = s for s <= delta^2, else
 *       2 delta sqrt(s) - delta^2, and the anchor weight sits inside: rho(w ||r||^2);
 *       a step is accepted iff it lowers the objective and keeps at least
 *       min_valid_frac of the valid anchors visible; lambda x10 / /10 clamped to
 *       [1e-12, 1e12], reset to lambda0 at every level; rejected steps still count
 *       as iterations (a fixed number of iterations per level, no early exit).
 */
#ifndef PILOT_ALIGN_H
#define PILOT_ALIGN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PILOT_MAX_LEVELS 4

typedef enum {
    PILOT_OK = 0,
    PILOT_EINVAL = -1,    /* malformed config/frame/result, or a size beyond the handle's */
    PILOT_ENOMEM = -2,    /* device or pinned host allocation failed */
    PILOT_ECUDA = -3,     /* a CUDA runtime call or kernel launch failed */
    PILOT_ETIMEOUT = -4,  /* a bounded device-side wait gave up */
    PILOT_EBUSY = -5      /* serving: not admitted yet (no slot or memory free) */
} pilot_status;

/* Storage type of the feature pyramids (query maps and reference descriptors).
 * Arithmetic is always FP32; values are (stored value) x (per-channel scale). */
typedef enum {
    PILOT_F32 = 0,
    PILOT_BF16 = 1,
    PILOT_F16 = 2,
    PILOT_FP8E4M3 = 3
} pilot_dtype;

typedef enum {
    PILOT_HYP_OK = 0,
    PILOT_HYP_FEW_VALID = 1,  /* final n_valid below min_valid_frac x valid anchors */
    PILOT_HYP_NOT_PD = 2,     /* the last attempted damped solve was not positive definite */
    PILOT_HYP_NONFINITE = 3,  /* final objective or pose not finite */
    PILOT_HYP_PRUNED = 4      /* dropped by keep_top_k after a coarser level */
} pilot_hyp_status;

/* Solver options.  A zero-initialised struct means the defaults noted here. */
typedef struct {
    int iters_per_level[PILOT_MAX_LEVELS]; /* LM iterations at level l (0 = finest) */
    double lambda0;          /* initial damping; 0 -> 1e-3 */
    int damping_mode;        /* 0: H + lambda I (Eq. 8); 1: H + lambda diag(H) */
    double huber_photo;      /* delta of the photo Huber (Eq. 2); 0 -> 0.1 */
    double huber_grav;       /* delta of the gravity Huber (Eq. 7); 0 -> 0.1 */
    double huber_range;      /* delta of the range Huber, metres (Eq. 7); 0 -> 1.0 */
    int keep_top_k[PILOT_MAX_LEVELS]; /* after level l > 0 keep the K lowest objectives
                                         for the finer levels; 0 = keep all */
    double min_valid_frac;   /* acceptance / status threshold, fraction of valid anchors
                                in [0, 1]; 0 = no threshold (0.05 is the usual value) */
    int max_points;          /* workspace sizing: largest N, M, C the handle accepts */
    int max_hyps;
    int max_channels;
    int profile;             /* 1: time every build-pass launch with CUDA events */
    int max_frames;          /* batched form: largest number of frames per call; 0 -> 64
                                (max_hyps then bounds the hypotheses of the whole batch) */
    double gate_grav;        /* residual gates of the sensor priors (Supp. "Sensor-Prior
                                Fusion in LM": an excessively large prior residual is
                                down-weighted): a gravity residual norm above gate_grav, or a */
    double gate_range;       /* range residual above gate_range metres, adds the constant
                                cost w rho(gate^2) and nothing to H and g; 0 = no gate */
} pilot_align_config;

/* One query frame.  All pointers are owned by the caller and are either all device
 * pointers (is_device = 1) or all host pointers (is_device = 0; the solver copies them to
 * its workspace).  Every coordinate is in one local metric frame (e.g. centred on the
 * crop); x east, y north, z up; gravity points along -z in the world.  Feature pointers
 * (ref_feat, qry_feat) are 32-byte aligned for a device frame (the maps are read with loads
 * of up to 32 bytes) and 16-byte aligned for a host frame; scale pointers 16-byte aligned;
 * EINVAL otherwise. */
typedef struct {
    int is_device;
    int N;                          /* anchors (geo-anchors P_j, Supp. geo-anchor lift) */
    const float* points;            /* 3 x N SoA: x[N], y[N], z[N] */
    const float* point_weight;      /* N or NULL (= 1): w_l(j) of Eq. 2 */
    const uint8_t* point_valid;     /* N or NULL (= all valid); 0 = anchor unused */
    int C;                          /* channels: 4, 8, 16, 32 or 64 */
    int L;                          /* pyramid levels, 1..PILOT_MAX_LEVELS */
    pilot_dtype feat_dtype;
    const void* ref_feat[PILOT_MAX_LEVELS];   /* f_l^r(p_j): N x C per level */
    const float* ref_scale[PILOT_MAX_LEVELS]; /* C per level or NULL (= 1) */
    const void* qry_feat[PILOT_MAX_LEVELS];   /* f_l^q: H_l x W_l x C (NHWC) per level */
    const float* qry_scale[PILOT_MAX_LEVELS]; /* C per level or NULL (= 1) */
    const float* qry_conf[PILOT_MAX_LEVELS];  /* per level H_l x W_l query confidence w^q_l (FP32, 4-byte
                                                 aligned), or NULL (= 1): an anchor's weight in Eq. 2 is
                                                 point_weight x w^q_l read bilinearly at its projection
                                                 (the cell of the feature taps), held constant when
                                                 linearising (the uncertainty map of Sec. IV-C) */
    int H[PILOT_MAX_LEVELS], W[PILOT_MAX_LEVELS]; /* each >= 2 */
    double fx, fy, cx, cy;          /* level-0 pinhole intrinsics in pixels */
    int M;                          /* hypotheses */
    const double* T_cw;             /* M x 12 initial hypotheses [R | t], world->camera */
    int use_gravity;                /* Eq. 3 */
    double gravity_cam[3];          /* gamma^imu: measured gravity direction, camera frame */
    double gravity_world[3];        /* gamma^W, world frame (normally (0, 0, -1)) */
    double w_grav;                  /* lambda_imu */
    int use_range;                  /* Eq. 4-6 */
    double range_m;                 /* d^range along the ray through pixel (W_0/2, H_0/2) */
    double w_range;                 /* lambda_range */
    const float* dsm;               /* dsm_H x dsm_W heights; cell (r, c) is centred at */
    int dsm_H, dsm_W;               /* (dsm_x0 + (c + 1/2) gsd, dsm_y0 + (r + 1/2) gsd)  */
    double dsm_x0, dsm_y0, dsm_gsd;
} pilot_frame;

/* Caller-owned HOST output buffers.  Any pointer may be NULL to skip that output. */
typedef struct {
    double* T_cw;          /* M x 12 final poses */
    double* cost;          /* M final objective (pruned: at the level they were pruned) */
    int* n_valid;          /* M visible anchors at the final evaluation */
    int* hyp_status;       /* M pilot_hyp_status */
    int* best;             /* 1: index of the lowest objective among OK hypotheses, or -1 */
    long long* hyp_iters;  /* 1: sum over levels of (hypotheses run) x (iterations) */
} pilot_result;

typedef struct pilot_align_handle pilot_align_handle;

/* Create a solver handle and its device workspace on the current CUDA device.
 * cfg: options (copied).  out: receives the handle.  Returns PILOT_EINVAL for bad
 * options, PILOT_ENOMEM / PILOT_ECUDA if the workspace cannot be allocated. */
pilot_status pilot_align_create(const pilot_align_config* cfg, pilot_align_handle** out);

/* Check a frame against a config without touching the GPU (host logic only).
 * Returns PILOT_OK or PILOT_EINVAL with the reason in pilot_align_last_error(). */
pilot_status pilot_align_validate(const pilot_align_config* cfg, const pilot_frame* frame);

/* Run the whole multi-hypothesis coarse-to-fine LM solve of one frame (Sec. IV-E):
 * levels L-1 .. 0, iters_per_level[l] iterations each, optional top-K between levels,
 * selection of the lowest objective (Sec. IV-E, last paragraph).  Synchronous on
 * `stream` when it returns.  M = 0 returns PILOT_OK with best = -1. */
pilot_status pilot_align_solve(pilot_align_handle* h, const pilot_frame* frame,
                               pilot_result* result, void* stream);

/* Schedule of the build pass: chosen per frame shape by pilot_align_autotune (or set by
 * pilot_align_set_schedule), else the defaults (tile 1024, as many CTAs per SM as fit,
 * larger frames first). */
typedef struct {
    int tile;         /* anchors per reduction tile: 512, 1024, 2048 or 4096 */
    int ctas_per_sm;  /* batched form: persistent CTAs per SM; 0 = as many as fit */
    int job_order;    /* batched form: 0 = frames with more anchors first, 1 = frames in the caller's order */
    int streams;      /* plain form: 1 = one launch per LM iteration over all hypotheses;
                         2..4 = the hypotheses in that many parts, each launched on its own
                         stream, so that the FP64 steps ending one part's launch overlap the
                         other parts' gathers; 0 = 2.  Bitwise the same results. */
} pilot_schedule;

/* Autotuner: time the candidate schedules (4 tiles; for the plain form 1 or 2 streams, for
 * the batched form 1 or 2 CTAs per SM and both job orders) on these frames, `reps` timed runs each after one warm-up, and
 * keep the fastest for frames of this shape (storage type, C, and the powers of two of the
 * mean anchor and hypothesis counts).  batched = 0 tunes pilot_align_solve on frames[0];
 * batched = 1 tunes pilot_align_solve_batch on all frames.  *chosen and *best_ms (may be
 * NULL) receive the winner and its mean time.  Results of later solves may differ from the
 * default schedule's in the last bits (the reduction tile changes the summation order). */
pilot_status pilot_align_autotune(pilot_align_handle* h, const pilot_frame* frames, int n_frames,
                                  int batched, int reps, pilot_schedule* chosen, double* best_ms,
                                  void* stream);

/* Use `schedule` for later solves of frames of this shape (the key pilot_align_autotune
 * uses), replacing any tuned schedule: pins a schedule across runs, since the tile changes
 * the summation order.  EINVAL if a field is outside the values listed above. */
pilot_status pilot_align_set_schedule(pilot_align_handle* h, const pilot_frame* frames, int n_frames,
                                      int batched, const pilot_schedule* schedule);

/* The schedule the next solve of such frames would use (tuned, set or default). */
pilot_status pilot_align_get_schedule(const pilot_align_handle* h, const pilot_frame* frames,
                                      int n_frames, int batched, pilot_schedule* out);

/* Batched form: solve n_frames independent frames (uneven N, M, map sizes, intrinsics,
 * priors) in one pass per pyramid level.  Each level is one persistent cooperative launch
 * that runs the level's LM iterations over all (frame, hypothesis) jobs; its CTAs claim work
 * items (runs of anchor tiles of one tile of jobs, frames with more anchors first unless the
 * schedule says otherwise) from one counter.  A level with at least 2^23 anchor x hypothesis
 * units per iteration, or 4096 anchors per job on average, takes the items of all iterations in iteration-major order without grid
 * barriers: the CTA that completes a job tile's iteration runs its FP64 steps (one warp per
 * job) and releases the tile's next iteration.  A smaller level runs in lockstep: every item
 * of an iteration, a grid barrier, every job's FP64 step on one warp.  The launches, the per-frame top-K
 * and the selection are replayed from a CUDA graph captured on the first call (and again
 * when the storage type, C, L or schedule changes).
 * Requirements: every frame is a DEVICE frame; all frames share C, L, feat_dtype, the
 * presence of per-channel scales and of query confidence maps (each given on every level
 * or on none); n_frames <= max_frames; the hypotheses of all frames
 * together <= max_hyps, at most 8192 per frame.  PILOT_ETIMEOUT if a grid barrier or flag
 * wait gave up (only when the device could not keep every CTA resident; results are then
 * invalid).  results[i] receives frame i's outputs
 * exactly as pilot_align_solve would: with the same tile (both untuned, or tuned alike)
 * the reduction order is the same, so each frame's outputs are bitwise those of its own
 * pilot_align_solve, whatever else is in the batch.
 * Synchronous on `stream`. */
pilot_status pilot_align_solve_batch(pilot_align_handle* h, const pilot_frame* frames, int n_frames,
                                     pilot_result* results, void* stream);

/* ---- TDOM/DSM reference crop (Supp. "TDOM/DSM Reference Crop"): the step before the
 * solver that turns the global maps and a pose prior into a pixel-aligned 2.5D reference and
 * its geo-anchors ---- */

/* A georeferenced TDOM/DSM pair on the DEVICE: cell (r, c) is centred at
 * (x0 + (c + 1/2) gsd, y0 + (r + 1/2) gsd); heights are read bilinearly between cell centres. */
typedef struct {
    const float* dsm;             /* H x W heights (metres), row-major; required */
    const unsigned char* tdom;    /* H x W x 3 RGB, or NULL */
    int H, W;                     /* >= 2 each */
    double x0, y0, gsd;           /* gsd > 0 */
} pilot_map;

typedef struct {
    double T_cw[12];              /* pose prior [R | t], world -> camera, row-major */
    double fx, fy, cx, cy;        /* intrinsics of the query image, pixel-corner convention */
    int img_w, img_h;             /* query image size: the corner rays pass through (0, 0), (W, 0), (W, H), (0, H) */
    double s_min, s_step;         /* ray samples s_k = s_min + k s_step metres along each unit corner ray */
    int n_samples;                /* 1 .. 4194304 */
    int S;                        /* crop side in pixels, 1 .. 8192 */
} pilot_crop_params;

/* Reference crop, asynchronous on `stream`; allocates nothing.  Map footprint: for each image
 * corner k the ray sample minimising |z_ray(s) - h_DSM(x_ray(s), y_ray(s))| (samples off the
 * DSM skipped; ties to the nearer sample).  The homography maps the normalised crop square's
 * corners (0, 0), (1, 0), (1, 1), (0, 1) to the footprint points of image corners 0..3 as
 * offsets from the origin, the footprint centroid.  Warp and lift: crop pixel (u, v) (index
 * v S + u) is read at its centre; its map coordinates come from the homography, and
 *   points[v S + u], points[S^2 + v S + u], points[2 S^2 + v S + u] = x - ox, y - oy, DSM height
 *   valid[v S + u] = 1 inside the DSM's cell-centre grid, else 0 (and zero outputs)
 *   rgb[3 (v S + u) + k] = bilinear TDOM channel k as float (rgb may be NULL; zeros without a TDOM)
 * geometry (28 doubles, device): H[9] (H[8] = 1), origin[2], footprint points[12] (x, y, z of
 * image corners 0..3), sample index per corner (as double, -1 when a ray never crosses the DSM),
 * and 1.0 when the crop is valid (all four rays found, homography non-singular), else 0.0 with
 * every pixel invalid.  All outputs are device buffers owned by the caller (points 3 S^2 floats,
 * valid S^2 bytes, rgb 3 S^2 floats, geometry 28 doubles, naturally aligned).  EINVAL on bad
 * arguments (nothing launched); the crop's own failure is reported in geometry[27]. */
pilot_status pilot_crop_reference(const pilot_map* map, const pilot_crop_params* params, float* points,
                                  unsigned char* valid, float* rgb, double* geometry, void* stream);

/* Geo-anchor sampling from a reference crop (Supp. "TDOM/DSM Reference Crop": the valid
 * geo-anchors are sampled from the crop).  Draws min(n_select, number of valid pixels) of the
 * pixels whose valid byte is non-zero, uniformly without replacement: pixel j gets the key
 * (upper 32 bits of the (j+1)-th output of the SplitMix64 generator seeded with `seed`) * 2^32
 * + j and the valid pixels with the smallest keys are taken -- integer arithmetic only, so the
 * draw is exact and repeatable.  SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): state +=
 * 0x9E3779B97F4A7C15; z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9; z = (z ^ (z >> 27)) *
 * 0x94D049BB133111EB; output z ^ (z >> 31).  DEVICE pointers, owned by the caller:
 *   valid       n_pixels bytes (a crop's valid mask)
 *   points      3 x n_pixels FP32 SoA (a crop's geo-anchors), read only when out_points is set
 *   out_idx     n_select ints: the selected pixel indices in increasing order
 *   out_points  3 x n_select FP32 SoA (row stride n_select) or NULL: the selected anchors
 *   out_count   1 int: the number selected
 * Entries of out_idx / out_points past *out_count are left as they were.  Asynchronous on
 * `stream` (one CTA); allocates nothing.  EINVAL on negative sizes or missing pointers. */
pilot_status pilot_sample_anchors(const unsigned char* valid, const float* points, int n_pixels, int n_select,
                                  unsigned long long seed, int* out_idx, float* out_points, int* out_count,
                                  void* stream);

/* ---------------------------------------------------------------- sequential tracking
 * Pieces of the online loop (Supp. "Runtime Analysis": map preparation and localisation run
 * as two asynchronous stages; Sec. V-A: failure recovery).  Poses are [R | t] world ->
 * camera, 12 doubles row-major. */

/* Constant-velocity prior `steps` frames after T_prev: with T_prev2 (the estimate one frame
 * earlier) T_out = (T_prev T_prev2^-1)^steps T_prev, i.e. the last inter-frame motion in the
 * body frame repeated; with T_prev2 = NULL, T_out = T_prev.  Host function, FP64; T_out may
 * alias an input.  EINVAL on NULL, steps < 0 or non-finite input. */
pilot_status pilot_pose_predict(const double* T_prev, const double* T_prev2, int steps, double* T_out);

/* The pose re-expressed for points given relative to (dx, dy, 0): t_out = t + R (dx, dy, 0).
 * A reference crop's anchors are offsets from its origin (ox, oy): pilot_pose_reorigin(T_world,
 * ox, oy) gives the crop-local pose, pilot_pose_reorigin(T_local, -ox, -oy) the world pose.
 * Host function; T_out may alias T. */
pilot_status pilot_pose_reorigin(const double* T, double dx, double dy, double* T_out);

#define PILOT_MAX_SEED_XY 32
#define PILOT_MAX_SEED_YAW 64

typedef struct {
    double T_prior[12];                       /* prior pose, world -> camera */
    double origin_x, origin_y;                /* crop origin: the seeds are written crop-local */
    int n_xy, n_yaw;                          /* 1..32, 1..64 */
    double grid_xy[PILOT_MAX_SEED_XY];        /* metres, applied to x and to y */
    double grid_yaw_deg[PILOT_MAX_SEED_YAW];  /* degrees */
} pilot_seed_params;

/* Multi-hypothesis seeds around a prior (Sec. IV-E; Supp. "Multi-Hypothesis Refinement"):
 * hypothesis m = (i_x n_xy + i_y) n_yaw + i_psi has its camera centre at C + (grid_xy[i_x],
 * grid_xy[i_y], 0) and is turned about the world +z axis through its centre by
 * grid_yaw_deg[i_psi] (R_wc' = Rz(psi) R_wc, roll and pitch kept), then re-origined to the
 * crop.  Writes n_xy^2 n_yaw x 12 doubles to the DEVICE buffer T_out (8-byte aligned, owned by
 * the caller) on `stream`, ready as a device frame's T_cw; asynchronous, allocates nothing.
 * EINVAL on bad arguments (nothing launched). */
pilot_status pilot_seed_hypotheses(const pilot_seed_params* params, double* T_out, void* stream);

/* Roofline probes (the paper has no counterpart): measured ceilings the build pass is
 * compared against.  pilot_probe_fma: FP32 FMA throughput in TFLOP/s (packed FP32x2 FMAs on
 * every SM).  pilot_probe_gather: GB/s of the build pass' access pattern without its
 * arithmetic -- `samples` 4-tap bilinear footprints (taps (r, c), (r, c + 1), (r + 1, c),
 * (r + 1, c + 1), C contiguous channels each) at uniformly random pixels of a device NHWC map
 * of H x W x C elements of `dtype`, one 16-byte load per lane; bytes counted = samples x 4 x
 * C x element size.  The map must be 16-byte aligned with C x element size in {16, 32, 64,
 * 128} bytes.  Each times one launch after a warm-up one on `stream`; synchronous. */
pilot_status pilot_probe_fma(double* tflops, void* stream);
pilot_status pilot_probe_gather(const void* map, int H, int W, int C, pilot_dtype dtype, long long samples,
                                double* gbps, void* stream);

/* Gather ceiling of the build pass' access pattern on a real frame (the paper has no
 * counterpart; a roofline probe).  Runs the build pass' loads without its arithmetic on
 * the same grid (ceil(N / tile) anchor tiles x tiles of the build pass' number of poses per
 * CTA, 256 threads, its lane layout): every (anchor, pose) projects the anchor (Eq. 1, level
 * intrinsics fx, fy, cx, cy in pixels of this map, corner convention) and reads its 4 taps,
 * and every anchor's reference row is read once for the CTA's poses, with the build pass'
 * loads by lane groups for maps without per-channel scales (32 bytes per lane for FP32 and
 * 16-bit taps of 32 bytes or more, 16 otherwise),
 * so the cache reuse between neighbouring anchors is the frame's own.  Two batches of anchors
 * are in flight per step.  DEVICE pointers: points 3 x N FP32 SoA; map H x W x C NHWC and ref
 * N x C in `dtype` (aligned to that load width; C x element size a power of two from 16 to
 * 256 bytes); poses32
 * M x 12 FP32 [R | t] world -> camera.  Times one launch after a warm-up one on `stream`
 * (synchronous) and returns the (anchor, pose) units per second in *units_per_s. */
pilot_status pilot_probe_gather_frame(const float* points, int N, const void* map, const void* ref, int H, int W,
                                      int C, pilot_dtype dtype, double fx, double fy, double cx, double cy,
                                      const float* poses32, int M, int tile, double* units_per_s, void* stream);

/* Failure-detection self-test of the batched form's grid barrier (the paper has no
 * counterpart; the persistent level kernel's barrier waits are bounded in time so that a
 * device that cannot keep every CTA resident yields PILOT_ETIMEOUT instead of a hang).
 * Launches that kernel with no work and a barrier that waits for one CTA more than the
 * launch has, so every CTA gives up after timeout_ms (1 .. 10000) and sets the error word.
 * Returns PILOT_OK when the timeout was reported and the launch ended (*elapsed_ms, may be
 * NULL, receives its device time); the handle stays usable.  Overwrites the handle's batch
 * descriptors, which the next pilot_align_solve_batch uploads again.  Synchronous. */
pilot_status pilot_align_selftest_barrier_timeout(pilot_align_handle* h, double timeout_ms, double* elapsed_ms,
                                                  void* stream);

/* Failure-detection self-test of the batched form's schedule without grid barriers (the paper
 * has no counterpart): solves the caller's n DEVICE frames (pilot_align_solve_batch's
 * requirements) with every wait for a job tile's published iteration asking for one more
 * than will ever be published, so the first waiting CTA gives up after timeout_ms (1 ..
 * 10000) and sets the error word, and every later wait and barrier of the solve ends at once.
 * Returns PILOT_OK when the solve reported the timeout (PILOT_ETIMEOUT) and ended (*elapsed_ms,
 * may be NULL, receives its host wall time); PILOT_EINVAL when no level of the batch takes
 * that schedule (fewer than 2^23 anchor x hypothesis units per iteration and fewer than 4096
 * anchors per job).  The results are discarded; the handle stays usable.  Synchronous. */
pilot_status pilot_align_selftest_flag_timeout(pilot_align_handle* h, const pilot_frame* frames, int n,
                                               double timeout_ms, double* elapsed_ms, void* stream);

/* Evaluate the normal equations of the total objective (Eq. 7, Eq. 8) at the given
 * poses on one level, without any LM step: out29 (HOST, M x 29 doubles) receives per
 * pose the 21 upper-triangle entries of J^T W J (row-major), the 6 entries of J^T W r,
 * the objective, and the number of visible anchors.  T_cw (HOST, M x 12) overrides
 * frame->T_cw.  This is the parity hook of the build pass. */
pilot_status pilot_align_debug_normal_eq(pilot_align_handle* h, const pilot_frame* frame,
                                         int level, const double* T_cw, double* out29,
                                         void* stream);

/* Timing of the last solve when cfg.profile = 1: total device time of the build-pass
 * launches (milliseconds, CUDA events on the solve's stream), their number, and the
 * number of kernels of this library launched by that solve. */
pilot_status pilot_align_profile(const pilot_align_handle* h, double* build_ms,
                                 int* build_launches, int* total_launches);

/* Normal equations at given poses, like pilot_align_debug_normal_eq, for callers that
 * cannot allocate device memory.  (The paper has no counterpart: this is a deployment
 * variant of the build-pass evaluation.)  Some callers may not call cudaMalloc: a process
 * whose device memory is handed out by an external pool it must go through, or a
 * latency-bound loop that cannot risk an allocation's implicit device synchronisation.
 * This call allocates nothing and needs no handle; its scratch is a fixed array of about
 * 2.3 MB that every GPU loading this library holds until the process exits.
 *   cfg:    options.  Read: huber_photo, huber_grav, huber_range (0 means the default),
 *           gate_grav, gate_range, and the fields pilot_align_validate checks.  Not read:
 *           max_points, max_hyps and max_channels -- the frame is checked against this
 *           call's own limits below instead of a handle's workspace sizes.
 *   frame:  a DEVICE frame (is_device = 1, else PILOT_EINVAL), N <= 65536 anchors, C <= 64.
 *           Scales: as in the handle-based calls, a frame giving only one of qry_scale /
 *           ref_scale on a level reads the missing one as ones.
 *   level:  pyramid level to evaluate
 *   T_cw:   DEVICE pointer, frame->M x 12 poses (frame->T_cw is ignored), M <= 256
 *   out29:  DEVICE pointer, frame->M x 29 doubles, written like debug_normal_eq's out29
 *           (the same kernels and tile: bitwise the same values)
 *   stream: cudaStream_t as void*; the call only enqueues work: out29 is ready when the
 *           stream reaches that point.
 * Sizes beyond the limits return PILOT_EINVAL with the limit in pilot_align_last_error().
 * The first call in a CUDA context (per device) looks up the scratch address for it (make
 * that first call before any stream capture); a context created anew, e.g. after
 * cudaDeviceReset, gets a new lookup on its first call.  All calls share the one scratch
 * array, which keeps the last call's contents: calls whose work overlaps on the GPU race on
 * it, so the caller must serialise them. */
pilot_status pilot_align_normal_eq_noalloc(const pilot_align_config* cfg, const pilot_frame* frame,
                                           int level, const double* T_cw, double* out29,
                                           void* stream);

/* Quantise feature rows for reduced-precision storage (the precision form of the path:
 * feature pyramids in BF16, FP16 or FP8-E4M3 with FP32 arithmetic).  DEVICE pointers:
 *   src   rows x C FP32 (16-byte aligned), e.g. an H x W x C map (rows = H W) or an
 *         N x C reference block
 *   dst   rows x C elements of `dtype` (BF16, F16 or FP8E4M3)
 *   scale C FP32 per-channel scales, written: s_c = absmax_c / q_max when per_channel = 1
 *         or dtype = FP8E4M3 (q_max = 448 for E4M3, 65504 for F16, 1 for BF16), else 1;
 *         a channel whose absmax is 0 gets s_c = 1
 * dst = round(src / s_c) (FP32 product with the reciprocal of s_c), rounded to nearest
 * even, E4M3 saturating at +-448.  The value the solver uses is dst x s_c: pass `scale` as
 * the frame's qry_scale / ref_scale.  Only enqueues work on `stream`; allocates nothing. */
pilot_status pilot_quantize_features(const float* src, long long rows, int C, pilot_dtype dtype,
                                     int per_channel, void* dst, float* scale, void* stream);

/* Release the handle and its device workspace.  NULL is ignored. */
void pilot_align_destroy(pilot_align_handle* h);

/* ---- Serving: continuous batching of frames from many concurrent streams ----
 *
 * A server owns a worker thread and the current CUDA device.  Frames are admitted when a
 * slot is free, their hypotheses fit in cfg.max_hyps (shared by all admitted frames) and
 * their data fit in the device arena of hbm_budget bytes; admission copies the frame into
 * the arena, where its pyramid and LM state stay until it completes.  The worker then runs
 * rounds: in each round every admitted frame advances one pyramid level, all frames sharing
 * one persistent launch (replayed from a CUDA graph) whatever level each is at; frames that
 * arrive meanwhile join at the next round.  A frame's outputs are exactly those
 * pilot_align_solve gives for it, however many other frames are being served.  All served
 * frames must share C, L, feat_dtype and the presence of scales and of query confidence
 * maps, each given on every level or on none (fixed by the first frame). */
typedef struct pilot_server pilot_server;

/* Counters since create.  round_device_ms: device time of all rounds (CUDA events around
 * each round's graph on the server's stream); round_wall_ms: host time from each round's
 * launch to its completion.  Wall time outside rounds is spent admitting and staging frames
 * or waiting for work. */
typedef struct {
    long long rounds, admitted, completed, pending, active, peak_active;
    long long arena_bytes_in_use, arena_bytes_peak;
    double round_device_ms, round_wall_ms;
} pilot_serve_stats;

/* cfg: solver options (max_hyps bounds the hypotheses of all admitted frames together);
 * hbm_budget: device bytes reserved for frame data; max_slots: most frames admitted at once. */
pilot_status pilot_serve_create(const pilot_align_config* cfg, size_t hbm_budget, int max_slots,
                                pilot_server** out);

/* Queue a frame (host or device pointers, which must stay valid and unchanged until the
 * ticket is reported done).  Returns PILOT_EBUSY when the pending queue (4 x max_slots + 64)
 * is full, PILOT_EINVAL for a frame that could never be admitted. */
pilot_status pilot_serve_submit(pilot_server* s, const pilot_frame* frame, uint64_t* ticket);

/* Non-blocking: *done = 1 once the frame completed; its outputs are then copied into
 * `result` (may be NULL), *latency_ms (may be NULL) is submit-to-completion wall time, and
 * the ticket is retired. */
pilot_status pilot_serve_poll(pilot_server* s, uint64_t ticket, pilot_result* result, int* done,
                              double* latency_ms);

/* Blocking form of poll; PILOT_ETIMEOUT after timeout_ms. */
pilot_status pilot_serve_wait(pilot_server* s, uint64_t ticket, pilot_result* result,
                              double* latency_ms, int timeout_ms);

/* Pyramid levels every admitted frame advances per round (1 by default: one level per round,
 * so frames that arrive meanwhile join after at most one level's work).  With n > 1 each round
 * runs n levels back to back (one persistent launch each; between them the device applies
 * the top-K and moves every listed frame to its next level), so a frame needs fewer rounds:
 * lower latency when the load is light, longer rounds for frames that arrive meanwhile.
 * With n = 0 the count is chosen per frame and round: a frame whose level work (anchors x
 * active hypotheses) is at most 2^21 runs all its remaining levels, a larger one one level.
 * Outputs are the same bitwise.  Only before the first pilot_serve_submit; EINVAL otherwise
 * or for n outside [0, 4]. */
pilot_status pilot_serve_set_levels_per_round(pilot_server* s, int levels);

/* SMs' worth of CTA slots the rounds' persistent launches leave unused (0 by default: every
 * slot).  A round holds the slots it takes for its whole duration, so work the clients enqueue
 * on other streams of the device (crops, feature extraction, seeding) waits for the round to
 * end unless some slots are left free; with n > 0 it runs beside the rounds, at the price of
 * about n / SM count of the rounds' throughput.  Outputs are the same bitwise (the work is
 * claimed dynamically; the reduction order does not depend on the grid).  Only before the
 * first pilot_serve_submit; EINVAL otherwise or for n outside [0, SM count). */
pilot_status pilot_serve_set_reserved_sms(pilot_server* s, int n_sms);

pilot_status pilot_serve_get_stats(pilot_server* s, pilot_serve_stats* out);

/* Stops the worker after its current round and releases everything; tickets not yet
 * polled are dropped.  NULL is ignored. */
void pilot_serve_destroy(pilot_server* s);

/* Message describing the last failure on the calling thread ("" if none). */
const char* pilot_align_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PILOT_ALIGN_H */
