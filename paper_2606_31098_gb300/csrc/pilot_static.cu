// pilot_align_normal_eq_noalloc: the normal-equation evaluation of the build pass for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a process whose device memory is handed out by
// an external pool or allocator it must go through, or a latency-bound loop (a flight
// controller, a serving thread) that may not risk an allocation's implicit device
// synchronisation.  This entry point allocates nothing.  Its scratch (hypothesis
// state, FP32 candidate poses, slot list and the per-tile partial sums) lives in one
// file-scope __device__ array of fixed size; every GPU that loads the library holds that
// array until the process exits.  The caller passes device pointers for all inputs and
// for the output.
//
// Host code cannot use the array's name as a device address (it names a host-side stand-in),
// so the first call in each CUDA context (per device, with that device current) looks the
// address up with cudaGetSymbolAddress and caches it under the context's unique id; a
// context created anew (after cudaDeviceReset, say) gets a fresh lookup.  That first call
// should come before any stream capture.  All calls share the one array: calls whose work
// overlaps on the GPU (two streams, or two threads) race on it and must be serialised by
// the caller.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "pilot_internal.cuh"

namespace pilot {
namespace {

constexpr int kStaticMaxHyps = 256;
constexpr int kStaticTile = 1024;
constexpr int kStaticMaxTiles = 64;                     // anchors <= 64 x 1024 = 65536
constexpr int kStaticMaxPoints = kStaticMaxTiles * kStaticTile;

constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kOffState = 0;
constexpr size_t kOffPose = align256(kOffState + sizeof(HypState) * kStaticMaxHyps);
constexpr size_t kOffActive = align256(kOffPose + sizeof(float) * 12 * kStaticMaxHyps);
constexpr size_t kOffMinValid = align256(kOffActive + sizeof(int) * kStaticMaxHyps);
constexpr size_t kOffPartial = align256(kOffMinValid + sizeof(double));
constexpr size_t kScratchBytes =
    align256(kOffPartial + sizeof(float) * kAcc * kStaticMaxTiles * (size_t)kStaticMaxHyps);

// The scratch: about 2.3 MB per device.  Every word a call reads is written earlier in
// the same call (poses, flags and slot list by set_poses, every partial record by the
// build pass), so nothing needs clearing between calls.
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Unit scales, read in place of a missing scale array when the frame gives only one of the
// pair (the handle-based entry points read a missing one as ones too).
__device__ __align__(16) float g_noalloc_ones[64] = {
    1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f,
    1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f,
    1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f,
    1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f};

constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct ScratchCache {
    unsigned long long ctx_id;     // 0: nothing cached
    unsigned char* scratch;
    float* ones;
};
ScratchCache g_cache[kMaxDevices] = {};

// Unique id of the calling thread's current CUDA context (0 when it cannot be read; the
// caller then looks the addresses up on every call).  Read through the runtime's driver
// entry-point query, so the library does not link the driver library itself.
unsigned long long current_context_id() {
    typedef CUresult (*GetCurrent)(CUcontext*);
    typedef CUresult (*GetId)(CUcontext, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        cudaDriverEntryPointQueryResult q1, q2;
        void* f1 = nullptr;
        void* f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<GetCurrent>(f1);
            get_id = reinterpret_cast<GetId>(f2);
        }
        looked_up = true;
    }
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

pilot_status fail_msg(pilot_status st, const std::string& msg) {
    record_error(msg.c_str());
    return st;
}

// Device addresses of the scratch and of the unit scales in the current context (looked
// up once per device and context).
pilot_status scratch_address(unsigned char** scratch, float** ones) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_msg(PILOT_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail_msg(PILOT_EINVAL, "device ordinal beyond 64");
    std::lock_guard<std::mutex> lock(g_mu);
    ScratchCache& c = g_cache[dev];
    const unsigned long long ctx = current_context_id();   // 0 before the thread's first runtime call
    if (ctx == 0 || c.ctx_id != ctx) {
        void* p = nullptr;
        void* q = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);     // makes the device's context current
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&q, g_noalloc_ones);
        if (e != cudaSuccess || !p || !q)
            return fail_msg(PILOT_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        c.scratch = static_cast<unsigned char*>(p);
        c.ones = static_cast<float*>(q);
        c.ctx_id = current_context_id();
    }
    *scratch = c.scratch;
    *ones = c.ones;
    return PILOT_OK;
}

cudaError_t dispatch(pilot_dtype dt, const BuildParams& b, cudaStream_t s) {
    switch (dt) {
        case PILOT_F32: return launch_build_dtype<PILOT_F32>(b, s);
        case PILOT_BF16: return launch_build_dtype<PILOT_BF16>(b, s);
        case PILOT_F16: return launch_build_dtype<PILOT_F16>(b, s);
        case PILOT_FP8E4M3: return launch_build_dtype<PILOT_FP8E4M3>(b, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace
}  // namespace pilot

using namespace pilot;

extern "C" pilot_status pilot_align_normal_eq_noalloc(const pilot_align_config* cfg,
                                                      const pilot_frame* f, int level,
                                                      const double* T_cw, double* out29,
                                                      void* stream) {
    if (!cfg || !f || !T_cw || !out29) return fail_msg(PILOT_EINVAL, "config, frame, T_cw or out29 is NULL");
    if (f->N > kStaticMaxPoints)
        return fail_msg(PILOT_EINVAL, "N = " + std::to_string(f->N) + " exceeds the fixed scratch limit of " +
                                          std::to_string(kStaticMaxPoints) + " anchors");
    if (f->M > kStaticMaxHyps)
        return fail_msg(PILOT_EINVAL, "M = " + std::to_string(f->M) + " exceeds the fixed scratch limit of " +
                                          std::to_string(kStaticMaxHyps) + " poses");
    // the frame is checked against this call's own fixed limits, not the caller's workspace
    // sizes (max_points, max_hyps, max_channels are not read)
    pilot_align_config lim = *cfg;
    lim.max_points = kStaticMaxPoints;
    lim.max_hyps = kStaticMaxHyps;
    lim.max_channels = 64;
    pilot_status st = pilot_align_validate(&lim, f);
    if (st != PILOT_OK) return st;
    if (!f->is_device)
        return fail_msg(PILOT_EINVAL, "pilot_align_normal_eq_noalloc needs a device frame (is_device = 1)");
    if (level < 0 || level >= f->L) return fail_msg(PILOT_EINVAL, "level outside [0, L)");
    if (f->M == 0) return PILOT_OK;
    unsigned char* base = nullptr;
    float* ones = nullptr;
    if ((st = scratch_address(&base, &ones)) != PILOT_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    HypState* state = reinterpret_cast<HypState*>(base + kOffState);
    float* pose32 = reinterpret_cast<float*>(base + kOffPose);
    int* active = reinterpret_cast<int*>(base + kOffActive);
    double* min_valid = reinterpret_cast<double*>(base + kOffMinValid);
    float* partial = reinterpret_cast<float*>(base + kOffPartial);

    const double huber_photo = cfg->huber_photo == 0.0 ? 0.1 : cfg->huber_photo;
    const double huber_grav = cfg->huber_grav == 0.0 ? 0.1 : cfg->huber_grav;
    const double huber_range = cfg->huber_range == 0.0 ? 1.0 : cfg->huber_range;

    cudaError_t e = launch_set_poses(state, pose32, T_cw, active, f->M, s);
    if (e != cudaSuccess) return fail_msg(PILOT_ECUDA, std::string("set_poses launch: ") + cudaGetErrorString(e));

    BuildParams b{};
    const size_t N = (size_t)f->N;
    b.px = f->points;
    b.py = f->points ? f->points + N : nullptr;
    b.pz = f->points ? f->points + 2 * N : nullptr;
    b.weight = f->point_weight;
    b.valid = f->point_valid;
    b.qry = f->qry_feat[level];
    b.ref = f->ref_feat[level];
    // scales: a missing one of the pair reads as ones, as in the handle-based entry points
    if (f->qry_scale[level] || f->ref_scale[level]) {
        b.qscale = f->qry_scale[level] ? f->qry_scale[level] : ones;
        b.rscale = f->ref_scale[level] ? f->ref_scale[level] : ones;
    }
    b.conf = f->qry_conf[level];
    b.N = f->N;
    b.C = f->C;
    b.H = f->H[level];
    b.W = f->W[level];
    const double sc = ldexp(1.0, -level);
    b.fx = (float)(f->fx * sc);
    b.fy = (float)(f->fy * sc);
    b.cx = (float)(f->cx * sc);
    b.cy = (float)(f->cy * sc);
    b.huber = (float)huber_photo;
    b.pose32 = pose32;
    b.active_idx = active;
    b.state = state;
    b.partial = partial;
    b.n_active = f->M;
    b.tile = kStaticTile;
    b.n_tiles = f->N > 0 ? (f->N + kStaticTile - 1) / kStaticTile : 1;
    e = dispatch(f->feat_dtype, b, s);
    if (e != cudaSuccess) return fail_msg(PILOT_ECUDA, std::string("build-pass launch: ") + cudaGetErrorString(e));

    EpilogueParams ep{};
    ep.state = state;
    ep.pose32 = pose32;
    ep.partial = partial;
    ep.active_idx = active;
    ep.n_active = f->M;
    ep.n_tiles = b.n_tiles;
    ep.mode = kEpiEval;
    ep.eval_out = out29;
    PriorParams& pp = ep.prior;
    pp.use_gravity = f->use_gravity;
    for (int i = 0; i < 3; ++i) {
        pp.g_cam[i] = f->gravity_cam[i];
        pp.g_world[i] = f->gravity_world[i];
    }
    pp.w_grav = f->w_grav;
    pp.huber_grav = huber_grav;
    pp.use_range = f->use_range;
    if (f->use_range) {
        const double k[3] = {(0.5 * f->W[0] - f->cx) / f->fx, (0.5 * f->H[0] - f->cy) / f->fy, 1.0};
        const double nk = sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
        for (int i = 0; i < 3; ++i) pp.q[i] = f->range_m * k[i] / nk;
    }
    pp.w_range = f->w_range;
    pp.huber_range = huber_range;
    pp.dsm = f->use_range ? f->dsm : nullptr;
    pp.dsm_H = f->dsm_H;
    pp.dsm_W = f->dsm_W;
    pp.dsm_x0 = f->dsm_x0;
    pp.dsm_y0 = f->dsm_y0;
    pp.dsm_gsd = f->dsm_gsd;
    pp.dsm_inv_gsd = 1.0 / f->dsm_gsd;
    pp.gate_grav = cfg->gate_grav;
    pp.gate_range = cfg->gate_range;
    e = launch_epilogue(ep, min_valid, s);
    if (e != cudaSuccess) return fail_msg(PILOT_ECUDA, std::string("epilogue launch: ") + cudaGetErrorString(e));
    return PILOT_OK;
}
