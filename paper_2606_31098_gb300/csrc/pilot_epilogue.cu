// Per-hypothesis FP64 epilogue of each build pass, and the small bookkeeping kernels.
//
//   tile sums     FP64 sum of the build pass' FP32 partial records, fixed order
//   gravity term  Eq. 3: r = R gamma^W - gamma^imu, J = [0 | -[a]x], a = R gamma^W
//   range term    Eq. 4-6: P = R^T (q - t), r = P_z - D(P_x, P_y), J = [-n | n x q]
//                 with n = R (-D_x, -D_y, 1) and q = d v
//   assembly      Supp. "Sensor-Prior Fusion in LM": H, g are sums over the terms
//   LM step       Eq. 8: (H + lambda I) dxi = -g by 6x6 Cholesky, Eq. 9: T' = exp(dxi) T
//   acceptance    keep T' iff its objective is lower and enough anchors stay visible
//   top-K         Supp. "Multi-Hypothesis Refinement": keep the K lowest objectives
//   selection     Sec. IV-E: argmin of the final objective over usable hypotheses
#include <math.h>

#include "pilot_fp64.cuh"
#include "pilot_internal.cuh"

namespace pilot {

namespace {

// One block of 256 threads per hypothesis slot: FP64 sum of the tile records (8 partial
// chains per value, combined in a fixed order), then the FP64 LM step on warp 0.
__global__ void epilogue_kernel(const EpilogueParams p, const double* min_valid_ptr) {
    const int slot = blockIdx.x;
    __shared__ double part[8][kAcc];
    __shared__ double E[kAcc];
    const int v = threadIdx.x & 31, c = threadIdx.x >> 5;
    const HypState& st = p.state[p.active_idx[slot]];
    const bool evaluated = (p.mode == kEpiStep) ? (st.has_cand != 0) : true;
    if (evaluated) {
        const float* src = p.partial + (size_t)slot * p.n_tiles * kAcc + v;
        double acc = 0.0;
        for (int t = c; t < p.n_tiles; t += 8) acc += (double)src[(size_t)t * kAcc];
        part[c][v] = acc;
        __syncthreads();
        if (threadIdx.x < kAcc) {
            double sum = 0.0;
            for (int k = 0; k < 8; ++k) sum += part[k][threadIdx.x];
            E[threadIdx.x] = sum;
        }
    }
    __syncthreads();
    if (threadIdx.x >= 32) return;                 // warp 0 runs the FP64 step
    const double min_valid = (p.mode == kEpiEval) ? 0.0 : *min_valid_ptr;
    lm_step(p, slot, E, &part[0][0], min_valid, threadIdx.x);
}

__global__ void hyp_init_kernel(HypState* st, const double* T_cw, int* active_idx, int M) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    HypState& s = st[m];
    for (int i = 0; i < 12; ++i) s.T[i] = s.Tc[i] = T_cw[12 * m + i];
    for (int i = 0; i < 21; ++i) s.H[i] = 0.0;
    for (int i = 0; i < 6; ++i) s.g[i] = 0.0;
    s.cost = 0.0;
    s.lambda = 0.0;
    s.n_valid = 0;
    s.has_cand = 0;
    s.last_fail = 0;
    s.active = 1;
    s.status = PILOT_HYP_OK;
    active_idx[m] = m;
}

__global__ void set_poses_kernel(HypState* st, float* pose32, const double* T_cw, int* active_idx,
                                 int M) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    for (int i = 0; i < 12; ++i) st[m].T[i] = T_cw[12 * m + i];
    store_pose32(pose32 + 12 * m, st[m].T);
    st[m].has_cand = 1;
    active_idx[m] = m;
}

__global__ void level_init_kernel(HypState* st, float* pose32, const int* active_idx, int n_active,
                                  double lambda0) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_active) return;
    const int m = active_idx[s];
    st[m].lambda = lambda0;
    st[m].last_fail = 0;
    st[m].has_cand = 1;
    store_pose32(pose32 + 12 * m, st[m].T);
}

// Ranking key of a hypothesis: (unusable, cost, index), unusable = non-finite objective or
// too few visible anchors; unusable ones compare by index only.  The cost is compared as an
// order-preserving 64-bit integer image of the double (both zeros map to one value), which
// orders exactly as the doubles do but keeps the n^2 comparisons off the FP64 pipe.
__device__ __forceinline__ void rank_key(const HypState& h, double min_valid, int* bad,
                                         unsigned long long* c) {
    *bad = !(isfinite(h.cost) && h.n_valid >= min_valid);
    const unsigned long long u = (unsigned long long)__double_as_longlong((isfinite(h.cost) ? h.cost : 0.0) + 0.0);
    *c = (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

// The (unusable, cost image, index) order as one lexicographic comparison of two 64-bit
// words: hi = unusable bit | cost image >> 1, lo = lowest cost-image bit | index.
__device__ __forceinline__ ulonglong2 order_key(int bad, unsigned long long c, int idx) {
    return make_ulonglong2(((unsigned long long)(bad != 0) << 63) | (c >> 1),
                           ((c & 1ull) << 63) | (unsigned long long)(unsigned)idx);
}

// Top-K (Supp. "Multi-Hypothesis Refinement") over the n hypotheses listed in act[0, n) of
// S, in two passes.  rank_mark: each thread of a block takes one listed hypothesis from
// [s_begin, s_begin + blockDim.x), counts the listed hypotheses that rank before it (keys
// streamed through shared memory blockDim.x at a time) and marks it pruned if that count is
// K or more; many blocks share the n^2 comparisons.  compact_active (one block, blockDim.x a
// multiple of 32, at most 1024, after every rank_mark block has finished): writes the
// survivors' indices, in their order in act, to act_out[0, K) (act_out may be act) by a
// block-wide prefix count.
constexpr int kRankThreads = 256;

__device__ void rank_mark(HypState* S, const int* act, int n, int K, double min_valid, int s_begin) {
    __shared__ ulonglong2 kk[kRankThreads];      // order keys of the current chunk
    const int tid = threadIdx.x;
    const int s = s_begin + tid;
    int m = -1, rank = 0;
    ulonglong2 key = make_ulonglong2(~0ull, ~0ull);
    if (s < n) {
        int bad;
        unsigned long long c;
        m = act[s];
        rank_key(S[m], min_valid, &bad, &c);
        key = order_key(bad, c, m);
    }
    for (int c0 = 0; c0 < n; c0 += kRankThreads) {
        __syncthreads();
        if (c0 + tid < n) {
            int bad;
            unsigned long long c;
            const int m2 = act[c0 + tid];
            rank_key(S[m2], min_valid, &bad, &c);
            kk[tid] = order_key(bad, c, m2);
        }
        __syncthreads();
        if (s < n) {
            const int lim = min(kRankThreads, n - c0);
#pragma unroll 4
            for (int j = 0; j < lim; ++j) {
                const ulonglong2 o = kk[j];
                rank += (o.x < key.x) | ((o.x == key.x) & (o.y < key.y));
            }
        }
    }
    if (s < n && rank >= K) {
        S[m].active = 0;
        S[m].status = PILOT_HYP_PRUNED;
    }
}

__device__ void compact_active(const HypState* S, const int* act, int* act_out, int n) {
    __shared__ int wsum[32];
    __shared__ int s_base;
    const int bd = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_base = 0;
    __syncthreads();
    for (int c0 = 0; c0 < n; c0 += bd) {
        const int s = c0 + tid;
        int m = -1;
        bool keep = false;
        if (s < n) {
            m = act[s];
            keep = S[m].active != 0;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) wsum[warp] = __popc(bal);
        __syncthreads();
        int off = s_base;
        for (int w = 0; w < warp; ++w) off += wsum[w];
        if (keep) act_out[off + __popc(bal & ((1u << lane) - 1u))] = m;
        __syncthreads();
        if (tid == 0) {
            int t = 0;
            for (int w = 0; w < bd / 32; ++w) t += wsum[w];
            s_base += t;
        }
        __syncthreads();
    }
}

// Plain form: blockIdx.x ranks listed hypotheses [256 blockIdx.x, + 256).
__global__ void prune_rank_kernel(HypState* st, const int* active_in, int n, int K, const double* min_valid_ptr) {
    rank_mark(st, active_in, n, K, *min_valid_ptr, blockIdx.x * kRankThreads);
}

// Plain form: the survivors, in their order in active_in, to active_out.
__global__ void prune_compact_kernel(const HypState* st, const int* active_in, int* active_out, int n) {
    compact_active(st, active_in, active_out, n);
}

// One block of 1024 threads: number of valid anchors (4 flags per load when aligned).
__global__ void count_valid_kernel(const uint8_t* valid, int N, double frac, double* min_valid) {
    __shared__ int part[32];
    int c = 0;
    if (!valid) {
        c = (threadIdx.x == 0) ? N : 0;
    } else if (((uintptr_t)valid & 3) == 0) {
        const uint32_t* w = reinterpret_cast<const uint32_t*>(valid);
        for (int k = threadIdx.x; k < N / 4; k += blockDim.x) {
            const uint32_t v = w[k];
            c += ((v & 0xffu) != 0) + ((v & 0xff00u) != 0) + ((v & 0xff0000u) != 0) + ((v >> 24) != 0);
        }
        for (int j = (N / 4) * 4 + threadIdx.x; j < N; j += blockDim.x) c += valid[j] != 0;
    } else {
        for (int j = threadIdx.x; j < N; j += blockDim.x) c += valid[j] != 0;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x < 32) {
        int v = (threadIdx.x < (blockDim.x >> 5)) ? part[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) *min_valid = frac * (double)v;
    }
}

// One block (blockDim.x a power of two, at most 1024): final statuses, result block, argmin
// (ties -> lowest index).
__global__ void finalize_kernel(HypState* st, int M, const double* min_valid_ptr,
                                unsigned char* res, ResultLayout lay) {
    const double min_valid = *min_valid_ptr;
    double* T = reinterpret_cast<double*>(res + lay.off_T);
    double* cost = reinterpret_cast<double*>(res + lay.off_cost);
    int* nv = reinterpret_cast<int*>(res + lay.off_nvalid);
    int* status = reinterpret_cast<int*>(res + lay.off_status);
    int* best = reinterpret_cast<int*>(res + lay.off_best);
    __shared__ double bc[1024];
    __shared__ int bi[1024];
    double my_c = 0.0;
    int my_i = -1;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        HypState& s = st[m];
        if (s.active) {
            bool finite = isfinite(s.cost);
            for (int i = 0; i < 12; ++i) finite = finite && isfinite(s.T[i]);
            int code;
            if (!finite) code = PILOT_HYP_NONFINITE;
            else if (s.n_valid < min_valid) code = PILOT_HYP_FEW_VALID;
            else if (s.last_fail) code = PILOT_HYP_NOT_PD;
            else code = PILOT_HYP_OK;
            s.status = code;
        }
        for (int i = 0; i < 12; ++i) T[12 * m + i] = s.T[i];
        cost[m] = s.cost;
        nv[m] = s.n_valid;
        status[m] = s.status;
        if (s.status == PILOT_HYP_OK && (my_i < 0 || s.cost < my_c)) {
            my_c = s.cost;
            my_i = m;
        }
    }
    bc[threadIdx.x] = my_c;
    bi[threadIdx.x] = my_i;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const int j = threadIdx.x + s;
            const bool take = bi[j] >= 0 &&
                              (bi[threadIdx.x] < 0 || bc[j] < bc[threadIdx.x] ||
                               (bc[j] == bc[threadIdx.x] && bi[j] < bi[threadIdx.x]));
            if (take) {
                bc[threadIdx.x] = bc[j];
                bi[threadIdx.x] = bi[j];
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *best = bi[0];
}

// ---- batched form and serving rounds: one block per frame ----

__device__ void init_frame(const FrameDesc& f, HypState* st, int* active) {
    for (int m = threadIdx.x; m < f.M; m += blockDim.x) {
        HypState& s = st[f.hyp_offset + m];
        for (int i = 0; i < 12; ++i) s.T[i] = s.Tc[i] = f.T_cw[12 * m + i];
        for (int i = 0; i < 21; ++i) s.H[i] = 0.0;
        for (int i = 0; i < 6; ++i) s.g[i] = 0.0;
        s.cost = 0.0;
        s.lambda = 0.0;
        s.n_valid = 0;
        s.has_cand = 0;
        s.last_fail = 0;
        s.active = 1;
        s.status = PILOT_HYP_OK;
        active[f.hyp_offset + m] = m;
    }
}

// min_valid of one frame (block-wide; blockDim.x a multiple of 32, <= 1024)
__device__ void count_frame(const FrameDesc& f, double frac, double* min_valid) {
    __shared__ int part[32];
    int c = 0;
    for (int j = threadIdx.x; j < f.N; j += blockDim.x) c += f.valid ? (f.valid[j] != 0) : 1;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x < 32) {
        int v = (threadIdx.x < (blockDim.x >> 5)) ? part[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) *min_valid = frac * (double)v;
    }
    __syncthreads();
}

// Statuses, per-hypothesis outputs (at the global hypothesis index) and the argmin of
// one frame.  blockDim.x <= 1024, a power of two.
__device__ void finalize_frame(const FrameDesc& f, int fi, HypState* st, double mv,
                               unsigned char* res, int max_hyps) {
    const ResultLayout lay = ResultLayout::make(max_hyps);
    double* T = reinterpret_cast<double*>(res + lay.off_T);
    double* cost = reinterpret_cast<double*>(res + lay.off_cost);
    int* nv = reinterpret_cast<int*>(res + lay.off_nvalid);
    int* status = reinterpret_cast<int*>(res + lay.off_status);
    int* best = reinterpret_cast<int*>(res + lay.bytes);      // one int per frame after the block
    __shared__ double bc[1024];
    __shared__ int bi[1024];
    double my_c = 0.0;
    int my_i = -1;
    for (int m = threadIdx.x; m < f.M; m += blockDim.x) {
        const int g = f.hyp_offset + m;
        HypState& s = st[g];
        if (s.active) {
            bool finite = isfinite(s.cost);
            for (int i = 0; i < 12; ++i) finite = finite && isfinite(s.T[i]);
            int code;
            if (!finite) code = PILOT_HYP_NONFINITE;
            else if (s.n_valid < mv) code = PILOT_HYP_FEW_VALID;
            else if (s.last_fail) code = PILOT_HYP_NOT_PD;
            else code = PILOT_HYP_OK;
            s.status = code;
        }
        for (int i = 0; i < 12; ++i) T[12 * (size_t)g + i] = s.T[i];
        cost[g] = s.cost;
        nv[g] = s.n_valid;
        status[g] = s.status;
        if (s.status == PILOT_HYP_OK && (my_i < 0 || s.cost < my_c)) {
            my_c = s.cost;
            my_i = m;
        }
    }
    bc[threadIdx.x] = my_c;
    bi[threadIdx.x] = my_i;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) {
            const int j = threadIdx.x + k;
            const bool take = bi[j] >= 0 &&
                              (bi[threadIdx.x] < 0 || bc[j] < bc[threadIdx.x] ||
                               (bc[j] == bc[threadIdx.x] && bi[j] < bi[threadIdx.x]));
            if (take) {
                bc[threadIdx.x] = bc[j];
                bi[threadIdx.x] = bi[j];
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) best[fi] = bi[0];
}

__global__ void batch_init_kernel(const BatchHeader* hdr, const FrameDesc* frames, HypState* st,
                                  int* active) {
    if ((int)blockIdx.x >= hdr->n_frames) return;
    init_frame(frames[blockIdx.x], st, active);
}

__global__ void batch_count_valid_kernel(const BatchHeader* hdr, const FrameDesc* frames, double frac,
                                         double* min_valid) {
    if ((int)blockIdx.x >= hdr->n_frames) return;
    count_frame(frames[blockIdx.x], frac, min_valid + blockIdx.x);
}

// Batched form, top-K after a level: blockIdx.x is the frame, blockIdx.y a block of 256 of
// its listed hypotheses (frames whose count is at most K keep all of them).
__global__ void batch_rank_kernel(const BatchHeader* hdr, const FrameDesc* frames, HypState* st,
                                  const int* active, const int* n_active, int K, const double* min_valid) {
    const int fi = blockIdx.x;
    if (fi >= hdr->n_frames) return;
    const int n = n_active[fi];
    if (K <= 0 || K >= n || (int)blockIdx.y * kRankThreads >= n) return;
    const FrameDesc& f = frames[fi];
    rank_mark(st + f.hyp_offset, active + f.hyp_offset, n, K, min_valid[fi], blockIdx.y * kRankThreads);
}

// Batched form: each pruned frame's active list compacted in place.
__global__ void batch_compact_kernel(const BatchHeader* hdr, const FrameDesc* frames, const HypState* st,
                                     int* active, const int* n_active, int K) {
    const int fi = blockIdx.x;
    if (fi >= hdr->n_frames) return;
    const int n = n_active[fi];
    if (K <= 0 || K >= n) return;
    const FrameDesc& f = frames[fi];
    compact_active(st + f.hyp_offset, active + f.hyp_offset, active + f.hyp_offset, n);
}

__global__ void batch_finalize_kernel(const BatchHeader* hdr, const FrameDesc* frames, HypState* st,
                                      const double* min_valid, unsigned char* res, int max_hyps) {
    const int fi = blockIdx.x;
    if (fi >= hdr->n_frames) return;
    finalize_frame(frames[fi], fi, st, min_valid[fi], res, max_hyps);
}

__global__ void round_prepare_kernel(const BatchHeader* hdr, const FrameDesc* frames, HypState* st,
                                     int* active, double frac, double* min_valid) {
    const int fi = blockIdx.x;
    if (fi >= hdr->n_frames) return;
    const FrameDesc& f = frames[fi];
    if (!(f.flags & kFlagInit)) return;
    init_frame(f, st, active);
    count_frame(f, frac, min_valid + fi);
}

// Serving round, top-K of the frames that finished a pruning level (as batch_rank_kernel).
__global__ void round_rank_kernel(const BatchHeader* hdr, const FrameDesc* frames, HypState* st,
                                  const int* active, const double* min_valid) {
    const int fi = blockIdx.x;
    if (fi >= hdr->n_frames) return;
    const FrameDesc& f = frames[fi];
    if (!(f.flags & kFlagPrune) || (int)blockIdx.y * kRankThreads >= f.n_active) return;
    rank_mark(st + f.hyp_offset, active + f.hyp_offset, f.n_active, f.keep, min_valid[fi], blockIdx.y * kRankThreads);
}

__global__ void round_finish_kernel(const BatchHeader* hdr, const FrameDesc* frames, HypState* st,
                                    int* active, const double* min_valid, unsigned char* res,
                                    int max_hyps) {
    const int fi = blockIdx.x;
    if (fi >= hdr->n_frames) return;
    const FrameDesc& f = frames[fi];
    if (f.flags & kFlagPrune)
        compact_active(st + f.hyp_offset, active + f.hyp_offset, active + f.hyp_offset, f.n_active);
    if (f.flags & kFlagFinalize) finalize_frame(f, fi, st, min_valid[fi], res, max_hyps);
}

// Serving round with several levels: after a level's finish, every listed frame moves on to
// its next level on the device (what the host does between one-level rounds): a frame that
// finished level 0 (finalised), or that has used its quota of levels for the round, drops out
// with no jobs; the others take their top-K, step to the next finer level and get that
// level's flags; the job and item tables are rebuilt in list order.  One thread: at most
// max_slots frames.
__global__ void round_advance_kernel(const BatchHeader* hdr, FrameDesc* frames, const int* fr_list, int* fr_item,
                                     int* fr_job, LevelKeep keep, int tile, int tpi) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const int nl = hdr->n_listed[0];
    if (hdr->tiles_per_item > 0) tpi = hdr->tiles_per_item;   // the round's own work-item size
    fr_item[0] = 0;
    fr_job[0] = 0;
    for (int i = 0; i < nl; ++i) {
        FrameDesc& f = frames[fr_list[i]];
        f.quota -= 1;
        if (f.n_active > 0 && f.quota <= 0) {
            // this frame's levels for the round are done: it idles until the next round (the
            // host carries its level and active count over)
            f.n_active = 0;
            f.flags = 0;
        } else if (f.n_active > 0) {
            if (f.level == 0) {
                f.n_active = 0;
                f.flags = 0;
            } else {
                if (f.flags & kFlagPrune) f.n_active = f.keep;
                f.level -= 1;
                const int K = keep.k[f.level];
                f.keep = K;
                f.flags = ((f.level > 0 && K > 0 && K < f.n_active) ? kFlagPrune : 0) | (f.level == 0 ? kFlagFinalize : 0);
            }
        } else {
            f.flags = 0;
        }
        fr_job[i + 1] = fr_job[i] + f.n_active;
        fr_item[i + 1] = fr_item[i] + frame_items(f.n_active, f.N, tile, tpi);
    }
}

}  // namespace

cudaError_t launch_round_advance(const BatchHeader* hdr, FrameDesc* frames, const int* fr_list, int* fr_item,
                                 int* fr_job, const LevelKeep& keep, int tile, int tpi, cudaStream_t s) {
    round_advance_kernel<<<1, 32, 0, s>>>(hdr, frames, fr_list, fr_item, fr_job, keep, tile, tpi);
    return cudaGetLastError();
}

cudaError_t launch_batch_init(const BatchHeader* hdr, const FrameDesc* frames, HypState* st,
                              int* active, int max_frames, cudaStream_t s) {
    batch_init_kernel<<<max_frames, 128, 0, s>>>(hdr, frames, st, active);
    return cudaGetLastError();
}

cudaError_t launch_batch_count_valid(const BatchHeader* hdr, const FrameDesc* frames, double frac,
                                     double* min_valid, int max_frames, cudaStream_t s) {
    batch_count_valid_kernel<<<max_frames, 1024, 0, s>>>(hdr, frames, frac, min_valid);
    return cudaGetLastError();
}

cudaError_t launch_batch_prune(const BatchHeader* hdr, const FrameDesc* frames, HypState* st,
                               int* active, const int* n_active, int keep, const double* min_valid,
                               int max_frames, int max_frame_hyps, cudaStream_t s) {
    const dim3 grid(max_frames, (max_frame_hyps + kRankThreads - 1) / kRankThreads);
    batch_rank_kernel<<<grid, kRankThreads, 0, s>>>(hdr, frames, st, active, n_active, keep, min_valid);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    batch_compact_kernel<<<max_frames, 1024, 0, s>>>(hdr, frames, st, active, n_active, keep);
    return cudaGetLastError();
}

cudaError_t launch_batch_finalize(const BatchHeader* hdr, const FrameDesc* frames, HypState* st,
                                  const double* min_valid, unsigned char* result, int max_hyps,
                                  int max_frames, cudaStream_t s) {
    batch_finalize_kernel<<<max_frames, 1024, 0, s>>>(hdr, frames, st, min_valid, result, max_hyps);
    return cudaGetLastError();
}

cudaError_t launch_round_prepare(const BatchHeader* hdr, const FrameDesc* frames, HypState* st,
                                 int* active, double frac, double* min_valid, int max_frames,
                                 cudaStream_t s) {
    round_prepare_kernel<<<max_frames, 1024, 0, s>>>(hdr, frames, st, active, frac, min_valid);
    return cudaGetLastError();
}

cudaError_t launch_round_finish(const BatchHeader* hdr, const FrameDesc* frames, HypState* st,
                                int* active, const double* min_valid, unsigned char* result,
                                int max_hyps, int max_frames, int max_frame_hyps, cudaStream_t s) {
    const dim3 grid(max_frames, (max_frame_hyps + kRankThreads - 1) / kRankThreads);
    round_rank_kernel<<<grid, kRankThreads, 0, s>>>(hdr, frames, st, active, min_valid);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    round_finish_kernel<<<max_frames, 1024, 0, s>>>(hdr, frames, st, active, min_valid, result, max_hyps);
    return cudaGetLastError();
}

cudaError_t launch_epilogue(const EpilogueParams& p, const double* min_valid, cudaStream_t s) {
    if (p.n_active <= 0) return cudaSuccess;
    epilogue_kernel<<<p.n_active, 256, 0, s>>>(p, min_valid);
    return cudaGetLastError();
}

cudaError_t launch_hyp_init(HypState* st, const double* T_cw, int* active_idx, int M,
                            cudaStream_t s) {
    if (M <= 0) return cudaSuccess;
    hyp_init_kernel<<<(M + 127) / 128, 128, 0, s>>>(st, T_cw, active_idx, M);
    return cudaGetLastError();
}

cudaError_t launch_set_poses(HypState* st, float* pose32, const double* T_cw, int* active_idx,
                             int M, cudaStream_t s) {
    if (M <= 0) return cudaSuccess;
    set_poses_kernel<<<(M + 127) / 128, 128, 0, s>>>(st, pose32, T_cw, active_idx, M);
    return cudaGetLastError();
}

cudaError_t launch_level_init(HypState* st, float* pose32, const int* active_idx, int n_active,
                              double lambda0, cudaStream_t s) {
    if (n_active <= 0) return cudaSuccess;
    level_init_kernel<<<(n_active + 127) / 128, 128, 0, s>>>(st, pose32, active_idx, n_active, lambda0);
    return cudaGetLastError();
}

cudaError_t launch_prune(HypState* st, const int* active_in, int* active_out, int n_active,
                         int keep, const double* min_valid, cudaStream_t s) {
    if (n_active <= 0) return cudaSuccess;
    prune_rank_kernel<<<(n_active + kRankThreads - 1) / kRankThreads, kRankThreads, 0, s>>>(st, active_in, n_active,
                                                                                            keep, min_valid);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    prune_compact_kernel<<<1, 1024, 0, s>>>(st, active_in, active_out, n_active);
    return cudaGetLastError();
}

cudaError_t launch_count_valid(const uint8_t* valid, int N, double frac, double* min_valid,
                               cudaStream_t s) {
    count_valid_kernel<<<1, 1024, 0, s>>>(valid, N, frac, min_valid);
    return cudaGetLastError();
}

cudaError_t launch_finalize(HypState* st, int M, const double* min_valid, unsigned char* result,
                            ResultLayout lay, cudaStream_t s) {
    finalize_kernel<<<1, 1024, 0, s>>>(st, M, min_valid, result, lay);
    return cudaGetLastError();
}

}  // namespace pilot
