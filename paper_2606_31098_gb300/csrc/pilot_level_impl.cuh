// Batched form's persistent level kernel (one cooperative launch per pyramid level for a
// whole batch of frames, or for a serving round).  It reuses the build pass' anchor loop
// (accumulate_anchors, cta_reduce) and the FP64 step (lm_update), in the plain form's
// summation order, so a frame's results are bitwise those of its plain solve.
#pragma once

#include "pilot_build_impl.cuh"

namespace pilot {

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier of the persistent level kernel (cooperative launch: all CTAs resident).
// sync[1] counts arrivals over all generations, sync[2] is the number of completed
// generations; a generation completes when gridDim.x + extra CTAs have arrived (extra is 0
// except in the failure self-test, where it makes the barrier impossible).  The wait is
// bounded in time: past timeout_ns, or as soon as another CTA has given up, the error word
// is set, false is returned and the kernel returns; the host reports the error.
__device__ __forceinline__ bool grid_sync(unsigned long long* sync, unsigned* error, unsigned& gen,
                                          unsigned long long timeout_ns, int extra) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        int ok = 1;
        const unsigned long long target = (unsigned long long)(gen + 1) * (gridDim.x + (unsigned)extra);
        if (atomicAdd(sync + 1, 1ull) + 1ull == target) {
            atomicExch(sync + 2, (unsigned long long)(gen + 1));
        } else {
            const unsigned long long t0 = global_ns();
            while (__ldcg(sync + 2) < (unsigned long long)(gen + 1)) {
                if (__ldcg(error) != 0u) {
                    ok = 0;
                    break;
                }
                if (global_ns() - t0 > timeout_ns) {
                    atomicExch(error, 1u);
                    ok = 0;
                    break;
                }
                __nanosleep(256);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    ++gen;
    return s_ok != 0;
}

// Batched and served forms: one persistent (cooperative) launch per level for a whole batch
// of frames, running the level's LM iterations over all jobs (a job = one hypothesis of one
// frame).  The CTAs claim work items (runs of up to tiles_per_item consecutive anchor tiles of
// one tile of kHypTile jobs of a frame, the hypotheses a plain form's CTA holds) from one
// counter and write each tile's FP32 records exactly as build_fused_kernel does (same thread
// mapping, same sums); each job's FP64 step runs on one warp (all lanes), on the tile records
// summed in the plain form's 8-chain FP64 order, and writes the job's next candidate.  A
// frame's result is therefore bitwise the one its plain solve gives, whatever else is in the
// batch.  FLOW selects the schedule: without grid barriers (the items of all iterations in
// iteration-major order, per-job-tile flags) or lockstep phases (below).  Tile t of job
// kHypTile p + h, whose job tile's first item is q, keeps its record at
// partial[(q tiles_per_item + t) kHypTile + h].
// One job's FP64 step in the schedule without grid barriers: its tile records (slot h of the
// job tile whose first item is `first`) summed in the plain form's 8-chain FP64 order, then
// lm_update; all 32 lanes of one warp.  Not inlined: the item loop that calls it keeps its own
// registers for the anchor loop.
static __device__ __noinline__ void flow_step(const LevelArgs& a, int job, int first, int frame, int level, int k,
                                              int h, int tpi, double* E, double* W) {
    constexpr unsigned kEval = 0x80000000u;
    const int lane = threadIdx.x & 31;
    const FrameDesc* fd = a.frames + frame;
    const int iters = a.iters[level];
    const unsigned meta = __ldcg(a.job_meta + job);
    const int hyp = (int)(meta & ~kEval);
    if ((meta & kEval) != 0 && lane < kNumSums) {
        const int n_t = fd->N > 0 ? (fd->N + a.tile - 1) / a.tile : 1;
        const float* src = a.partial + ((size_t)first * tpi * kHypTile + h) * kAcc + lane;
        double sum = 0.0;
        for (int c = 0; c < 8; ++c) {
            double part = 0.0;
            for (int t = c; t < n_t; t += 8) part += (double)__ldcg(src + (size_t)t * kHypTile * kAcc);
            sum += part;
        }
        E[lane] = sum;
    }
    __syncwarp();
    HypState& st = a.state[hyp];
    lm_update(st, k == 0 ? kEpiInit : kEpiStep, k < iters, a.damping_mode, fd->prior, E, W, a.min_valid[frame],
              a.pose32 + 12 * (size_t)job, nullptr, lane);
    if (lane == 0) a.job_meta[job] = (unsigned)hyp | (st.has_cand ? kEval : 0u);
    __syncwarp();
}

template <pilot_dtype DT, int C, bool SCALED, bool CONF, bool FLOW>
__global__ void __launch_bounds__(kBuildThreads, 2)
level_persistent_kernel(const __grid_constant__ LevelArgs a) {
    constexpr int kWarps = kBuildThreads / 32;
    constexpr unsigned kEval = 0x80000000u;          // job_meta: "has a pose to evaluate" bit
    __shared__ float red[kWarps][kHypTile][kAcc];
    __shared__ double E[kWarps][kAcc];
    __shared__ double Wsh[kWarps][128];         // FP64 step scratch, one block per warp
    __shared__ float pose[kHypTile][12];
    __shared__ unsigned s_meta[kHypTile];
    // the claimed work item: its frame, first record slot, tile range and job tile (s_item < 0:
    // none left in this phase)
    __shared__ long long s_item;
    __shared__ int s_frame, s_level, s_job, s_njobs, s_first, s_t0, s_t1, s_run;
    // CTA-uniform loop state, kept here and read where it is used: held in registers it would
    // live through the anchor loop and push the loop's own values into local memory
    __shared__ int s_nfr, s_items, s_jobs, s_IA, s_JA, s_k, s_ipj, s_last;
    __shared__ unsigned long long s_base;
    // frame tables, staged when the launch lists few frames
    __shared__ int s_fitem[kSmemFrames + 1], s_fjob[kSmemFrames + 1], s_flist[kSmemFrames], s_fipj[kSmemFrames];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // work-item size: the tables' own (served rounds choose it per round) or the launch's
    const int tpi = a.header->tiles_per_item > 0 ? a.header->tiles_per_item : a.tiles_per_item;
    if (tid == 0) s_nfr = a.header->n_listed[a.list_index];
    __syncthreads();
    if (s_nfr <= kSmemFrames)
        for (int i = tid; i <= s_nfr; i += kBuildThreads) {
            s_fitem[i] = a.fr_item[i];
            s_fjob[i] = a.fr_job[i];
            if (i < s_nfr) {
                s_flist[i] = a.fr_list[i];
                s_fipj[i] = items_per_job(a.frames[s_flist[i]].N, a.tile, tpi);
            }
        }
    __syncthreads();
    auto staged = [&]() { return s_nfr <= kSmemFrames; };
    auto fitem = [&](int i) { return staged() ? s_fitem[i] : a.fr_item[i]; };
    auto fjob = [&](int i) { return staged() ? s_fjob[i] : a.fr_job[i]; };
    auto flist = [&](int i) { return staged() ? s_flist[i] : a.fr_list[i]; };
    auto fipj = [&](int i) { return staged() ? s_fipj[i] : items_per_job(a.frames[a.fr_list[i]].N, a.tile, tpi); };
    // listed frame holding x: last i < n_fr with table(i) <= x (empty frames are skipped)
    auto find = [&](bool items, long long x) {
        int lo = 0, hi = s_nfr - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((items ? fitem(mid) : fjob(mid)) <= x) lo = mid;
            else hi = mid - 1;
        }
        return lo;
    };
    if (tid == 0) {
        s_items = fitem(s_nfr);
        s_jobs = fjob(s_nfr);
    }
    __syncthreads();
    unsigned gen = 0;
    // level start of every job: its hypothesis, LM state and FP32 start pose (pose32 and
    // job_meta are indexed by job within this launch).  Job j's state is only ever read and
    // written by global warp j (mod the warp count; lane 0 here, all lanes in the steps below),
    // so one SM's L1 sees all its accesses; other CTAs read pose32 and job_meta from L2.
    for (int job = blockIdx.x * kWarps + warp; job < s_jobs; job += gridDim.x * kWarps) {
        if (lane != 0) continue;
        const int i = find(false, job);
        const FrameDesc* fd = a.frames + flist(i);
        const int hyp = fd->hyp_offset + a.active[fd->hyp_offset + job - fjob(i)];
        HypState& st = a.state[hyp];
        st.lambda = a.lambda0;
        st.last_fail = 0;
        st.has_cand = 1;
        store_pose32(a.pose32 + 12 * (size_t)job, st.T);
        a.job_meta[job] = (unsigned)hyp | kEval;
    }
    // (in the schedule without barriers the failure self-test's extra applies to the flags)
    if (!grid_sync(a.sync, a.error, gen, a.barrier_timeout_ns, FLOW ? 0 : a.barrier_extra)) return;
    // Gather-heavy levels: the work items of every (iteration, job tile) are claimed in
    // iteration-major order from one counter and no grid barrier is taken.  The CTA that
    // completes a job tile's items of iteration k (counted in tile_done) runs the tile's FP64
    // steps, job h on warp h as the plain form's last CTA does, then publishes k + 1 in
    // tile_ready; an item of iteration k + 1 waits (bounded) until its tile has published k + 1.
    // Records and steps are the lockstep schedule's, so the results are the same.  Progress:
    // the earliest unfinished item in claim order never waits, since everything it depends on
    // was claimed before it and is finished or held by a CTA that is working, not waiting (all
    // CTAs are resident).  Items of iterations beyond a frame's count are claimed and skipped
    // and touch no flag.
    if constexpr (FLOW) {
        for (;;) {
            if (tid == 0) {
                const long long g = (long long)atomicAdd(a.sync, 1ull);
                const int n_items = s_items;
                s_item = g < (long long)(a.k_max + 1) * n_items ? g : -1;
                if (s_item >= 0) {
                    const int k = (int)(g / n_items);
                    const int local = (int)(g - (long long)k * n_items);
                    const int i = find(true, local);
                    const int ipj = fipj(i);
                    const int loc = local - fitem(i);
                    const int jt = loc / ipj;      // job tile within the frame
                    const FrameDesc* fd = a.frames + flist(i);
                    const int level = a.level >= 0 ? a.level : fd->level;
                    s_k = k;
                    s_run = k <= a.iters[level];
                    s_job = fjob(i) + kHypTile * jt;
                    s_njobs = min(kHypTile, fjob(i + 1) - s_job);
                    s_first = fitem(i) + jt * ipj;
                    s_ipj = ipj;
                    s_t0 = (loc - jt * ipj) * tpi;
                    s_t1 = min(s_t0 + tpi, fd->N > 0 ? (fd->N + a.tile - 1) / a.tile : 1);
                    s_frame = flist(i);
                    s_level = level;
                    if (s_run && k > 0) {
                        const unsigned long long t0 = global_ns();
                        while (ld_acquire_gpu(a.tile_ready + s_first) < (unsigned)(k + a.barrier_extra)) {
                            if (__ldcg(a.error) != 0u || global_ns() - t0 > a.barrier_timeout_ns) {
                                atomicExch(a.error, 1u);
                                s_item = -1;
                                break;
                            }
                            __nanosleep(128);
                        }
                    }
                }
            }
            __syncthreads();
            if (s_item < 0) return;
            if (!s_run) {
                __syncthreads();           // the shared item state is rewritten by the next claim
                continue;
            }
            if (tid < 12 * kHypTile) {
                const int h = tid / 12;
                pose[h][tid % 12] = __ldcg(a.pose32 + 12 * (size_t)(s_job + (h < s_njobs ? h : 0)) + tid % 12);
            }
            if (tid < kHypTile) s_meta[tid] = tid < s_njobs ? __ldcg(a.job_meta + s_job + tid) : 0u;
            __syncthreads();
            SlotPoses sp;
            bool any = false;
#pragma unroll
            for (int h = 0; h < kHypTile; ++h) {
                sp.p[h] = pose[h];
                sp.act[h] = (s_meta[h] & kEval) != 0;
                any = any || sp.act[h];
            }
            if (any) {
                const FrameDesc* fd = a.frames + s_frame;
                const int level = s_level;
                const LevelView v{fd->px, fd->py, fd->pz, fd->weight, fd->valid, fd->qry[level], fd->ref[level],
                                  fd->qscale[level], fd->rscale[level], fd->conf[level], fd->H[level], fd->W[level],
                                  fd->fx[level], fd->fy[level], fd->cx[level], fd->cy[level], a.huber};
                for (int t = s_t0; t < s_t1; ++t) {
                    float acc[kNumSums];
#pragma unroll
                    for (int i = 0; i < kNumSums; ++i) acc[i] = 0.f;
                    const int j0 = t * a.tile;
                    accumulate_anchors<DT, C, SCALED, CONF, kBuildThreads, DT == PILOT_F32, true>(
                        v, sp, j0, min(j0 + a.tile, fd->N), acc);
                    const float val = cta_reduce_slots<kBuildThreads, GroupShape<DT, C, SCALED>::APB>(acc, red);
                    if (tid < kHypTile * kAcc && tid / kAcc < s_njobs)
                        a.partial[(((size_t)s_first * tpi + t) * kHypTile + tid / kAcc) * kAcc + tid % kAcc] = val;
                    if (t + 1 < s_t1) __syncthreads();
                }
            }
            // count the item for its job tile; the CTA that completes the tile's iteration steps it
            __syncthreads();
            if (tid == 0) {
                __threadfence();
                const unsigned done = atomicAdd(a.tile_done + s_first, 1u) + 1u;
                s_last = done == (unsigned)(s_k + 1) * (unsigned)s_ipj;
                if (s_last) __threadfence();
            }
            __syncthreads();
            if (s_last) {
                if (warp < s_njobs)
                    flow_step(a, s_job + warp, s_first, s_frame, s_level, s_k, warp, tpi, E[warp], Wsh[warp]);
                __syncthreads();
                if (tid == 0) {
                    __threadfence();
                    st_release_gpu(a.tile_ready + s_first, (unsigned)s_k + 1u);
                }
            }
            __syncthreads();               // the shared item state is rewritten by the next claim
        }
    } else {
        // Lockstep phases (levels below kSplitUnits units per iteration, which the host does not
        // give the flags of the schedule above): phase 2k gathers every job's items of
        // iteration k, phase 2k + 1 steps every job (iteration k), a grid barrier ending each
        // phase.  The loop is written for two halves A = jobs [0, JA) with items [0, IA) and B
        // = the rest, stepping one half while the other gathers; here A is every job and B
        // none, so B's gathers and steps are empty.
        if (tid == 0) {
            s_IA = s_items;
            s_JA = s_jobs;
            // claims made before the current phase: a gathering phase takes one claim per item of
            // its half plus one unsuccessful claim per CTA
            s_base = 0;
        }
        __syncthreads();
        for (int ph = 0; ph <= 2 * a.k_max + 2; ++ph) {
            // FP64 steps of the half gathered in the previous phase: job j on global warp j (mod
            // the warp count), all 32 lanes
            if (ph >= 1) {
                const int k = (ph - 1) / 2;
                const int jlo = (ph & 1) ? 0 : s_JA, jhi = (ph & 1) ? s_JA : s_jobs;
                for (int job = jlo + blockIdx.x * kWarps + warp; job < jhi; job += gridDim.x * kWarps) {
                    const int i = find(false, job);
                    const int f = flist(i);
                    const FrameDesc* fd = a.frames + f;
                    const int level = a.level >= 0 ? a.level : fd->level;
                    const int iters = a.iters[level];
                    if (k > iters) continue;
                    const unsigned meta = __ldcg(a.job_meta + job);
                    const int hyp = (int)(meta & ~kEval);
                    const bool evaluated = (meta & kEval) != 0;
                    if (evaluated && lane < kNumSums) {
                        const int n_t = fd->N > 0 ? (fd->N + a.tile - 1) / a.tile : 1;
                        const int jl = job - fjob(i);
                        const int first = fitem(i) + (jl / kHypTile) * fipj(i);
                        const float* src = a.partial + ((size_t)first * tpi * kHypTile + jl % kHypTile) * kAcc + lane;
                        double sum = 0.0;
                        for (int c = 0; c < 8; ++c) {
                            double part = 0.0;
                            for (int t = c; t < n_t; t += 8) part += (double)__ldcg(src + (size_t)t * kHypTile * kAcc);
                            sum += part;
                        }
                        E[warp][lane] = sum;
                    }
                    __syncwarp();
                    HypState& st = a.state[hyp];
                    lm_update(st, k == 0 ? kEpiInit : kEpiStep, k < iters, a.damping_mode, fd->prior, E[warp], Wsh[warp],
                              a.min_valid[f], a.pose32 + 12 * (size_t)job, nullptr, lane);
                    if (lane == 0) a.job_meta[job] = (unsigned)hyp | (st.has_cand ? kEval : 0u);
                    __syncwarp();
                }
            }
            // gathers of one half at iteration k, its work items claimed one at a time
            if (ph <= 2 * a.k_max + 1) {
                for (;;) {
                    if (tid == 0) {
                        const int k = ph / 2;
                        const int ilo = (ph & 1) ? s_IA : 0, ihi = (ph & 1) ? s_items : s_IA;
                        long long item = ilo + (long long)(atomicAdd(a.sync, 1ull) - s_base);
                        if (item < ilo) {              // cannot happen: the counts above are exact
                            atomicExch(a.error, 1u);
                            item = ihi;
                        }
                        s_item = item < ihi ? item : -1;
                        if (item < ihi) {
                            const int i = find(true, item);
                            const int ipj = fipj(i);
                            const int local = (int)(item - fitem(i));
                            const int jt = local / ipj;      // job tile within the frame
                            const FrameDesc* fd = a.frames + flist(i);
                            const int level = a.level >= 0 ? a.level : fd->level;
                            s_job = fjob(i) + kHypTile * jt;
                            s_njobs = min(kHypTile, fjob(i + 1) - s_job);
                            s_first = fitem(i) + jt * ipj;
                            s_t0 = (local - jt * ipj) * tpi;
                            s_t1 = min(s_t0 + tpi, fd->N > 0 ? (fd->N + a.tile - 1) / a.tile : 1);
                            s_run = k <= a.iters[level];
                            s_frame = flist(i);
                            s_level = level;
                        }
                    }
                    __syncthreads();
                    if (s_item < 0) break;
                    if (tid < 12 * kHypTile) {
                        const int h = tid / 12;
                        pose[h][tid % 12] = __ldcg(a.pose32 + 12 * (size_t)(s_job + (h < s_njobs ? h : 0)) + tid % 12);
                    }
                    if (tid < kHypTile) s_meta[tid] = tid < s_njobs ? __ldcg(a.job_meta + s_job + tid) : 0u;
                    __syncthreads();
                    SlotPoses sp;
                    bool any = false;
    #pragma unroll
                    for (int h = 0; h < kHypTile; ++h) {
                        sp.p[h] = pose[h];
                        sp.act[h] = (s_meta[h] & kEval) != 0;
                        any = any || sp.act[h];
                    }
                    if (s_run && any) {
                        const FrameDesc* fd = a.frames + s_frame;
                        const int level = s_level;
                        const LevelView v{fd->px, fd->py, fd->pz, fd->weight, fd->valid, fd->qry[level], fd->ref[level],
                                          fd->qscale[level], fd->rscale[level], fd->conf[level], fd->H[level],
                                          fd->W[level], fd->fx[level], fd->fy[level], fd->cx[level], fd->cy[level],
                                          a.huber};
                        for (int t = s_t0; t < s_t1; ++t) {
                            float acc[kNumSums];
    #pragma unroll
                            for (int i = 0; i < kNumSums; ++i) acc[i] = 0.f;
                            const int j0 = t * a.tile;
                            // no anchor prefetch for the narrow types: the frame's level inputs
                            // already take the registers that kernel parameters cost the plain form
                            accumulate_anchors<DT, C, SCALED, CONF, kBuildThreads, DT == PILOT_F32>(
                                v, sp, j0, min(j0 + a.tile, fd->N), acc);
                            const float val = cta_reduce_slots<kBuildThreads, GroupShape<DT, C, SCALED>::APB>(acc, red);
                            if (tid < kHypTile * kAcc && tid / kAcc < s_njobs)
                                a.partial[(((size_t)s_first * tpi + t) * kHypTile + tid / kAcc) * kAcc + tid % kAcc] =
                                    val;
                            // the next tile's reduction reuses red: wait until every slot's sums are read
                            if (t + 1 < s_t1) __syncthreads();
                        }
                    }
                    __syncthreads();
                }
                if (tid == 0) s_base += (unsigned long long)((ph & 1) ? s_items - s_IA : s_IA) + gridDim.x;
            }
            if (!grid_sync(a.sync, a.error, gen, a.barrier_timeout_ns, a.barrier_extra)) return;
        }
    }
}

// With per-job-tile flags (a.tile_done) the schedule without grid barriers, else lockstep.
template <pilot_dtype DT, int C, bool SCALED, bool CONF>
cudaError_t launch_level_kernel(const cudaLaunchConfig_t& cfg, const LevelArgs& a) {
    return a.tile_done ? cudaLaunchKernelEx(&cfg, level_persistent_kernel<DT, C, SCALED, CONF, true>, a)
                       : cudaLaunchKernelEx(&cfg, level_persistent_kernel<DT, C, SCALED, CONF, false>, a);
}

template <pilot_dtype DT, int C>
cudaError_t launch_level_persistent_typed(int variant, const LevelArgs& a, int grid, cudaStream_t s) {
    // cooperative: every CTA resident at once (the lockstep schedule's grid barriers, the
    // other schedule's waits on flags set by other CTAs)
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kBuildThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    switch (variant) {
        case 0: return launch_level_kernel<DT, C, false, false>(cfg, a);
        case kVariantScaled: return launch_level_kernel<DT, C, true, false>(cfg, a);
        case kVariantConf: return launch_level_kernel<DT, C, false, true>(cfg, a);
        case kVariantScaled | kVariantConf: return launch_level_kernel<DT, C, true, true>(cfg, a);
        default: return cudaErrorInvalidValue;
    }
}

template <pilot_dtype DT>
cudaError_t launch_level_persistent_dtype(int C, int variant, const LevelArgs& a, int grid,
                                          cudaStream_t s) {
    switch (C) {
        case 4: return launch_level_persistent_typed<DT, 4>(variant, a, grid, s);
        case 8: return launch_level_persistent_typed<DT, 8>(variant, a, grid, s);
        case 16: return launch_level_persistent_typed<DT, 16>(variant, a, grid, s);
        case 32: return launch_level_persistent_typed<DT, 32>(variant, a, grid, s);
        case 64: return launch_level_persistent_typed<DT, 64>(variant, a, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

// CTAs per SM that both schedules' kernels can keep resident.
template <pilot_dtype DT, int C, bool SCALED, bool CONF>
cudaError_t occupancy_both(int* n) {
    int n0 = 0, n1 = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &n0, level_persistent_kernel<DT, C, SCALED, CONF, false>, kBuildThreads, 0);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n1, level_persistent_kernel<DT, C, SCALED, CONF, true>,
                                                          kBuildThreads, 0);
    *n = n0 < n1 ? n0 : n1;
    return e;
}

template <pilot_dtype DT, int C>
cudaError_t occupancy_typed(int variant, int* n) {
    switch (variant) {
        case 0: return occupancy_both<DT, C, false, false>(n);
        case kVariantScaled: return occupancy_both<DT, C, true, false>(n);
        case kVariantConf: return occupancy_both<DT, C, false, true>(n);
        case kVariantScaled | kVariantConf: return occupancy_both<DT, C, true, true>(n);
        default: return cudaErrorInvalidValue;
    }
}

template <pilot_dtype DT>
cudaError_t level_persistent_occupancy(int C, int variant, int* n) {
    switch (C) {
        case 4: return occupancy_typed<DT, 4>(variant, n);
        case 8: return occupancy_typed<DT, 8>(variant, n);
        case 16: return occupancy_typed<DT, 16>(variant, n);
        case 32: return occupancy_typed<DT, 32>(variant, n);
        case 64: return occupancy_typed<DT, 64>(variant, n);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pilot
