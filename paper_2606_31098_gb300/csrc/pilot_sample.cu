// Geo-anchor sampling on the GPU (Supp. "TDOM/DSM Reference Crop": the valid geo-anchors
// the solver uses are sampled from the reference crop).
//
// Pixel j of the crop gets the key (upper 32 bits of the (j+1)-th output of the SplitMix64
// generator started at `seed`) * 2^32 + j -- unique per pixel, uniformly ordered over the
// pixels by the generator -- and the n_select valid pixels with the smallest keys are
// taken: a uniform draw without replacement, decided in integer arithmetic only.
// SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
// OOPSLA 2014): state += 0x9E3779B97F4A7C15, then
//   z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9; z = (z ^ (z >> 27)) * 0x94D049BB133111EB;
//   output z ^ (z >> 31).
//
// One CTA of 1024 threads: a radix select finds the n_select-th smallest key among the
// valid pixels (8 passes of 8 bits, a 256-bin shared-memory histogram each), then an
// exclusive scan over contiguous per-thread chunks lists the selected pixels in increasing
// pixel order and gathers their geo-anchor coordinates.
#include <cuda_runtime.h>
#include <stdint.h>

#include "pilot_internal.cuh"

namespace pilot {
namespace {

constexpr int kSampleThreads = 1024;

__device__ __forceinline__ unsigned long long splitmix64_output(unsigned long long seed, unsigned long long j) {
    unsigned long long z = seed + (j + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ unsigned long long sample_key(unsigned long long seed, int j) {
    return ((splitmix64_output(seed, (unsigned long long)j) >> 32) << 32) | (unsigned long long)(unsigned)j;
}

__global__ void __launch_bounds__(kSampleThreads)
sample_anchors_kernel(const uint8_t* valid, const float* points, int n, int k, unsigned long long seed,
                      int* out_idx, float* out_pts, int* out_count) {
    __shared__ unsigned hist[256];
    __shared__ unsigned long long s_prefix;
    __shared__ unsigned s_rank;
    __shared__ unsigned s_warp[kSampleThreads / 32];
    __shared__ unsigned s_nvalid;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_nvalid = 0;
    __syncthreads();
    unsigned mine = 0;
    for (int j = tid; j < n; j += kSampleThreads) mine += valid[j] ? 1u : 0u;
    atomicAdd(&s_nvalid, mine);
    __syncthreads();
    const unsigned nvalid = s_nvalid;
    const unsigned take = (unsigned)k < nvalid ? (unsigned)k : nvalid;

    // the take-th smallest key (all valid pixels when take = nvalid)
    unsigned long long kth = ~0ull;
    if (take > 0 && take < nvalid) {
        unsigned long long prefix = 0, mask = 0;
        unsigned rank = take;                           // 1-based rank within the prefix
        for (int shift = 56; shift >= 0; shift -= 8) {
            for (int b = tid; b < 256; b += kSampleThreads) hist[b] = 0;
            __syncthreads();
            for (int j = tid; j < n; j += kSampleThreads) {
                if (!valid[j]) continue;
                const unsigned long long key = sample_key(seed, j);
                if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255ull], 1u);
            }
            __syncthreads();
            if (tid == 0) {
                unsigned cum = 0;
                int d = 0;
                for (; d < 255; ++d) {
                    if (cum + hist[d] >= rank) break;
                    cum += hist[d];
                }
                s_prefix = prefix | ((unsigned long long)d << shift);
                s_rank = rank - cum;
            }
            __syncthreads();
            prefix = s_prefix;
            rank = s_rank;
            mask |= 0xFFull << shift;
            __syncthreads();
        }
        kth = prefix;
    }

    // selected pixels in increasing order: contiguous chunks per thread, exclusive scan
    const int chunk = (n + kSampleThreads - 1) / kSampleThreads;
    const int lo = min(n, tid * chunk), hi = min(n, lo + chunk);
    unsigned cnt = 0;
    if (take > 0)
        for (int j = lo; j < hi; ++j) cnt += (valid[j] && sample_key(seed, j) <= kth) ? 1u : 0u;
    unsigned incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        unsigned w = lane < kSampleThreads / 32 ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kSampleThreads / 32) s_warp[lane] = w;    // inclusive over warps
    }
    __syncthreads();
    unsigned pos = (warp > 0 ? s_warp[warp - 1] : 0u) + incl - cnt;
    if (take > 0)
        for (int j = lo; j < hi && pos < take; ++j) {
            if (!(valid[j] && sample_key(seed, j) <= kth)) continue;
            out_idx[pos] = j;
            if (out_pts) {
                out_pts[pos] = points[j];
                out_pts[k + pos] = points[(size_t)n + j];
                out_pts[2 * (size_t)k + pos] = points[2 * (size_t)n + j];
            }
            ++pos;
        }
    if (tid == 0) *out_count = (int)take;
}

}  // namespace
}  // namespace pilot

using namespace pilot;

extern "C" pilot_status pilot_sample_anchors(const unsigned char* valid, const float* points, int n_pixels, int n_select,
                                             unsigned long long seed, int* out_idx, float* out_points,
                                             int* out_count, void* stream) {
    if (n_pixels < 0 || n_select < 0) {
        record_error("pilot_sample_anchors: n_pixels and n_select must be >= 0");
        return PILOT_EINVAL;
    }
    if (!out_count || (n_pixels > 0 && !valid) || (n_select > 0 && !out_idx) || (out_points && !points)) {
        record_error("pilot_sample_anchors: valid, out_idx and out_count are required (points with out_points)");
        return PILOT_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    sample_anchors_kernel<<<1, kSampleThreads, 0, s>>>(valid, points, n_pixels, n_select, seed, out_idx,
                                                       out_points, out_count);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        record_error(cudaGetErrorString(e));
        return PILOT_ECUDA;
    }
    return PILOT_OK;
}
