// Roofline probes: measured ceilings for the build pass on the device at hand.
//
//   pilot_probe_fma     FP32 FMA throughput: packed fma.rn.f32x2 on four independent
//                       chains per thread, every SM busy.
//   pilot_probe_gather  the build pass' access pattern without its arithmetic: 4-tap
//                       bilinear footprints of C contiguous channels at uniformly random
//                       pixels of an NHWC map, one 16-byte load per lane, lane groups
//                       covering a whole tap (so each load instruction touches one line per
//                       group).  Random pixels give no reuse between samples, so this is the
//                       L2-to-SM gather rate of the map's layout.
//   pilot_probe_gather_frame  the build pass' loads with the locality of a real frame:
//                       the same grid (anchor tiles x poses) and lane groups, anchors
//                       projected under real poses, 4 taps and the reference row of every
//                       (anchor, pose), no arithmetic: the gather ceiling of that pattern.
#include <cuda_runtime.h>

#include "pilot_internal.cuh"

namespace pilot {
namespace {

__device__ unsigned g_probe_sink;      // keeps the probes' results live

__device__ __forceinline__ unsigned mix32(unsigned x) {
    // a 32-bit integer hash (xorshift-multiply rounds) for uniform pixel choices
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

__global__ void fma_probe_kernel(int iters, float a, float b) {
    unsigned long long x[4];
    for (int i = 0; i < 4; ++i) {
        const float lo = threadIdx.x * 1e-3f + 2 * i, hi = lo + 1.0f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(x[i]) : "f"(lo), "f"(hi));
    }
    unsigned long long A, Bv;
    asm("mov.b64 %0, {%1, %1};" : "=l"(A) : "f"(a));
    asm("mov.b64 %0, {%1, %1};" : "=l"(Bv) : "f"(b));
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 4; ++i) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[i]) : "l"(A), "l"(Bv));
    }
    unsigned acc = 0;
    for (int i = 0; i < 4; ++i) acc ^= (unsigned)x[i] ^ (unsigned)(x[i] >> 32);
    if (acc == 0x9e3779b9u) atomicXor(&g_probe_sink, acc);
}

// LP lanes per sample, each reading 16 bytes of each of the 4 taps (a tap = 16 * LP bytes).
template <int LP>
__global__ void gather_probe_kernel(const uint4* map, int H, int W, long long samples, unsigned seed) {
    const int q = threadIdx.x & (LP - 1);
    const long long groups = (long long)gridDim.x * blockDim.x / LP;
    const long long g0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / LP;
    const size_t row = (size_t)W * LP;          // uint4s per map row
    unsigned acc = 0;
    for (long long sidx = g0; sidx < samples; sidx += 2 * groups) {
        // two samples per step for two footprints in flight
        unsigned v[2][4][4];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const long long si = sidx + u * groups;
            const unsigned h = mix32((unsigned)si ^ seed);
            const int r = (int)((h >> 16) % (unsigned)(H - 1)), c = (int)((h & 0xffffu) % (unsigned)(W - 1));
            const uint4* t00 = map + (size_t)r * row + (size_t)c * LP + q;
            const bool live = si < samples;
            const uint4 z = make_uint4(0, 0, 0, 0);
            const uint4 a = live ? __ldg(t00) : z, b = live ? __ldg(t00 + LP) : z;
            const uint4 cc = live ? __ldg(t00 + row) : z, d = live ? __ldg(t00 + row + LP) : z;
            v[u][0][0] = a.x ^ a.y; v[u][0][1] = a.z ^ a.w;
            v[u][1][0] = b.x ^ b.y; v[u][1][1] = b.z ^ b.w;
            v[u][2][0] = cc.x ^ cc.y; v[u][2][1] = cc.z ^ cc.w;
            v[u][3][0] = d.x ^ d.y; v[u][3][1] = d.z ^ d.w;
        }
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc ^= v[u][k][0] ^ v[u][k][1];
    }
    if (acc == 0x9e3779b9u) atomicXor(&g_probe_sink, acc);
}

// One vector of VB bytes (16 or 32, the build pass' load width) read through the read-only
// path, folded to one word.
template <int VB> struct ProbeVec;
template <> struct ProbeVec<16> {
    static __device__ __forceinline__ unsigned fold(const unsigned char* p) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
        return v.x ^ v.w;
    }
};
template <> struct ProbeVec<32> {
    static __device__ __forceinline__ unsigned fold(const unsigned char* p) {
        unsigned w[8];
        asm("ld.global.nc.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
            : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7])
            : "l"(p));
        return w[0] ^ w[7];
    }
};

// The build pass' own access pattern without its arithmetic: grid (anchor tiles x tiles of
// kHypTile poses), 256 threads, the build pass' lane layout (LP lanes per tap; a group takes
// APB anchors under HG poses at a time, NS groups over the same anchors): each lane projects
// one (anchor, pose) record and publishes the tap offset to its group (shuffles), then the
// group reads the reference row of each of its anchors once and the 4 taps of each record,
// NV loads of VB bytes per lane and tap (row 0 for a record that is not visible, as the build
// pass does).  Two batches are in flight per step.  Loaded words are XOR-folded.
template <int LP, int NV, int VB>
__global__ void __launch_bounds__(256) frame_gather_probe_kernel(const float* pts, int N, const unsigned char* map,
                                                                 const unsigned char* ref, int H, int W, float fx,
                                                                 float fy, float cx, float cy,
                                                                 const float* poses, int M, int tile) {
    using PV = ProbeVec<VB>;
    constexpr int HG = LP < kHypTile ? LP : kHypTile, NS = kHypTile / HG, APB = LP / HG;
    constexpr int V = LP * NV;                 // vectors per tap (= per reference row)
    constexpr int ASTEP = 256 / (LP * NS) * APB;
    const int lane = threadIdx.x & 31, q = lane & (LP - 1), src0 = lane & ~(LP - 1);
    const int slot = (lane / APB) % kHypTile, qa = q % APB;
    const unsigned gmask = LP > 1 ? (((1u << LP) - 1u) << src0) : (1u << lane);
    const float* P = poses + 12 * min(kHypTile * (int)blockIdx.y + slot, M - 1);
    const float R00 = P[0], R01 = P[1], R02 = P[2], T0 = P[3], R10 = P[4], R11 = P[5], R12 = P[6], T1 = P[7];
    const float R20 = P[8], R21 = P[9], R22 = P[10], T2 = P[11];
    const int j0 = blockIdx.x * tile, j1 = min(j0 + tile, N);
    const size_t row = (size_t)W * V * VB;     // bytes per map row
    unsigned acc = 0;
    // tap offset of anchor j under this lane's pose (-1: not visible)
    auto project = [&](int j) {
        int off = -1;
        if (j < j1) {
            const float X = __ldg(pts + j), Y = __ldg(pts + N + j), Z = __ldg(pts + 2 * N + j);
            const float x = fmaf(R00, X, fmaf(R01, Y, fmaf(R02, Z, T0)));
            const float y = fmaf(R10, X, fmaf(R11, Y, fmaf(R12, Z, T1)));
            const float z = fmaf(R20, X, fmaf(R21, Y, fmaf(R22, Z, T2)));
            if (z > kZNear) {
                const float iz = 1.0f / z;
                const float xs = fmaf(fx * x, iz, cx) - 0.5f, ys = fmaf(fy * y, iz, cy) - 0.5f;
                if (xs >= 0.f && xs <= (float)(W - 1) && ys >= 0.f && ys <= (float)(H - 1))
                    off = min((int)ys, H - 2) * W + min((int)xs, W - 2);
            }
        }
        return off;
    };
    for (int jb = j0 + (int)(threadIdx.x / (LP * NS)) * APB; jb < j1; jb += 2 * ASTEP) {
        const int offA = project(jb + qa), offB = project(jb + ASTEP + qa);
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int off = b ? offB : offA, jbb = jb + ASTEP * b;
#pragma unroll
            for (int a = 0; a < APB; ++a) {
                const unsigned char* fr = ref + (size_t)(jbb + a < j1 ? jbb + a : j0) * V * VB;
#pragma unroll
                for (int k = 0; k < NV; ++k) acc ^= PV::fold(fr + (size_t)(q + k * LP) * VB);
            }
#pragma unroll
            for (int i = 0; i < LP; ++i) {
                const int oi = LP > 1 ? __shfl_sync(gmask, off, src0 + i) : off;
                const unsigned char* t00 = map + (size_t)(oi >= 0 ? oi : 0) * V * VB;
#pragma unroll
                for (int k = 0; k < NV; ++k) {
                    const size_t c = (size_t)(q + k * LP) * VB;
                    acc ^= PV::fold(t00 + c) ^ PV::fold(t00 + V * VB + c) ^ PV::fold(t00 + row + c) ^
                           PV::fold(t00 + row + V * VB + c);
                }
            }
        }
    }
    if (acc == 0x9e3779b9u) atomicXor(&g_probe_sink, acc);
}

template <int LP>
cudaError_t launch_gather(const void* map, int H, int W, long long samples, unsigned seed, int grid,
                          cudaStream_t s) {
    gather_probe_kernel<LP><<<grid, 256, 0, s>>>(static_cast<const uint4*>(map), H, W, samples, seed);
    return cudaGetLastError();
}

// Device time of one launch after a warm-up one.
template <typename F>
cudaError_t time_launch(F launch, cudaStream_t s, float* ms) {
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e;
}

pilot_status probe_fail(pilot_status st, const char* m) {
    record_error(m);
    return st;
}

int sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return sms;
}

}  // namespace
}  // namespace pilot

using namespace pilot;

extern "C" {

pilot_status pilot_probe_fma(double* tflops, void* stream) {
    if (!tflops) return probe_fail(PILOT_EINVAL, "tflops is NULL");
    const int sms = sm_count();
    if (sms <= 0) return probe_fail(PILOT_ECUDA, "no CUDA device");
    const int grid = sms * 8, threads = 256, iters = 1 << 14;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float ms = 0.f;
    const cudaError_t e = time_launch(
        [&]() {
            fma_probe_kernel<<<grid, threads, 0, s>>>(iters, 0.999f, 0.001f);
            return cudaGetLastError();
        },
        s, &ms);
    if (e != cudaSuccess) return probe_fail(PILOT_ECUDA, cudaGetErrorString(e));
    // 4 packed FMAs = 8 FMAs = 16 flops per thread and iteration
    *tflops = 16.0 * iters * (double)grid * threads / (ms * 1e-3) / 1e12;
    return PILOT_OK;
}

pilot_status pilot_probe_gather(const void* map, int H, int W, int C, pilot_dtype dtype, long long samples,
                                double* gbps, void* stream) {
    if (!map || !gbps) return probe_fail(PILOT_EINVAL, "map or gbps is NULL");
    if (H < 2 || W < 2 || H > 65535 || W > 65535) return probe_fail(PILOT_EINVAL, "map must be 2..65535 on each side");
    if (samples < 1) return probe_fail(PILOT_EINVAL, "samples must be positive");
    if (reinterpret_cast<uintptr_t>(map) % 16) return probe_fail(PILOT_EINVAL, "map must be 16-byte aligned");
    const int elem = dtype == PILOT_F32 ? 4 : (dtype == PILOT_FP8E4M3 ? 1 : 2);
    const int tap = C * elem;
    if (tap % 16 || tap / 16 < 1 || tap / 16 > 8 || (tap / 16 & (tap / 16 - 1)))
        return probe_fail(PILOT_EINVAL, "a tap (C x element size) must be 16, 32, 64 or 128 bytes");
    const int sms = sm_count();
    if (sms <= 0) return probe_fail(PILOT_ECUDA, "no CUDA device");
    const int grid = sms * 8;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float ms = 0.f;
    cudaError_t e = cudaSuccess;
    auto go = [&]() {
        switch (tap / 16) {
            case 1: return launch_gather<1>(map, H, W, samples, 0x1234567u, grid, s);
            case 2: return launch_gather<2>(map, H, W, samples, 0x1234567u, grid, s);
            case 4: return launch_gather<4>(map, H, W, samples, 0x1234567u, grid, s);
            default: return launch_gather<8>(map, H, W, samples, 0x1234567u, grid, s);
        }
    };
    e = time_launch(go, s, &ms);
    if (e != cudaSuccess) return probe_fail(PILOT_ECUDA, cudaGetErrorString(e));
    *gbps = (double)samples * 4.0 * tap / (ms * 1e-3) / 1e9;
    return PILOT_OK;
}

pilot_status pilot_probe_gather_frame(const float* points, int N, const void* map, const void* ref, int H, int W,
                                      int C, pilot_dtype dtype, double fx, double fy, double cx, double cy,
                                      const float* poses32, int M, int tile, double* units_per_s, void* stream) {
    if (!points || !map || !ref || !poses32 || !units_per_s) return probe_fail(PILOT_EINVAL, "NULL argument");
    if (N < 1 || M < 1 || M > 65535 || tile < 1) return probe_fail(PILOT_EINVAL, "N, M and tile must be positive, M <= 65535");
    if (H < 2 || W < 2) return probe_fail(PILOT_EINVAL, "map must be at least 2 x 2");
    const int elem = dtype == PILOT_F32 ? 4 : (dtype == PILOT_FP8E4M3 ? 1 : 2);
    // the build pass' load width for maps without per-channel scales: 32 bytes for FP32 and
    // 16-bit taps of 32 bytes or more, else 16
    const int vb = (dtype != PILOT_FP8E4M3 && C * elem >= 32) ? 32 : 16;
    if (reinterpret_cast<uintptr_t>(map) % vb || reinterpret_cast<uintptr_t>(ref) % vb)
        return probe_fail(PILOT_EINVAL, "map and ref must be aligned to the load width (16 or 32 bytes)");
    const int vec = C * elem / vb;               // vectors per tap
    if (C * elem % 16 || vec < 1 || vec > 16 || (vec & (vec - 1)))
        return probe_fail(PILOT_EINVAL, "a tap (C x element size) must be 16 .. 256 bytes, a power of two");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const dim3 grid((N + tile - 1) / tile, (M + kHypTile - 1) / kHypTile);
    const float f[4] = {(float)fx, (float)fy, (float)cx, (float)cy};
    const unsigned char* mp = static_cast<const unsigned char*>(map);
    const unsigned char* rp = static_cast<const unsigned char*>(ref);
    auto go = [&]() {
#define PILOT_FRAME_PROBE(LP, NV, VB)                                                                             \
    frame_gather_probe_kernel<LP, NV, VB><<<grid, 256, 0, s>>>(points, N, mp, rp, H, W, f[0], f[1], f[2], f[3], \
                                                               poses32, M, tile)
        if (vb == 32) {
            switch (vec) {
                case 1: PILOT_FRAME_PROBE(1, 1, 32); break;
                case 2: PILOT_FRAME_PROBE(2, 1, 32); break;
                case 4: PILOT_FRAME_PROBE(4, 1, 32); break;
                default: PILOT_FRAME_PROBE(8, 1, 32); break;
            }
        } else {
            switch (vec) {
                case 1: PILOT_FRAME_PROBE(1, 1, 16); break;
                case 2: PILOT_FRAME_PROBE(2, 1, 16); break;
                case 4: PILOT_FRAME_PROBE(4, 1, 16); break;
                case 8: PILOT_FRAME_PROBE(8, 1, 16); break;
                default: PILOT_FRAME_PROBE(8, 2, 16); break;
            }
        }
#undef PILOT_FRAME_PROBE
        return cudaGetLastError();
    };
    float ms = 0.f;
    const cudaError_t e = time_launch(go, s, &ms);
    if (e != cudaSuccess) return probe_fail(PILOT_ECUDA, cudaGetErrorString(e));
    // every CTA evaluates kHypTile poses (a short last tile repeats the last pose)
    *units_per_s = (double)N * (double)grid.y * kHypTile / (ms * 1e-3);
    return PILOT_OK;
}

}  // extern "C"
