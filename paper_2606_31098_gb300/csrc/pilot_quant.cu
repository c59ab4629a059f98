// Feature quantiser: FP32 rows of C channels -> BF16 / FP16 / FP8-E4M3 storage with one
// FP32 scale per channel, stored value = round(x / s_c), value used = stored x s_c.
//
//   s_c = absmax_c / q_max   (q_max = 448 for E4M3; 65504 for FP16; 1 for BF16, i.e. unit
//                             absmax) when per-channel scaling is requested or the storage
//                             is E4M3; otherwise s_c = 1.
//   rounding: to nearest, ties to even; E4M3 saturates to +-448 (no infinities in E4M3).
//
// The absmax is reduced into the caller's scale array (as the bit patterns of the
// non-negative floats, whose unsigned order is their numeric order), which is then turned
// into the scales in place: no memory is allocated.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <string>

#include "pilot_internal.cuh"

namespace pilot {
namespace {

constexpr int kQuantThreads = 256;

__global__ void absmax_kernel(const float* __restrict__ src, long long rows, int C,
                              unsigned* __restrict__ bits) {
    extern __shared__ unsigned smax[];
    for (int c = threadIdx.x; c < C; c += blockDim.x) smax[c] = 0u;
    __syncthreads();
    const long long n4 = rows * C / 4;
    const float4* s4 = reinterpret_cast<const float4*>(src);
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n4;
         k += (long long)gridDim.x * blockDim.x) {
        const float4 v = __ldg(s4 + k);
        const int c = (int)((k * 4) % C);
        atomicMax(&smax[c], __float_as_uint(fabsf(v.x)));
        atomicMax(&smax[c + 1], __float_as_uint(fabsf(v.y)));
        atomicMax(&smax[c + 2], __float_as_uint(fabsf(v.z)));
        atomicMax(&smax[c + 3], __float_as_uint(fabsf(v.w)));
    }
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x) atomicMax(bits + c, smax[c]);
}

__global__ void scales_kernel(float* scale, int C, float qmax, int use_absmax) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const float amax = __uint_as_float(reinterpret_cast<unsigned*>(scale)[c]);
    float s = 1.0f;
    if (use_absmax && amax > 0.0f && isfinite(amax)) s = amax / qmax;
    scale[c] = s;
}

template <pilot_dtype DT>
__global__ void convert_kernel(const float* __restrict__ src, long long rows, int C,
                               const float* __restrict__ scale, void* __restrict__ dst) {
    const long long n4 = rows * C / 4;
    const float4* s4 = reinterpret_cast<const float4*>(src);
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n4;
         k += (long long)gridDim.x * blockDim.x) {
        const float4 v = __ldg(s4 + k);
        const int c = (int)((k * 4) % C);
        const float y0 = v.x * (1.0f / __ldg(scale + c));
        const float y1 = v.y * (1.0f / __ldg(scale + c + 1));
        const float y2 = v.z * (1.0f / __ldg(scale + c + 2));
        const float y3 = v.w * (1.0f / __ldg(scale + c + 3));
        if constexpr (DT == PILOT_BF16) {
            __nv_bfloat16* d = static_cast<__nv_bfloat16*>(dst) + 4 * k;
            d[0] = __float2bfloat16_rn(y0);
            d[1] = __float2bfloat16_rn(y1);
            d[2] = __float2bfloat16_rn(y2);
            d[3] = __float2bfloat16_rn(y3);
        } else if constexpr (DT == PILOT_F16) {
            __half* d = static_cast<__half*>(dst) + 4 * k;
            d[0] = __float2half_rn(y0);
            d[1] = __float2half_rn(y1);
            d[2] = __float2half_rn(y2);
            d[3] = __float2half_rn(y3);
        } else {
            uint8_t* d = static_cast<uint8_t*>(dst) + 4 * k;
            d[0] = __nv_cvt_float_to_fp8(y0, __NV_SATFINITE, __NV_E4M3);
            d[1] = __nv_cvt_float_to_fp8(y1, __NV_SATFINITE, __NV_E4M3);
            d[2] = __nv_cvt_float_to_fp8(y2, __NV_SATFINITE, __NV_E4M3);
            d[3] = __nv_cvt_float_to_fp8(y3, __NV_SATFINITE, __NV_E4M3);
        }
    }
}

int grid_for(long long n4) {
    long long b = (n4 + kQuantThreads - 1) / kQuantThreads;
    if (b > 152 * 8) b = 152 * 8;
    return b < 1 ? 1 : (int)b;
}

pilot_status qfail(pilot_status st, const std::string& m) {
    record_error(m.c_str());
    return st;
}

}  // namespace
}  // namespace pilot

using namespace pilot;

extern "C" pilot_status pilot_quantize_features(const float* src, long long rows, int C,
                                                pilot_dtype dtype, int per_channel, void* dst,
                                                float* scale, void* stream) {
    if (!src || !dst || !scale) return qfail(PILOT_EINVAL, "src, dst or scale is NULL");
    if (rows < 0 || C < 4 || C % 4 != 0 || C > 4096) return qfail(PILOT_EINVAL, "rows >= 0 and C a multiple of 4 in [4, 4096]");
    if (dtype != PILOT_BF16 && dtype != PILOT_F16 && dtype != PILOT_FP8E4M3)
        return qfail(PILOT_EINVAL, "dtype must be BF16, F16 or FP8E4M3");
    if (((uintptr_t)src & 15) != 0) return qfail(PILOT_EINVAL, "src must be 16-byte aligned");
    if (((uintptr_t)dst & 3) != 0) return qfail(PILOT_EINVAL, "dst must be 4-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long n4 = rows * C / 4;
    const bool use_absmax = per_channel != 0 || dtype == PILOT_FP8E4M3;
    const float qmax = dtype == PILOT_FP8E4M3 ? 448.0f : (dtype == PILOT_F16 ? 65504.0f : 1.0f);
    cudaError_t e = cudaMemsetAsync(scale, 0, sizeof(float) * C, s);
    if (e == cudaSuccess && use_absmax && n4 > 0) {
        absmax_kernel<<<grid_for(n4), kQuantThreads, sizeof(unsigned) * C, s>>>(
            src, rows, C, reinterpret_cast<unsigned*>(scale));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        scales_kernel<<<(C + 127) / 128, 128, 0, s>>>(scale, C, qmax, use_absmax ? 1 : 0);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && n4 > 0) {
        if (dtype == PILOT_BF16)
            convert_kernel<PILOT_BF16><<<grid_for(n4), kQuantThreads, 0, s>>>(src, rows, C, scale, dst);
        else if (dtype == PILOT_F16)
            convert_kernel<PILOT_F16><<<grid_for(n4), kQuantThreads, 0, s>>>(src, rows, C, scale, dst);
        else
            convert_kernel<PILOT_FP8E4M3><<<grid_for(n4), kQuantThreads, 0, s>>>(src, rows, C, scale, dst);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return qfail(PILOT_ECUDA, std::string("quantiser launch: ") + cudaGetErrorString(e));
    return PILOT_OK;
}
