// Build pass: for one level, every (anchor tile, hypothesis) pair evaluates the photo
// term of the objective and its normal equations at the hypothesis' candidate pose.
//
//   Eq. 1  r_j = f^q(pi(K_l, T, P_j)) - f^r(p_j)   (bilinear read of C channels)
//   Eq. 2  cost += rho(w_j ||r_j||^2)              (Huber on the squared norm)
//   Eq. 8  H += w_j rho' J_j^T J_j, g += w_j rho' J_j^T r_j
//
// with J_j = G_j A_j: G_j (C x 2) the analytic gradient of the bilinear interpolant and
// A_j (2 x 6) = d(u,v)/dp [I | -[p]x] the projection Jacobian times the se(3)
// generators (left perturbation, camera frame).  The dense C x 6 Jacobian is never
// formed: per anchor only the 2x2 Gram matrix M = G^T G, b = G^T r and s = ||r||^2 are
// summed over channels, then H_j = w A^T M A and g_j = w A^T b.
//
// Thread mapping.  A group of LP = C/4 consecutive lanes owns one anchor; lane q of the
// group reads channels [4q, 4q+4) of each of the 4 taps, so one tap of one anchor is a
// single contiguous C-element segment read by LP lanes (one 128-byte line at C = 32 in
// FP32).  The per-anchor sums are all-reduced inside the group with xor shuffles
// (bit-identical in every lane), every lane of the group then accumulates the same
// 29 sums, and the CTA reduces them across groups and warps in a fixed order: the
// result is deterministic and independent of the grid shape.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "pilot_internal.cuh"

namespace pilot {

// Load 4 consecutive channels starting at element `idx` and widen them to FP32.
template <pilot_dtype DT>
__device__ __forceinline__ float4 load4(const void* base, size_t idx) {
    if constexpr (DT == PILOT_F32) {
        return __ldg(reinterpret_cast<const float4*>(static_cast<const float*>(base) + idx));
    } else if constexpr (DT == PILOT_BF16) {
        // bfloat16 is the upper half of an IEEE binary32: widening is a 16-bit shift
        const uint2 r = __ldg(reinterpret_cast<const uint2*>(static_cast<const uint16_t*>(base) + idx));
        return make_float4(__uint_as_float(r.x << 16), __uint_as_float(r.x & 0xffff0000u),
                           __uint_as_float(r.y << 16), __uint_as_float(r.y & 0xffff0000u));
    } else if constexpr (DT == PILOT_F16) {
        const uint2 r = __ldg(reinterpret_cast<const uint2*>(static_cast<const uint16_t*>(base) + idx));
        __half2 h0, h1;
        memcpy(&h0, &r.x, 4);
        memcpy(&h1, &r.y, 4);
        const float2 a = __half22float2(h0), b = __half22float2(h1);
        return make_float4(a.x, a.y, b.x, b.y);
    } else {
        const uint32_t r = __ldg(reinterpret_cast<const uint32_t*>(static_cast<const uint8_t*>(base) + idx));
        const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(r & 0xffffu), __NV_E4M3);
        const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(r >> 16), __NV_E4M3);
        const float2 a = __half22float2(__half2(lo)), b = __half22float2(__half2(hi));
        return make_float4(a.x, a.y, b.x, b.y);
    }
}

struct ChanSums {
    float s, m00, m01, m11, b0, b1;
};

// One channel: bilinear value and in-cell gradient, residual, and the six sums.
__device__ __forceinline__ void channel(ChanSums& a, float t00, float t01, float t10, float t11,
                                        float fr, float ax, float ay, bool scaled, float sq,
                                        float sr) {
    const float bq = t01 - t00;              // d/dx along the upper row
    const float cq = t10 - t00;              // d/dy along the left column
    const float dq = (t11 - t10) - bq;       // bilinear cross term
    float fu = fmaf(dq, ay, bq);             // df/du inside the cell
    float fv = fmaf(dq, ax, cq);             // df/dv inside the cell
    float f = fmaf(ax, fu, fmaf(ay, cq, t00));
    if (scaled) {
        f *= sq;
        fu *= sq;
        fv *= sq;
        fr *= sr;
    }
    const float r = f - fr;
    a.s = fmaf(r, r, a.s);
    a.m00 = fmaf(fu, fu, a.m00);
    a.m01 = fmaf(fu, fv, a.m01);
    a.m11 = fmaf(fv, fv, a.m11);
    a.b0 = fmaf(fu, r, a.b0);
    a.b1 = fmaf(fv, r, a.b1);
}

template <pilot_dtype DT, int C>
__global__ void __launch_bounds__(kBuildThreads)
build_kernel(const BuildParams p) {
    static_assert(C % 4 == 0 && C >= 4 && C <= 128, "channels");
    constexpr int LP = C / 4;                       // lanes per anchor
    constexpr int GROUPS = kBuildThreads / LP;      // anchors in flight per CTA
    static_assert(LP <= 32, "group larger than a warp");
    __shared__ float red[kBuildThreads / 32][kAcc];

    const int slot = blockIdx.y;
    const int hyp = p.active_idx[slot];
    float* out = p.partial + ((size_t)slot * p.n_tiles + blockIdx.x) * kAcc;
    if (!p.state[hyp].has_cand) return;            // uniform over the CTA

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int q = tid % LP, grp = tid / LP;
    const unsigned gmask = (LP == 32) ? 0xffffffffu : (((1u << LP) - 1u) << (lane & ~(LP - 1)));

    const float* P = p.pose32 + 12 * hyp;
    const float R00 = P[0], R01 = P[1], R02 = P[2], T0 = P[3];
    const float R10 = P[4], R11 = P[5], R12 = P[6], T1 = P[7];
    const float R20 = P[8], R21 = P[9], R22 = P[10], T2 = P[11];

    const bool scaled = p.qscale != nullptr;
    float4 qs = make_float4(1.f, 1.f, 1.f, 1.f), rs = qs;
    if (scaled) {
        qs = __ldg(reinterpret_cast<const float4*>(p.qscale) + q);
        rs = __ldg(reinterpret_cast<const float4*>(p.rscale) + q);
    }

    float acc[kNumSums];
#pragma unroll
    for (int i = 0; i < kNumSums; ++i) acc[i] = 0.f;

    const int j0 = blockIdx.x * p.tile;
    const int j1 = min(j0 + p.tile, p.N);
    const size_t WC = (size_t)p.W * C;
    const float xmax = (float)(p.W - 1), ymax = (float)(p.H - 1);
    const float d2 = p.huber * p.huber;

    for (int j = j0 + grp; j < j1; j += GROUPS) {
        if (p.valid && !p.valid[j]) continue;
        const float X = __ldg(p.px + j), Y = __ldg(p.py + j), Z = __ldg(p.pz + j);
        // p = R P + t  (world -> camera)
        const float x = fmaf(R00, X, fmaf(R01, Y, fmaf(R02, Z, T0)));
        const float y = fmaf(R10, X, fmaf(R11, Y, fmaf(R12, Z, T1)));
        const float z = fmaf(R20, X, fmaf(R21, Y, fmaf(R22, Z, T2)));
        if (!(z > kZNear)) continue;
        const float iz = 1.0f / z;
        // pixel i covers [i, i+1): array coordinate = pixel - 1/2
        const float xs = fmaf(p.fx * x, iz, p.cx) - 0.5f;
        const float ys = fmaf(p.fy * y, iz, p.cy) - 0.5f;
        if (!(xs >= 0.f && xs <= xmax && ys >= 0.f && ys <= ymax)) continue;
        const int c0 = min((int)xs, p.W - 2);
        const int r0 = min((int)ys, p.H - 2);
        const float ax = xs - (float)c0, ay = ys - (float)r0;

        const size_t base = ((size_t)r0 * p.W + c0) * C + 4 * q;
        const float4 a00 = load4<DT>(p.qry, base);
        const float4 a01 = load4<DT>(p.qry, base + C);
        const float4 a10 = load4<DT>(p.qry, base + WC);
        const float4 a11 = load4<DT>(p.qry, base + WC + C);
        const float4 fr = load4<DT>(p.ref, (size_t)j * C + 4 * q);

        ChanSums cs{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        channel(cs, a00.x, a01.x, a10.x, a11.x, fr.x, ax, ay, scaled, qs.x, rs.x);
        channel(cs, a00.y, a01.y, a10.y, a11.y, fr.y, ax, ay, scaled, qs.y, rs.y);
        channel(cs, a00.z, a01.z, a10.z, a11.z, fr.z, ax, ay, scaled, qs.z, rs.z);
        channel(cs, a00.w, a01.w, a10.w, a11.w, fr.w, ax, ay, scaled, qs.w, rs.w);
#pragma unroll
        for (int off = 1; off < LP; off <<= 1) {
            cs.s += __shfl_xor_sync(gmask, cs.s, off);
            cs.m00 += __shfl_xor_sync(gmask, cs.m00, off);
            cs.m01 += __shfl_xor_sync(gmask, cs.m01, off);
            cs.m11 += __shfl_xor_sync(gmask, cs.m11, off);
            cs.b0 += __shfl_xor_sync(gmask, cs.b0, off);
            cs.b1 += __shfl_xor_sync(gmask, cs.b1, off);
        }

        // Huber on w ||r||^2 and the IRLS weight w rho'
        const float w = p.weight ? __ldg(p.weight + j) : 1.0f;
        const float sw = w * cs.s;
        float rho, drho;
        if (sw <= d2) {
            rho = sw;
            drho = 1.0f;
        } else {
            const float rt = sqrtf(sw);
            rho = 2.0f * p.huber * rt - d2;
            drho = p.huber / rt;
        }
        const float om = w * drho;

        // A = d(u,v)/dp [I | -[p]x]; the rotational part of each row a is p x a
        const float du_dx = p.fx * iz, du_dz = -p.fx * x * iz * iz;
        const float dv_dy = p.fy * iz, dv_dz = -p.fy * y * iz * iz;
        const float A0[6] = {du_dx, 0.f, du_dz, y * du_dz, z * du_dx - x * du_dz, -y * du_dx};
        const float A1[6] = {0.f, dv_dy, dv_dz, y * dv_dz - z * dv_dy, -x * dv_dz, x * dv_dy};
        float B0[6], B1[6], W0[6], W1[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            B0[k] = fmaf(cs.m00, A0[k], cs.m01 * A1[k]);
            B1[k] = fmaf(cs.m01, A0[k], cs.m11 * A1[k]);
            W0[k] = om * A0[k];
            W1[k] = om * A1[k];
        }
        int e = 0;
#pragma unroll
        for (int a = 0; a < 6; ++a) {
#pragma unroll
            for (int b = a; b < 6; ++b) {
                acc[e] = fmaf(W0[a], B0[b], fmaf(W1[a], B1[b], acc[e]));
                ++e;
            }
        }
#pragma unroll
        for (int a = 0; a < 6; ++a) acc[21 + a] = fmaf(W0[a], cs.b0, fmaf(W1[a], cs.b1, acc[21 + a]));
        acc[27] += rho;
        acc[28] += 1.0f;
    }

    // Every lane of a group holds the group's sums: reduce across groups, then warps.
#pragma unroll
    for (int off = LP; off < 32; off <<= 1) {
#pragma unroll
        for (int i = 0; i < kNumSums; ++i) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], off);
    }
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < kNumSums; ++i) red[warp][i] = acc[i];
    }
    __syncthreads();
    if (tid < kAcc) {
        float v = 0.f;
        if (tid < kNumSums) {
#pragma unroll
            for (int w = 0; w < kBuildThreads / 32; ++w) v += red[w][tid];
        }
        out[tid] = v;
    }
}

template <pilot_dtype DT, int C>
cudaError_t launch_build_typed(const BuildParams& p, cudaStream_t s) {
    dim3 grid(p.n_tiles, p.n_active);
    build_kernel<DT, C><<<grid, kBuildThreads, 0, s>>>(p);
    return cudaGetLastError();
}

template <pilot_dtype DT>
cudaError_t launch_build_dtype(const BuildParams& p, cudaStream_t s) {
    switch (p.C) {
        case 4: return launch_build_typed<DT, 4>(p, s);
        case 8: return launch_build_typed<DT, 8>(p, s);
        case 16: return launch_build_typed<DT, 16>(p, s);
        case 32: return launch_build_typed<DT, 32>(p, s);
        case 64: return launch_build_typed<DT, 64>(p, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pilot
