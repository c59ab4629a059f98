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
// Thread mapping.  A group of LP = C / CPL consecutive lanes (CPL = 4 channels per lane,
// 8 at C = 64) works on LP anchors at a time.  Each lane projects one of them and
// broadcasts its tap offset and bilinear weights to the group; the group then reads the
// 4 taps of every anchor together, lane q taking channels [CPL q, CPL q + CPL), so one
// tap is one contiguous C-element segment read by LP lanes (one 128-byte line at C = 32
// in FP32).  A butterfly reduce-scatter over the group leaves in lane q the channel
// sums of anchor q, and each lane finishes its own anchor (Huber weight, A, 21 + 6
// sums) exactly once.  The CTA reduces the lanes' sums in a fixed order: the result is
// deterministic and independent of the grid shape.
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
    static_assert(C % 4 == 0 && C >= 4 && C <= 64, "channels");
    constexpr int CPL = (C >= 64) ? 8 : 4;          // channels per lane
    constexpr int NV = CPL / 4;                     // 4-channel vectors per lane and tap
    constexpr int LP = C / CPL;                     // lanes per group = anchors per batch
    constexpr int GROUPS = kBuildThreads / LP;
    constexpr int BATCH = GROUPS * LP;              // anchors per CTA pass
    static_assert(LP >= 1 && LP <= 16 && (LP & (LP - 1)) == 0, "group size");
    __shared__ float red[kBuildThreads / 32][kAcc];

    const int slot = blockIdx.y;
    const int hyp = p.active_idx[slot];
    float* out = p.partial + ((size_t)slot * p.n_tiles + blockIdx.x) * kAcc;
    if (!p.state[hyp].has_cand) return;            // uniform over the CTA

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int q = lane & (LP - 1);                  // lane within the group
    const int grp = tid / LP;
    const int src0 = lane & ~(LP - 1);              // first lane of the group
    const unsigned gmask = (LP == 32) ? 0xffffffffu : (((1u << LP) - 1u) << src0);

    const float* P = p.pose32 + 12 * hyp;
    const float R00 = P[0], R01 = P[1], R02 = P[2], T0 = P[3];
    const float R10 = P[4], R11 = P[5], R12 = P[6], T1 = P[7];
    const float R20 = P[8], R21 = P[9], R22 = P[10], T2 = P[11];

    const bool scaled = p.qscale != nullptr;
    float qs[CPL], rs[CPL];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        float4 a = make_float4(1.f, 1.f, 1.f, 1.f), b = a;
        if (scaled) {
            a = __ldg(reinterpret_cast<const float4*>(p.qscale) + q * NV + v);
            b = __ldg(reinterpret_cast<const float4*>(p.rscale) + q * NV + v);
        }
        qs[4 * v] = a.x; qs[4 * v + 1] = a.y; qs[4 * v + 2] = a.z; qs[4 * v + 3] = a.w;
        rs[4 * v] = b.x; rs[4 * v + 1] = b.y; rs[4 * v + 2] = b.z; rs[4 * v + 3] = b.w;
    }

    float acc[kNumSums];
#pragma unroll
    for (int i = 0; i < kNumSums; ++i) acc[i] = 0.f;

    const int j0 = blockIdx.x * p.tile;
    const int j1 = min(j0 + p.tile, p.N);
    const int WC = p.W * C;
    const float xmax = (float)(p.W - 1), ymax = (float)(p.H - 1);
    const float d2 = p.huber * p.huber;

    for (int jb = j0 + grp * LP; jb < j1; jb += BATCH) {
        // 1. every lane projects its own anchor jb + q
        const int jo = jb + q;
        bool vis = false;
        int off = 0;
        float ax = 0.f, ay = 0.f, x = 0.f, y = 0.f, z = 1.f, iz = 1.f;
        if (jo < j1 && (!p.valid || p.valid[jo])) {
            const float X = __ldg(p.px + jo), Y = __ldg(p.py + jo), Z = __ldg(p.pz + jo);
            // p = R P + t  (world -> camera)
            x = fmaf(R00, X, fmaf(R01, Y, fmaf(R02, Z, T0)));
            y = fmaf(R10, X, fmaf(R11, Y, fmaf(R12, Z, T1)));
            z = fmaf(R20, X, fmaf(R21, Y, fmaf(R22, Z, T2)));
            if (z > kZNear) {
                iz = 1.0f / z;
                // pixel i covers [i, i+1): array coordinate = pixel - 1/2
                const float xs = fmaf(p.fx * x, iz, p.cx) - 0.5f;
                const float ys = fmaf(p.fy * y, iz, p.cy) - 0.5f;
                if (xs >= 0.f && xs <= xmax && ys >= 0.f && ys <= ymax) {
                    const int c0 = min((int)xs, p.W - 2);
                    const int r0 = min((int)ys, p.H - 2);
                    ax = xs - (float)c0;
                    ay = ys - (float)r0;
                    off = (r0 * p.W + c0) * C;
                    vis = true;
                }
            }
        }

        // 2. the group gathers its LP anchors together: lane q reads channels
        //    [CPL q, CPL q + CPL) of the 4 taps and of the reference row of each
        float S[LP][6];
#pragma unroll
        for (int i = 0; i < LP; ++i) {
            const int vi = __shfl_sync(gmask, (int)vis, src0 + i);
            const int oi = __shfl_sync(gmask, off, src0 + i) + CPL * q;
            const float axi = __shfl_sync(gmask, ax, src0 + i);
            const float ayi = __shfl_sync(gmask, ay, src0 + i);
            const int ri = (vi ? jb + i : 0) * C + CPL * q;   // row 0 is a safe dummy
            ChanSums cs{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const float4 a00 = load4<DT>(p.qry, (size_t)oi + 4 * v);
                const float4 a01 = load4<DT>(p.qry, (size_t)oi + C + 4 * v);
                const float4 a10 = load4<DT>(p.qry, (size_t)oi + WC + 4 * v);
                const float4 a11 = load4<DT>(p.qry, (size_t)oi + WC + C + 4 * v);
                const float4 fr = load4<DT>(p.ref, (size_t)ri + 4 * v);
                channel(cs, a00.x, a01.x, a10.x, a11.x, fr.x, axi, ayi, scaled, qs[4 * v], rs[4 * v]);
                channel(cs, a00.y, a01.y, a10.y, a11.y, fr.y, axi, ayi, scaled, qs[4 * v + 1], rs[4 * v + 1]);
                channel(cs, a00.z, a01.z, a10.z, a11.z, fr.z, axi, ayi, scaled, qs[4 * v + 2], rs[4 * v + 2]);
                channel(cs, a00.w, a01.w, a10.w, a11.w, fr.w, axi, ayi, scaled, qs[4 * v + 3], rs[4 * v + 3]);
            }
            const float m = vi ? 1.0f : 0.0f;
            S[i][0] = cs.s * m;
            S[i][1] = cs.m00 * m;
            S[i][2] = cs.m01 * m;
            S[i][3] = cs.m11 * m;
            S[i][4] = cs.b0 * m;
            S[i][5] = cs.b1 * m;
        }

        // 3. butterfly reduce-scatter: afterwards S[0] of lane q holds anchor q's sums
#pragma unroll
        for (int half = LP / 2; half >= 1; half >>= 1) {
            const bool upper = (q & half) != 0;
#pragma unroll
            for (int t = 0; t < half; ++t) {
#pragma unroll
                for (int v = 0; v < 6; ++v) {
                    const float send = upper ? S[t][v] : S[t + half][v];
                    const float keep = upper ? S[t + half][v] : S[t][v];
                    S[t][v] = keep + __shfl_xor_sync(gmask, send, half);
                }
            }
        }

        // 4. each lane finishes its own anchor: Huber weight, A = d(u,v)/dp [I | -[p]x],
        //    H += w A^T M A, g += w A^T b
        if (vis) {
            const float s = S[0][0], m00 = S[0][1], m01 = S[0][2], m11 = S[0][3];
            const float b0 = S[0][4], b1 = S[0][5];
            const float w = p.weight ? __ldg(p.weight + jo) : 1.0f;
            const float sw = w * s;
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
            // the rotational part of each row a of d(u,v)/dp is p x a
            const float du_dx = p.fx * iz, du_dz = -p.fx * x * iz * iz;
            const float dv_dy = p.fy * iz, dv_dz = -p.fy * y * iz * iz;
            const float A0[6] = {du_dx, 0.f, du_dz, y * du_dz, z * du_dx - x * du_dz, -y * du_dx};
            const float A1[6] = {0.f, dv_dy, dv_dz, y * dv_dz - z * dv_dy, -x * dv_dz, x * dv_dy};
            float B0[6], B1[6], W0[6], W1[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                B0[k] = fmaf(m00, A0[k], m01 * A1[k]);
                B1[k] = fmaf(m01, A0[k], m11 * A1[k]);
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
            for (int a = 0; a < 6; ++a) acc[21 + a] = fmaf(W0[a], b0, fmaf(W1[a], b1, acc[21 + a]));
            acc[27] += rho;
            acc[28] += 1.0f;
        }
    }

    // Each lane holds distinct anchors: reduce across the warp, then across warps.
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
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
