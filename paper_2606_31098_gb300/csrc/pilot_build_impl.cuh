// Build pass: for one level, every (anchor tile, tile of hypotheses) evaluates the photo
// term of the objective and its normal equations at the hypotheses' candidate poses.
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
// Thread mapping.  A CTA holds kHypTile (HT) hypotheses over one anchor tile.  A group of
// LP consecutive lanes reads one tap with one load per lane, 32 bytes for FP32 and 16-bit
// maps and 16 bytes for FP8 and for maps with per-channel scales (LP = C x element size /
// load width, at most 8: 4 lanes for FP32 at C = 32, 2 for BF16, 2 for FP8), i.e. one L1
// wavefront per record and tap, where a record is one (anchor, hypothesis) pair.  A group works on LP
// records at a time: APB anchors under HG = min(HT, LP) hypotheses (APB HG = LP); with
// LP < HT, HT / HG neighbouring groups take the same anchors under the other hypotheses.
// Each lane projects one record (lane q of the group: anchor q mod APB under the group's
// hypothesis q div APB) and broadcasts its tap offset and bilinear weights to the group; the
// group then reads the 4 taps of every record and the reference row of every anchor
// together -- once for all the hypotheses of the CTA (vector k of lane q holds channels
// VW (q + k LP) .. + VW).  A butterfly reduce-scatter over the group leaves in lane q the
// channel sums of record q, and each lane finishes its own record (Huber weight, A, 21 + 6
// sums) exactly once.  An invisible record's partial sums stay in its own reduce-scatter
// slot and are discarded by its owner.  The hypothesis slot of a lane is read from lane bits
// log2 APB .. log2 (APB HT) - 1; the CTA reduces the lanes of each slot over the other lane
// bits, then the warps, in a fixed order.  A hypothesis' sums do not depend on which slot
// it takes or on the other hypotheses (the lanes of all slots run the same anchors in the
// same order, and the reduction trees are translates of one another), so the result is
// deterministic and independent of the grid shape and of how hypotheses are grouped.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "pilot_fp64.cuh"
#include "pilot_internal.cuh"

namespace pilot {

template <pilot_dtype DT> struct Storage;
template <> struct Storage<PILOT_F32> { using T = float; static constexpr int VEC = 8; };   // 32-byte loads
template <> struct Storage<PILOT_BF16> { using T = uint16_t; static constexpr int VEC = 16; };  // 32-byte loads
template <> struct Storage<PILOT_F16> { using T = uint16_t; static constexpr int VEC = 16; };
template <> struct Storage<PILOT_FP8E4M3> { using T = uint8_t; static constexpr int VEC = 16; };

// Load W (4, 8 or 16) consecutive channels at p and widen them to FP32 (one load of W
// elements: 4 to 16 bytes for the narrow types, 16 or 32 bytes for FP32).
template <pilot_dtype DT, int W>
__device__ __forceinline__ void load_vec(const typename Storage<DT>::T* p, float* out) {
    static_assert(W == 4 || W == 8 || W == 16, "vector width");
    if constexpr (DT == PILOT_F32) {
        static_assert(W <= 8, "FP32 vectors are at most 8 wide");
        if constexpr (W == 8) {
            // one 256-bit load (32-byte aligned: device feature pointers are validated for it)
            asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                : "=f"(out[0]), "=f"(out[1]), "=f"(out[2]), "=f"(out[3]), "=f"(out[4]), "=f"(out[5]),
                  "=f"(out[6]), "=f"(out[7])
                : "l"(p));
        } else {
            const float4 v = __ldg(reinterpret_cast<const float4*>(p));
            out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
        }
    } else if constexpr (DT == PILOT_BF16 || DT == PILOT_F16) {
        uint32_t w[W / 2];
        if constexpr (W == 16) {
            // one 256-bit load (32-byte aligned: device feature pointers are validated for it)
            asm("ld.global.nc.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7])
                : "l"(p));
        } else if constexpr (W == 8) {
            const uint4 r = __ldg(reinterpret_cast<const uint4*>(p));
            w[0] = r.x; w[1] = r.y; w[2] = r.z; w[3] = r.w;
        } else {
            const uint2 r = __ldg(reinterpret_cast<const uint2*>(p));
            w[0] = r.x; w[1] = r.y;
        }
#pragma unroll
        for (int k = 0; k < W / 2; ++k) {
            if constexpr (DT == PILOT_BF16) {
                // bfloat16 is the upper half of an IEEE binary32: widening is a 16-bit shift
                out[2 * k] = __uint_as_float(w[k] << 16);
                out[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
            } else {
                __half2 h;
                memcpy(&h, &w[k], 4);
                const float2 f = __half22float2(h);
                out[2 * k] = f.x;
                out[2 * k + 1] = f.y;
            }
        }
    } else {
        uint32_t w[W / 4];
        if constexpr (W == 16) {
            const uint4 r = __ldg(reinterpret_cast<const uint4*>(p));
            w[0] = r.x; w[1] = r.y; w[2] = r.z; w[3] = r.w;
        } else if constexpr (W == 8) {
            const uint2 r = __ldg(reinterpret_cast<const uint2*>(p));
            w[0] = r.x; w[1] = r.y;
        } else {
            w[0] = __ldg(reinterpret_cast<const uint32_t*>(p));
        }
#pragma unroll
        for (int k = 0; k < W / 4; ++k) {
            const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[k] & 0xffffu), __NV_E4M3);
            const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[k] >> 16), __NV_E4M3);
            const float2 a = __half22float2(__half2(lo)), b = __half22float2(__half2(hi));
            out[4 * k] = a.x; out[4 * k + 1] = a.y; out[4 * k + 2] = b.x; out[4 * k + 3] = b.y;
        }
    }
}

struct ChanSums {
    float s, m00, m01, m11, b0, b1;
};

// One channel: bilinear value and in-cell gradient, residual, and the six sums.
template <bool SCALED>
__device__ __forceinline__ void channel(ChanSums& a, float t00, float t01, float t10, float t11,
                                        float fr, float ax, float ay, float sq, float sr) {
    const float bq = t01 - t00;              // d/dx along the upper row
    const float cq = t10 - t00;              // d/dy along the left column
    const float dq = (t11 - t10) - bq;       // bilinear cross term
    float fu = fmaf(dq, ay, bq);             // df/du inside the cell
    float fv = fmaf(dq, ax, cq);             // df/dv inside the cell
    float f = fmaf(ax, fu, fmaf(ay, cq, t00));
    if constexpr (SCALED) {
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

// ---- two channels per instruction: packed FP32x2 arithmetic (each lane of the pair is
// rounded exactly like the scalar operation) ----
typedef unsigned long long f2;

__device__ __forceinline__ f2 pk(float lo, float hi) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk(f2 v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// Six sums over channel pairs: lane .lo of each accumulates even channels, .hi odd ones.
struct ChanSums2 {
    f2 s, m00, m01, m11, b0, b1;
};

// Two channels at once: the same operations as channel(), in packed form.
template <bool SCALED>
__device__ __forceinline__ void channel_pair(ChanSums2& a, f2 t00, f2 t01, f2 t10, f2 t11, f2 fr,
                                             f2 ax, f2 ay, f2 sq, f2 sr) {
    const f2 bq = sub2(t01, t00);
    const f2 cq = sub2(t10, t00);
    const f2 dq = sub2(sub2(t11, t10), bq);
    f2 fu = fma2(dq, ay, bq);
    f2 fv = fma2(dq, ax, cq);
    f2 f = fma2(ax, fu, fma2(ay, cq, t00));
    if constexpr (SCALED) {
        f = mul2(f, sq);
        fu = mul2(fu, sq);
        fv = mul2(fv, sq);
        fr = mul2(fr, sr);
    }
    const f2 r = sub2(f, fr);
    a.s = fma2(r, r, a.s);
    a.m00 = fma2(fu, fu, a.m00);
    a.m01 = fma2(fu, fv, a.m01);
    a.m11 = fma2(fv, fv, a.m11);
    a.b0 = fma2(fu, r, a.b0);
    a.b1 = fma2(fv, r, a.b1);
}

__device__ __forceinline__ float hsum(f2 v) {
    float lo, hi;
    upk(v, lo, hi);
    return lo + hi;
}

// Lane layout of the build pass for C channels stored as DT (see the top of the file): LP
// lanes per tap = records per group batch, HG hypotheses per group, NS = kHypTile / HG
// groups over the same anchors, APB anchors per group batch.  The slot of lane l is
// (l / APB) mod kHypTile.  Maps with per-channel scales keep 16-byte loads: the wider lane
// share of channels would hold twice the scale registers and spill.
template <pilot_dtype DT, int C, bool SCALED> struct GroupShape {
    static constexpr int VEC = SCALED ? 16 / (int)sizeof(typename Storage<DT>::T) : Storage<DT>::VEC;  // per load
    static constexpr int VW = (C < VEC) ? C : VEC;            // channels per vector load
    static constexpr int LP = (C / VW < 8) ? C / VW : 8;      // lanes per tap
    static constexpr int HG = LP < kHypTile ? LP : kHypTile;  // hypotheses per group
    static constexpr int NS = kHypTile / HG;                  // groups over the same anchors
    static constexpr int APB = LP / HG;                       // anchors per group batch
    static constexpr int NV = C / LP / VW;                    // vector loads per lane and tap
    static_assert(APB * kHypTile <= 32, "a warp holds every slot of an anchor");
};

// The CTA's hypotheses: their FP32 poses and whether each slot has one to evaluate.
struct SlotPoses {
    const float* p[kHypTile];
    bool act[kHypTile];
};

// The level-specific inputs of the anchor loop.
struct LevelView {
    const float* px;
    const float* py;
    const float* pz;
    const float* weight;
    const uint8_t* valid;
    const void* qry;
    const void* ref;
    const float* qscale;
    const float* rscale;
    const float* conf;
    int H, W;
    float fx, fy, cx, cy, huber;
};

__device__ __forceinline__ LevelView level_view(const BuildParams& p) {
    return LevelView{p.px, p.py, p.pz, p.weight, p.valid, p.qry, p.ref, p.qscale, p.rscale, p.conf,
                     p.H, p.W, p.fx, p.fy, p.cx, p.cy, p.huber};
}

// Channel sums of one record over this lane's channels (vector k covers VW (q + k LP) ..
// + VW): the 4 taps at t00 (row below at t00 + WC) against the reference values rr (already
// loaded, shared by the two hypotheses of an anchor): bilinear value and in-cell gradient,
// residual, and the six partial sums.
template <pilot_dtype DT, int C, bool SCALED>
__device__ __forceinline__ void record_partials(const typename Storage<DT>::T* t00, int WC, const float* rr,
                                                float ax, float ay, int q, const float* qs, const float* rs,
                                                float* p) {
    using G = GroupShape<DT, C, SCALED>;
    constexpr int VW = G::VW, LP = G::LP, NV = G::NV;
    const typename Storage<DT>::T* t10 = t00 + WC;
    const f2 ax2 = pk(ax, ax), ay2 = pk(ay, ay), z2 = pk(0.f, 0.f);
    ChanSums2 cs{z2, z2, z2, z2, z2, z2};
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const int c = VW * (q + k * LP);
        float a00[VW], a01[VW], a10[VW], a11[VW];
        load_vec<DT, VW>(t00 + c, a00);
        load_vec<DT, VW>(t00 + c + C, a01);
        load_vec<DT, VW>(t10 + c, a10);
        load_vec<DT, VW>(t10 + c + C, a11);
        const float* r = rr + k * VW;
#pragma unroll
        for (int e = 0; e < VW; e += 2)
            channel_pair<SCALED>(cs, pk(a00[e], a00[e + 1]), pk(a01[e], a01[e + 1]), pk(a10[e], a10[e + 1]),
                                 pk(a11[e], a11[e + 1]), pk(r[e], r[e + 1]), ax2, ay2,
                                 pk(qs[k * VW + e], qs[k * VW + e + 1]), pk(rs[k * VW + e], rs[k * VW + e + 1]));
    }
    p[0] = hsum(cs.s);
    p[1] = hsum(cs.m00);
    p[2] = hsum(cs.m01);
    p[3] = hsum(cs.m11);
    p[4] = hsum(cs.b0);
    p[5] = hsum(cs.b1);
}

// Accumulate anchors [j_begin, j_end) under the CTA's kHypTile hypotheses into this lane's
// 29 sums (the lane's own slot, see GroupShape).  sp: the slots' poses (12 FP32 values each)
// and whether each has a pose to evaluate (an inactive slot's lanes finish nothing).  Every
// thread of the CTA calls it with the same arguments; threads are grouped as described at
// the top of the file.
// PREFETCH: read the next batch's anchor coordinates one batch ahead (four more registers
// through the loop; the sums are the same either way).  FRESH_TID: read the thread index
// through a volatile move, so that the lane layout derived from it is recomputed at each call
// instead of being hoisted into an enclosing loop and held across that loop's function calls.
template <pilot_dtype DT, int C, bool SCALED, bool CONF, int NTHREADS, bool PREFETCH = true, bool FRESH_TID = false>
__device__ __forceinline__ void accumulate_anchors(const LevelView& v, const SlotPoses& sp, int j_begin, int j_end,
                                                   float* acc) {
    using Elem = typename Storage<DT>::T;
    using G = GroupShape<DT, C, SCALED>;
    constexpr int VW = G::VW, LP = G::LP, HG = G::HG, NS = G::NS, APB = G::APB, NV = G::NV;
    constexpr int CPL = C / LP;                      // channels per lane
    constexpr int ASTEP = NTHREADS / (LP * NS) * APB;   // anchors per CTA batch
    static_assert(C % 4 == 0 && C >= 4 && C <= 64 && LP >= 1 && LP <= 8, "channels");

    int tid = threadIdx.x;
    if constexpr (FRESH_TID) asm volatile("mov.u32 %0, %%tid.x;" : "=r"(tid));
    const int lane = tid & 31;
    const int q = lane & (LP - 1);
    const int slot = (lane / APB) % kHypTile;        // this lane's hypothesis slot
    const int qa = q % APB;                          // this lane's anchor in the batch
    const int src0 = lane & ~(LP - 1);
    const unsigned gmask = LP > 1 ? (((1u << LP) - 1u) << src0) : (1u << lane);

    const float* P = sp.p[0];
    bool act = sp.act[0];
#pragma unroll
    for (int h = 1; h < kHypTile; ++h)
        if (slot == h) {
            P = sp.p[h];
            act = sp.act[h];
        }
    const float R00 = P[0], R01 = P[1], R02 = P[2], T0 = P[3];
    const float R10 = P[4], R11 = P[5], R12 = P[6], T1 = P[7];
    const float R20 = P[8], R21 = P[9], R22 = P[10], T2 = P[11];

    // channels owned by this lane: vector k covers VW (q + k LP) .. + VW
    float qs[CPL], rs[CPL];
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int e = 0; e < VW; ++e) {
            const int ch = VW * (q + k * LP) + e;
            qs[k * VW + e] = SCALED ? __ldg(v.qscale + ch) : 1.0f;
            rs[k * VW + e] = SCALED ? __ldg(v.rscale + ch) : 1.0f;
        }

    const Elem* qry = static_cast<const Elem*>(v.qry);
    const Elem* ref = static_cast<const Elem*>(v.ref);
    const int WC = v.W * C;
    const float xmax = (float)(v.W - 1), ymax = (float)(v.H - 1);
    const float d2 = v.huber * v.huber;

    // with PREFETCH the anchor coordinates of the next batch are read one batch ahead, so
    // that their load latency overlaps the current batch's gathers
    const int jfirst = j_begin + (tid / (LP * NS)) * APB;
    float nX = 0.f, nY = 0.f, nZ = 0.f;
    bool nok = false;
    if (PREFETCH && jfirst + qa < j_end) {
        const int j = jfirst + qa;
        nok = act && (!v.valid || v.valid[j]);
        nX = __ldg(v.px + j), nY = __ldg(v.py + j), nZ = __ldg(v.pz + j);
    }
    for (int jb = jfirst; jb < j_end; jb += ASTEP) {
        // 1. every lane projects its own record: anchor jb + qa under its hypothesis
        const int jo = jb + qa;
        float X = nX, Y = nY, Z = nZ;
        bool ok = nok && jo < j_end;
        if constexpr (PREFETCH) {
            nok = false;
            if (jo + ASTEP < j_end) {
                const int j = jo + ASTEP;
                nok = act && (!v.valid || v.valid[j]);
                nX = __ldg(v.px + j), nY = __ldg(v.py + j), nZ = __ldg(v.pz + j);
            }
        } else if (jo < j_end) {
            ok = act && (!v.valid || v.valid[jo]);
            X = __ldg(v.px + jo), Y = __ldg(v.py + jo), Z = __ldg(v.pz + jo);
        }
        bool vis = false;
        int off = 0;
        float ax = 0.f, ay = 0.f, x = 0.f, y = 0.f, z = 1.f, iz = 1.f, wq = 1.f;
        if (ok) {
            // p = R P + t  (world -> camera)
            x = fmaf(R00, X, fmaf(R01, Y, fmaf(R02, Z, T0)));
            y = fmaf(R10, X, fmaf(R11, Y, fmaf(R12, Z, T1)));
            z = fmaf(R20, X, fmaf(R21, Y, fmaf(R22, Z, T2)));
            if (z > kZNear) {
                iz = 1.0f / z;
                // pixel i covers [i, i+1): array coordinate = pixel - 1/2
                const float xs = fmaf(v.fx * x, iz, v.cx) - 0.5f;
                const float ys = fmaf(v.fy * y, iz, v.cy) - 0.5f;
                if (xs >= 0.f && xs <= xmax && ys >= 0.f && ys <= ymax) {
                    const int c0 = min((int)xs, v.W - 2);
                    const int r0 = min((int)ys, v.H - 2);
                    ax = xs - (float)c0;
                    ay = ys - (float)r0;
                    off = (r0 * v.W + c0) * C;
                    vis = true;
                    if constexpr (CONF) {  // query confidence, bilinear in the same cell
                        const float* cp = v.conf + r0 * v.W + c0;
                        const float c00 = __ldg(cp), c01 = __ldg(cp + 1);
                        const float c10 = __ldg(cp + v.W), c11 = __ldg(cp + v.W + 1);
                        const float bq = c01 - c00, cq2 = c10 - c00, dq = (c11 - c10) - bq;
                        wq = fmaf(ax, fmaf(dq, ay, bq), fmaf(ay, cq2, c00));
                    }
                }
            }
        }

        float S[6];
        if constexpr (LP == 1) {
            // one lane per record: its own taps and reference row
            float rr[C];
            const Elem* fr = ref + (jo < j_end ? jo : j_begin) * C;
#pragma unroll
            for (int k = 0; k < NV; ++k) load_vec<DT, VW>(fr + VW * k, rr + VW * k);
            record_partials<DT, C, SCALED>(qry + off, WC, rr, ax, ay, 0, qs, rs, S);
        } else {
            // 2. the group reads its records two at a time: records t and t + LP/2, one
            //    anchor (t mod APB) under two of the group's hypotheses, against one read of
            //    the anchor's reference row (with four hypotheses per group, the rows are read
            //    once per batch and kept for both record pairs of an anchor); the first
            //    butterfly round (xor LP/2) keeps in each lane only the record it owns, so
            //    only LP/2 partial records stay live
            constexpr int HALF = LP / 2;
            float rra[HG > 2 ? APB : 1][CPL];
            if constexpr (HG > 2) {
#pragma unroll
                for (int a = 0; a < APB; ++a) {
                    const int ja = jb + a;
                    const Elem* fr = ref + (ja < j_end ? ja : j_begin) * C;
#pragma unroll
                    for (int k = 0; k < NV; ++k) load_vec<DT, VW>(fr + VW * (q + k * LP), rra[a] + k * VW);
                }
            }
            // one butterfly step: lane keeps the record of its half and adds the partner's
            auto combine = [&](float* lo, const float* hi, int half) {
                const bool upper = (q & half) != 0;
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    const float send = upper ? lo[k] : hi[k];
                    const float keep = upper ? hi[k] : lo[k];
                    lo[k] = keep + __shfl_xor_sync(gmask, send, half);
                }
            };
            // record pair t: records t and t + HALF (one anchor, two hypotheses) against one
            // reference read, then the first butterfly round
            auto pair = [&](int t, float* Bt) {
                float rrt[CPL];
                const float* rr = rra[HG > 2 ? t % APB : 0];
                if constexpr (HG <= 2) {
                    const int ja = jb + t;
                    const Elem* fr = ref + (ja < j_end ? ja : j_begin) * C;
#pragma unroll
                    for (int k = 0; k < NV; ++k) load_vec<DT, VW>(fr + VW * (q + k * LP), rrt + k * VW);
                    rr = rrt;
                }
                float P2[2][6];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int i = t + u * HALF;
                    // the tap offset carries visibility: -1 when the record is not visible
                    const int oi = __shfl_sync(gmask, vis ? off : -1, src0 + i);
                    const float axi = __shfl_sync(gmask, ax, src0 + i);
                    const float ayi = __shfl_sync(gmask, ay, src0 + i);
                    record_partials<DT, C, SCALED>(qry + (oi >= 0 ? oi : 0), WC, rr, axi, ayi, q, qs, rs, P2[u]);
                }
                combine(P2[0], P2[1], HALF);
#pragma unroll
                for (int k = 0; k < 6; ++k) Bt[k] = P2[0][k];
            };
            float B[HALF][6];
            if constexpr (HALF == 4) {
                // the pairs in the order 0, 2, 1, 3: the second round combines (0, 2) and
                // (1, 3) as soon as both exist, so fewer partial records stay live (the same
                // additions as the round-by-round order)
                pair(0, B[0]);
                pair(2, B[2]);
                combine(B[0], B[2], 2);
                pair(1, B[1]);
                pair(3, B[3]);
                combine(B[1], B[3], 2);
                combine(B[0], B[1], 1);
            } else {
#pragma unroll
                for (int t = 0; t < HALF; ++t) pair(t, B[t]);
                // remaining butterfly rounds: afterwards B[0] of lane q holds record q's sums
#pragma unroll
                for (int half = HALF / 2; half >= 1; half >>= 1)
#pragma unroll
                    for (int t = 0; t < half; ++t) combine(B[t], B[t + half], half);
            }
#pragma unroll
            for (int k = 0; k < 6; ++k) S[k] = B[0][k];
        }

        // 4. each lane finishes its own record: Huber weight, A = d(u,v)/dp [I | -[p]x],
        //    H += w A^T M A, g += w A^T b
        if (vis) {
            const float s = S[0], m00 = S[1], m01 = S[2], m11 = S[3];
            const float b0 = S[4], b1 = S[5];
            const float w = (v.weight ? __ldg(v.weight + jo) : 1.0f) * wq;
            const float sw = w * s;
            float rho, drho;
            if (sw <= d2) {
                rho = sw;
                drho = 1.0f;
            } else {
                const float rt = sqrtf(sw);
                rho = 2.0f * v.huber * rt - d2;
                drho = v.huber / rt;
            }
            const float om = w * drho;
            // the rotational part of each row a of d(u,v)/dp is p x a
            const float du_dx = v.fx * iz, du_dz = -v.fx * x * iz * iz;
            const float dv_dy = v.fy * iz, dv_dz = -v.fy * y * iz * iz;
            const float A0[6] = {du_dx, 0.f, du_dz, y * du_dz, z * du_dx - x * du_dz, -y * du_dx};
            const float A1[6] = {0.f, dv_dy, dv_dz, y * dv_dz - z * dv_dy, -x * dv_dz, x * dv_dy};
            // A0[1] = A1[0] = 0: the terms they multiply are left out (adding a zero product
            // leaves an FP32 sum unchanged, so the sums are the same as with them)
            float B0[6], B1[6], W0[6], W1[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                if (k == 0) {
                    B0[k] = m00 * A0[k];
                    B1[k] = m01 * A0[k];
                } else if (k == 1) {
                    B0[k] = m01 * A1[k];
                    B1[k] = m11 * A1[k];
                } else {
                    B0[k] = fmaf(m00, A0[k], m01 * A1[k]);
                    B1[k] = fmaf(m01, A0[k], m11 * A1[k]);
                }
                W0[k] = (k == 1) ? 0.f : om * A0[k];
                W1[k] = (k == 0) ? 0.f : om * A1[k];
            }
            int e = 0;
#pragma unroll
            for (int a = 0; a < 6; ++a) {
#pragma unroll
                for (int b = a; b < 6; ++b) {
                    if (a == 0) acc[e] = fmaf(W0[a], B0[b], acc[e]);
                    else if (a == 1) acc[e] = fmaf(W1[a], B1[b], acc[e]);
                    else acc[e] = fmaf(W0[a], B0[b], fmaf(W1[a], B1[b], acc[e]));
                    ++e;
                }
            }
#pragma unroll
            for (int a = 0; a < 6; ++a) {
                if (a == 0) acc[21 + a] = fmaf(W0[a], b0, acc[21 + a]);
                else if (a == 1) acc[21 + a] = fmaf(W1[a], b1, acc[21 + a]);
                else acc[21 + a] = fmaf(W0[a], b0, fmaf(W1[a], b1, acc[21 + a]));
            }
            acc[27] += rho;
            acc[28] += 1.0f;
        }
    }
}

// Fixed-order CTA reduction of the lanes' 29 sums, per hypothesis slot: the lanes of a slot
// are reduced by a butterfly over every lane bit but the slot bits (APB .. APB kHypTile / 2),
// then the warps in order.  Thread t < kHypTile kAcc returns sum t mod kAcc of slot t / kAcc
// (0 pads).
template <int NTHREADS, int APB>
__device__ __forceinline__ float cta_reduce_slots(float* acc, float (*red)[kHypTile][kAcc]) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        if (off >= APB && off < APB * kHypTile) continue;
#pragma unroll
        for (int i = 0; i < kNumSums; ++i) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], off);
    }
    if (lane % APB == 0 && lane < APB * kHypTile) {
#pragma unroll
        for (int i = 0; i < kNumSums; ++i) red[warp][lane / APB][i] = acc[i];
    }
    __syncthreads();
    float v = 0.f;
    if (tid < kHypTile * kAcc && (tid % kAcc) < kNumSums) {
#pragma unroll
        for (int w = 0; w < NTHREADS / 32; ++w) v += red[w][tid / kAcc][tid % kAcc];
    }
    return v;
}

// The CTA's hypotheses: slots kHypTile blockIdx.y + h of the active list, h < n.
struct TileSlots {
    int slot[kHypTile];
    int hyp[kHypTile];
    bool cand[kHypTile];
    int n;                                           // 1 .. kHypTile
};

__device__ __forceinline__ TileSlots tile_slots(const BuildParams& p) {
    TileSlots s;
    s.n = min(kHypTile, p.n_active - kHypTile * (int)blockIdx.y);
#pragma unroll
    for (int h = 0; h < kHypTile; ++h) {
        s.slot[h] = kHypTile * blockIdx.y + (h < s.n ? h : 0);
        s.hyp[h] = p.active_idx[s.slot[h]];
        s.cand[h] = h < s.n && p.state[s.hyp[h]].has_cand;
    }
    return s;
}

__device__ __forceinline__ SlotPoses slot_poses(const BuildParams& p, const TileSlots& ts) {
    SlotPoses sp;
#pragma unroll
    for (int h = 0; h < kHypTile; ++h) {
        sp.p[h] = p.pose32 + 12 * ts.hyp[h];
        sp.act[h] = ts.cand[h];
    }
    return sp;
}

__device__ __forceinline__ bool any_cand(const TileSlots& ts) {
    bool a = false;
#pragma unroll
    for (int h = 0; h < kHypTile; ++h) a = a || ts.cand[h];
    return a;
}

template <pilot_dtype DT, int C, bool SCALED, bool CONF>
__global__ void __launch_bounds__(kBuildThreads, 2)
build_kernel(const BuildParams p) {
    __shared__ float red[kBuildThreads / 32][kHypTile][kAcc];
    const TileSlots ts = tile_slots(p);
    if (!any_cand(ts)) return;                       // uniform over the CTA
    float acc[kNumSums];
#pragma unroll
    for (int i = 0; i < kNumSums; ++i) acc[i] = 0.f;
    const int j0 = blockIdx.x * p.tile;
    accumulate_anchors<DT, C, SCALED, CONF, kBuildThreads>(level_view(p), slot_poses(p, ts), j0,
                                                           min(j0 + p.tile, p.N), acc);
    const float v = cta_reduce_slots<kBuildThreads, GroupShape<DT, C, SCALED>::APB>(acc, red);
    const int h = threadIdx.x / kAcc;
    if (threadIdx.x < kHypTile * kAcc && h < ts.n && ts.cand[h])
        p.partial[((size_t)ts.slot[h] * p.n_tiles + blockIdx.x) * kAcc + threadIdx.x % kAcc] = v;
}

// The same pass with the per-hypothesis FP64 step fused in: the CTA that takes the last
// ticket of its hypothesis tile sums the tile records of its hypotheses (FP64, 8 chains per
// value, fixed order) and runs lm_step for hypothesis h on warp h.  A tile of hypotheses with
// no candidate runs its steps in tile 0's CTA.
template <pilot_dtype DT, int C, bool SCALED, bool CONF>
__global__ void __launch_bounds__(kBuildThreads, 2)
build_fused_kernel(const FusedBuildParams fp) {
    const BuildParams& p = fp.b;
    __shared__ float red[kBuildThreads / 32][kHypTile][kAcc];
    __shared__ double part[kHypTile][8][kAcc];
    __shared__ double E[kHypTile][kAcc];
    __shared__ int s_last;
    const TileSlots ts = tile_slots(p);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (!any_cand(ts)) {                             // uniform over the CTA
        if (blockIdx.x == 0 && warp < ts.n) lm_step(fp.ep, ts.slot[warp], E[warp], &part[warp][0][0], *fp.min_valid, lane);
        return;
    }
    float acc[kNumSums];
#pragma unroll
    for (int i = 0; i < kNumSums; ++i) acc[i] = 0.f;
    const int j0 = blockIdx.x * p.tile;
    accumulate_anchors<DT, C, SCALED, CONF, kBuildThreads>(level_view(p), slot_poses(p, ts), j0,
                                                           min(j0 + p.tile, p.N), acc);
    const float v = cta_reduce_slots<kBuildThreads, GroupShape<DT, C, SCALED>::APB>(acc, red);
    const int hv = tid / kAcc, iv = tid % kAcc;     // slot and sum this thread holds (tid < kHypTile kAcc)
    if (p.n_tiles == 1) {
        // the only tile: its record is the sum (0 + x is what the 8-chain sum gives), no
        // round trip through the partial buffer and the ticket
        if (tid < kHypTile * kAcc) E[hv][iv] = 0.0 + (double)v;
        __syncthreads();
        if (warp < ts.n) lm_step(fp.ep, ts.slot[warp], E[warp], &part[warp][0][0], *fp.min_valid, lane);
        return;
    }
    if (tid < kHypTile * kAcc && hv < ts.n && ts.cand[hv])
        p.partial[((size_t)ts.slot[hv] * p.n_tiles + blockIdx.x) * kAcc + iv] = v;
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(fp.tickets + blockIdx.y, 1u) == (unsigned)(p.n_tiles - 1));
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // 8 chains per slot and value: thread (h, c, i) sums tiles c, c + 8, ... of sum i of slot h
    {
        constexpr int kTPC = kBuildThreads / (kHypTile * 8);     // threads per (slot, chain)
        const int h = tid / (8 * kTPC), c = (tid / kTPC) & 7;
        for (int ii = tid % kTPC; ii < kAcc; ii += kTPC) {
            double a = 0.0;
            if (h < ts.n && ts.cand[h]) {
                const float* src = p.partial + (size_t)ts.slot[h] * p.n_tiles * kAcc + ii;
                for (int t = c; t < p.n_tiles; t += 8) a += (double)__ldcg(src + (size_t)t * kAcc);
            }
            part[h][c][ii] = a;
        }
    }
    __syncthreads();
    if (tid < kHypTile * kAcc) {
        double sum = 0.0;
#pragma unroll
        for (int k = 0; k < 8; ++k) sum += part[hv][k][iv];
        E[hv][iv] = sum;
    }
    __syncthreads();
    if (warp < ts.n) {                               // the warp-cooperative FP64 steps
        lm_step(fp.ep, ts.slot[warp], E[warp], &part[warp][0][0], *fp.min_valid, lane);
    }
    if (tid == 0) fp.tickets[blockIdx.y] = 0u;
}

template <pilot_dtype DT, int C>
cudaError_t launch_build_typed(const BuildParams& p, cudaStream_t s) {
    dim3 grid(p.n_tiles, (p.n_active + kHypTile - 1) / kHypTile);
    if (p.qscale && p.conf)
        build_kernel<DT, C, true, true><<<grid, kBuildThreads, 0, s>>>(p);
    else if (p.qscale)
        build_kernel<DT, C, true, false><<<grid, kBuildThreads, 0, s>>>(p);
    else if (p.conf)
        build_kernel<DT, C, false, true><<<grid, kBuildThreads, 0, s>>>(p);
    else
        build_kernel<DT, C, false, false><<<grid, kBuildThreads, 0, s>>>(p);
    return cudaGetLastError();
}

template <pilot_dtype DT, int C>
cudaError_t launch_build_fused_typed(const FusedBuildParams& p, cudaStream_t s) {
    dim3 grid(p.b.n_tiles, (p.b.n_active + kHypTile - 1) / kHypTile);
    if (p.b.qscale && p.b.conf)
        build_fused_kernel<DT, C, true, true><<<grid, kBuildThreads, 0, s>>>(p);
    else if (p.b.qscale)
        build_fused_kernel<DT, C, true, false><<<grid, kBuildThreads, 0, s>>>(p);
    else if (p.b.conf)
        build_fused_kernel<DT, C, false, true><<<grid, kBuildThreads, 0, s>>>(p);
    else
        build_fused_kernel<DT, C, false, false><<<grid, kBuildThreads, 0, s>>>(p);
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

template <pilot_dtype DT>
cudaError_t launch_build_fused_dtype(const FusedBuildParams& p, cudaStream_t s) {
    switch (p.b.C) {
        case 4: return launch_build_fused_typed<DT, 4>(p, s);
        case 8: return launch_build_fused_typed<DT, 8>(p, s);
        case 16: return launch_build_fused_typed<DT, 16>(p, s);
        case 32: return launch_build_fused_typed<DT, 32>(p, s);
        case 64: return launch_build_fused_typed<DT, 64>(p, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pilot
