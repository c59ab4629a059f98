// FP64 per-hypothesis part of an LM iteration (device functions shared by the
// separately launched epilogue and by the build pass' fused last-CTA epilogue).
//
//   gravity term  Eq. 3: r = R gamma^W - gamma^imu, J = [0 | -[a]x], a = R gamma^W
//   range term    Eq. 4-6: P = R^T (q - t), r = P_z - D(P_x, P_y), J = [-n | n x q]
//                 with n = R (-D_x, -D_y, 1) and q = d v
//   assembly      Supp. "Sensor-Prior Fusion in LM": H, g are sums over the terms
//   LM step       Eq. 8: (H + lambda I) dxi = -g by 6x6 Cholesky, Eq. 9: T' = exp(dxi) T
//   acceptance    keep T' iff its objective is lower and enough anchors stay visible
#pragma once

#include <math.h>

#include "pilot_internal.cuh"

namespace pilot {

constexpr double kLambdaMin = 1e-12;
constexpr double kLambdaMax = 1e12;

__device__ __forceinline__ int tri_index(int a, int b) {
    // row-major upper triangle of a 6x6 matrix, a <= b
    return a * 6 - (a * (a - 1)) / 2 + (b - a);
}

__device__ __forceinline__ void huber64(double s, double delta, double* rho, double* drho) {
    const double d2 = delta * delta;
    if (s <= d2) {
        *rho = s;
        *drho = 1.0;
    } else {
        const double q = sqrt(s);
        *rho = 2.0 * delta * q - d2;
        *drho = delta / q;
    }
}

// The step is warp-cooperative: all 32 lanes of one warp run it together.  GB300 issues an
// FP64 instruction for the whole warp at a fraction of the FP32 rate, so one lane working
// alone pays for 32; here independent FP64 operations (the 21 + 6 + 1 entries a prior adds,
// the rows of the Cholesky factor, the three series, the entries of Exp, V and T') run one
// per lane, and scalar work (residuals, Huber weights, pivots) runs redundantly on every
// lane, which costs the same.  Each E entry's arithmetic is the one a single thread would
// do; W is 128 doubles of the warp's shared memory.

// (row, column) of upper-triangle entry k (row-major), k < 21
__device__ __forceinline__ void tri_pair(int k, int* a, int* b) {
    int r = 0, base = 0;           // row r starts at entry base; rows hold 6, 5, ..., 1 entries
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        if (r == i && k >= base + (6 - i)) {
            base += 6 - i;
            r = i + 1;
        }
    }
    *a = r;
    *b = r + (k - base);
}

__device__ __forceinline__ double shfl_d(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }

// Gravity direction prior (Eq. 3) at pose T, added to E = H21 | g6 | cost.
__device__ inline void add_gravity(const PriorParams& pp, const double* T, double* E, int lane) {
    double a[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
        a[i] = T[4 * i] * pp.g_world[0] + T[4 * i + 1] * pp.g_world[1] + T[4 * i + 2] * pp.g_world[2];
    const double r[3] = {a[0] - pp.g_cam[0], a[1] - pp.g_cam[1], a[2] - pp.g_cam[2]};
    double rho, drho;
    const double s = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    if (pp.gate_grav > 0.0 && s > pp.gate_grav * pp.gate_grav) {   // gated: constant, no pull
        huber64(pp.gate_grav * pp.gate_grav, pp.huber_grav, &rho, &drho);
        if (lane == 9) E[27] += pp.w_grav * rho;
        return;
    }
    huber64(s, pp.huber_grav, &rho, &drho);
    const double w = pp.w_grav * drho;
    // rotation block: w [a]x^T [a]x = w (|a|^2 I - a a^T); gradient: w [a]x r = w (a x r)
    const double aa = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
    if (lane < 6) {
        const int i = lane < 3 ? 0 : (lane < 5 ? 1 : 2);
        const int k = lane < 3 ? lane : (lane < 5 ? lane - 2 : 2);
        const double ai = i == 0 ? a[0] : (i == 1 ? a[1] : a[2]);
        const double ak = k == 0 ? a[0] : (k == 1 ? a[1] : a[2]);
        E[tri_index(3 + i, 3 + k)] += w * ((i == k ? aa : 0.0) - ai * ak);
    } else if (lane == 6) {
        E[21 + 3] += w * (a[1] * r[2] - a[2] * r[1]);
    } else if (lane == 7) {
        E[21 + 4] += w * (a[2] * r[0] - a[0] * r[2]);
    } else if (lane == 8) {
        E[21 + 5] += w * (a[0] * r[1] - a[1] * r[0]);
    } else if (lane == 9) {
        E[27] += pp.w_grav * rho;
    }
}

// Laser range prior (Eq. 4-6) at pose T; dropped when the range point leaves the DSM.
__device__ inline void add_range(const PriorParams& pp, const double* T, double* E, int lane) {
    const double d[3] = {pp.q[0] - T[3], pp.q[1] - T[7], pp.q[2] - T[11]};
    double P[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) P[i] = T[i] * d[0] + T[4 + i] * d[1] + T[8 + i] * d[2];  // R^T d
    const double inv_gsd = pp.dsm_inv_gsd;
    const double gx = (P[0] - pp.dsm_x0) * inv_gsd - 0.5;
    const double gy = (P[1] - pp.dsm_y0) * inv_gsd - 0.5;
    if (!(gx >= 0.0 && gx <= pp.dsm_W - 1.0 && gy >= 0.0 && gy <= pp.dsm_H - 1.0)) return;
    const int c0 = min((int)gx, pp.dsm_W - 2), r0 = min((int)gy, pp.dsm_H - 2);
    const double ax = gx - c0, ay = gy - r0;
    const float* row0 = pp.dsm + (size_t)r0 * pp.dsm_W + c0;
    const float* row1 = row0 + pp.dsm_W;
    const double h00 = row0[0], h01 = row0[1], h10 = row1[0], h11 = row1[1];
    const double bx = h01 - h00, cy = h10 - h00, dxy = (h11 - h10) - bx;
    const double D = h00 + ax * (bx + dxy * ay) + ay * cy;
    const double Dx = (bx + dxy * ay) * inv_gsd, Dy = (cy + dxy * ax) * inv_gsd;
    const double r = P[2] - D;
    double rho, drho;
    if (pp.gate_range > 0.0 && fabs(r) > pp.gate_range) {          // gated: constant, no pull
        huber64(pp.gate_range * pp.gate_range, pp.huber_range, &rho, &drho);
        if (lane == 27) E[27] += pp.w_range * rho;
        return;
    }
    // dr/dP = e = (-Dx, -Dy, 1); dP/ddelta = R^T [-I | [q]x]  =>  J = [-(R e) | (R e) x q]
    const double e[3] = {-Dx, -Dy, 1.0};
    double n[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) n[i] = T[4 * i] * e[0] + T[4 * i + 1] * e[1] + T[4 * i + 2] * e[2];
    const double J[6] = {-n[0], -n[1], -n[2],
                         n[1] * pp.q[2] - n[2] * pp.q[1],
                         n[2] * pp.q[0] - n[0] * pp.q[2],
                         n[0] * pp.q[1] - n[1] * pp.q[0]};
    huber64(r * r, pp.huber_range, &rho, &drho);
    const double w = pp.w_range * drho;
    if (lane < 21) {
        int a, b;
        tri_pair(lane, &a, &b);
        E[lane] += w * J[a] * J[b];
    } else if (lane < 27) {
        E[lane] += w * J[lane - 21] * r;
    } else if (lane == 27) {
        E[27] += pp.w_range * rho;
    }
}

// (H + damping) x = -g by Cholesky; lane i < 6 owns row i of the factor.  Returns false
// (on every lane) if the damped matrix is not positive definite.  H21 and g in shared memory.
__device__ inline bool damped_solve(const double* H21, const double* g, double lambda, int mode,
                                    double* x, double* Lsh, int lane) {
    const int i = lane < 6 ? lane : 5;
    double Lr[6], inv[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        // a_ij = A_ij - sum_{k<j} L_ik L_jk for this lane's row (meaningful when i >= j)
        double a = H21[tri_index(min(i, j), max(i, j))];
        if (i == j) a += (mode == 1) ? lambda * H21[tri_index(i, i)] : lambda;
#pragma unroll
        for (int k = 0; k < j; ++k) a -= Lr[k] * shfl_d(Lr[k], j);
        const double d = shfl_d(a, j);
        if (!(d > 0.0)) return false;
        const double ljj = sqrt(d);
        inv[j] = 1.0 / ljj;
        Lr[j] = (i == j) ? ljj : a * inv[j];
    }
    // L y = -g: once y_k is known every later row subtracts its term
    double s = -g[i];
    double y[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        y[k] = shfl_d(s, k) * inv[k];
        if (i > k) s -= Lr[k] * y[k];
    }
    // L^T x = y: row k of L (lane k) is read from shared memory
    if (lane < 6) {
#pragma unroll
        for (int k = 0; k < 6; ++k) Lsh[6 * lane + k] = Lr[k];
    }
    __syncwarp();
    double t = y[i];
#pragma unroll
    for (int k = 5; k >= 0; --k) {
        x[k] = shfl_d(t, k) * inv[k];
        if (i < k) t -= Lsh[6 * k + i] * x[k];
    }
    return true;
}

// Coefficients of Exp and V: A = sin(th)/th, B = (1 - cos th)/th^2, C = (th - sin th)/th^3.
// For th <= 0.25 rad (every LM step in practice) their Maclaurin series in x = th^2,
//   A = sum_k (-x)^k / (2k+1)!,  B = sum_k (-x)^k / (2k+2)!,  C = sum_k (-x)^k / (2k+3)!,
// are summed for k = 0..8 by Horner (the first omitted term is below 1e-27), lane 0 summing
// A, lane 1 B and lane 2 C; larger angles use sin and cos.
__device__ inline void exp_coefficients(double x, double* A, double* B, double* C, int lane) {
    if (x <= 0.0625) {
        // reciprocal factorials 1/n!, n = 1..19
        constexpr double f[20] = {1.0, 1.0, 1.0 / 2, 1.0 / 6, 1.0 / 24, 1.0 / 120, 1.0 / 720, 1.0 / 5040,
                                  1.0 / 40320, 1.0 / 362880, 1.0 / 3628800, 1.0 / 39916800,
                                  1.0 / 479001600, 1.0 / 6227020800.0, 1.0 / 87178291200.0,
                                  1.0 / 1307674368000.0, 1.0 / 20922789888000.0,
                                  1.0 / 355687428096000.0, 1.0 / 6402373705728000.0,
                                  1.0 / 121645100408832000.0};
        const int o = lane < 3 ? lane : 0;     // series o: coefficients f[2k + 1 + o]
        double v = o == 0 ? f[17] : (o == 1 ? f[18] : f[19]);
#pragma unroll
        for (int k = 7; k >= 0; --k) {
            const double c = o == 0 ? f[2 * k + 1] : (o == 1 ? f[2 * k + 2] : f[2 * k + 3]);
            v = c - x * v;
        }
        *A = shfl_d(v, 0);
        *B = shfl_d(v, 1);
        *C = shfl_d(v, 2);
    } else {
        const double th = sqrt(x);
        double sn, cs;
        sincos(th, &sn, &cs);
        *A = sn / th;
        *B = (1.0 - cs) / x;
        *C = (th - sn) / (x * th);
    }
}

// T' = exp(xi) T with xi = (nu, omega):  Exp(w) = I + A K + B K^2,
// V = I + B K + C K^2, K = [w]x, K^2 = w w^T - th^2 I.  Lanes 0..8 form Exp, 9..17 V
// (in W), then lanes 0..11 one entry of T' each, written to Tn.  T in shared memory.
__device__ inline void pose_update(const double* xi, const double* T, double* Tn, double* W, int lane) {
    const double w0 = xi[3], w1 = xi[4], w2 = xi[5];
    const double th2 = w0 * w0 + w1 * w1 + w2 * w2;
    double A, B, Cc;
    exp_coefficients(th2, &A, &B, &Cc, lane);
    if (lane < 18) {
        const int e = lane < 9 ? lane : lane - 9;
        const int i = e / 3, k = e % 3;
        const double wi = i == 0 ? w0 : (i == 1 ? w1 : w2);
        const double wk = k == 0 ? w0 : (k == 1 ? w1 : w2);
        // K[i][k] = -eps_ikl w_l
        double Kik = 0.0;
        if (i == 0 && k == 1) Kik = -w2;
        if (i == 0 && k == 2) Kik = w1;
        if (i == 1 && k == 0) Kik = w2;
        if (i == 1 && k == 2) Kik = -w0;
        if (i == 2 && k == 0) Kik = -w1;
        if (i == 2 && k == 1) Kik = w0;
        const double K2 = wi * wk - (i == k ? th2 : 0.0);
        const double I = (i == k) ? 1.0 : 0.0;
        W[lane] = lane < 9 ? I + A * Kik + B * K2 : I + B * Kik + Cc * K2;
    }
    __syncwarp();
    if (lane < 12) {
        const int i = lane >> 2, k = lane & 3;
        const double* Re = W + 3 * i;
        const double* V = W + 9 + 3 * i;
        double v = Re[0] * T[k] + Re[1] * T[4 + k] + Re[2] * T[8 + k];
        if (k == 3) v += V[0] * xi[0] + V[1] * xi[1] + V[2] * xi[2];
        Tn[lane] = v;
    }
}

__device__ __forceinline__ void store_pose32(float* dst, const double* T) {
    for (int i = 0; i < 12; ++i) dst[i] = (float)T[i];
}

// One hypothesis' FP64 step after a build pass at its candidate.  E (29 sums in the warp's
// shared memory, photo term only on entry) gets the priors at the evaluated pose; then
// (init) it becomes the current state, or (step) the candidate is accepted or rejected; then
// the next candidate is solved for and, if cand32 is given, written there in FP32.  All 32
// lanes of one warp call it with the same arguments; W is 128 doubles of the warp's shared
// memory.
//
// Not inlined: every kernel of a translation unit (plain fused, batched, served) then runs
// the same compiled instructions, so the compiler cannot contract a * b + c into an FMA in
// one caller and not in another, and the forms stay bitwise equal.
static __device__ __noinline__ void lm_update(HypState& st, int mode, int solve_next, int damping_mode,
                                              const PriorParams& prior, double* E, double* W,
                                              double min_valid, float* cand32, double* eval_out, int lane) {
    // every read of the state is issued here, before any write, as one round trip, from L2:
    // the persistent level kernel may step a hypothesis on another SM than the last time
    const int has_cand = __ldcg(&st.has_cand);
    const double cost0 = __ldcg(&st.cost);
    const double lambda0 = __ldcg(&st.lambda);
    const double* Tsrc = (mode == kEpiStep) ? st.Tc : st.T;
    double Tev[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) Tev[i] = __ldcg(Tsrc + i);
    const double Hg_own = lane < 21 ? __ldcg(st.H + lane) : (lane < 27 ? __ldcg(st.g + lane - 21) : 0.0);
    const double T_own = lane < 12 ? __ldcg(st.T + lane) : 0.0;
    const double Tc_own = lane < 12 ? __ldcg(st.Tc + lane) : 0.0;
    const bool evaluated = (mode == kEpiStep) ? (has_cand != 0) : true;
    if (evaluated) {
        if (prior.use_gravity) add_gravity(prior, Tev, E, lane);
        __syncwarp();
        if (prior.use_range) add_range(prior, Tev, E, lane);
        __syncwarp();
    }
    if (mode == kEpiEval) {
        if (lane < kNumSums) eval_out[lane] = E[lane];
        if (lane == 0) st.has_cand = 0;
        return;
    }
    // the state after acceptance, staged in W: H 0..20, g 21..26, T 32..43
    bool take = false;
    double lambda = lambda0;
    if (mode == kEpiInit) {
        take = true;
    } else if (evaluated) {
        take = E[27] < cost0 && E[28] >= min_valid;
        lambda = take ? fmax(lambda0 / 10.0, kLambdaMin) : fmin(lambda0 * 10.0, kLambdaMax);
    }
    if (lane < 27) W[lane] = take ? E[lane] : Hg_own;
    if (lane < 12) W[32 + lane] = (take && mode == kEpiStep) ? Tc_own : T_own;
    __syncwarp();
    if (take) {
        if (lane < 21) st.H[lane] = E[lane];
        else if (lane < 27) st.g[lane - 21] = E[lane];
        else if (lane == 27) st.cost = E[27];
        else if (lane == 28) st.n_valid = (int)E[28];
        if (mode == kEpiStep && lane < 12) st.T[lane] = W[32 + lane];
    }
    int cand = 0, fail = -1;
    if (solve_next) {
        double dxi[6];
        if (!damped_solve(W, W + 21, lambda, damping_mode, dxi, W + 64, lane)) {
            lambda = fmin(lambda * 10.0, kLambdaMax);
            fail = 1;
        } else {
            fail = 0;
            __syncwarp();
            pose_update(dxi, W + 32, W + 48, W + 100, lane);
            __syncwarp();
            if (lane < 12) {
                const double Tn = W[48 + lane];
                st.Tc[lane] = Tn;
                if (cand32) cand32[lane] = (float)Tn;
            }
            cand = 1;
        }
    }
    if (lane == 0) {
        st.lambda = lambda;
        if (fail >= 0) st.last_fail = fail;
        st.has_cand = cand;
    }
    __syncwarp();
}

// lm_update for slot `slot` of a launch described by p (candidate written to p.pose32); all
// 32 lanes of one warp call it.
__device__ inline void lm_step(const EpilogueParams& p, int slot, double* E, double* W, double min_valid, int lane) {
    const int hyp = p.active_idx[slot];
    lm_update(p.state[hyp], p.mode, p.solve_next, p.damping_mode, p.prior, E, W, min_valid,
              p.pose32 + 12 * hyp, p.eval_out ? p.eval_out + (size_t)slot * kNumSums : nullptr, lane);
}

}  // namespace pilot
