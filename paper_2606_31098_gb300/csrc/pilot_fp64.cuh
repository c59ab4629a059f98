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

// Gravity direction prior (Eq. 3) at pose T, added to E = H21 | g6 | cost.
__device__ inline void add_gravity(const PriorParams& pp, const double* T, double* E) {
    double a[3];
    for (int i = 0; i < 3; ++i)
        a[i] = T[4 * i] * pp.g_world[0] + T[4 * i + 1] * pp.g_world[1] + T[4 * i + 2] * pp.g_world[2];
    const double r[3] = {a[0] - pp.g_cam[0], a[1] - pp.g_cam[1], a[2] - pp.g_cam[2]};
    double rho, drho;
    const double s = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    if (pp.gate_grav > 0.0 && s > pp.gate_grav * pp.gate_grav) {   // gated: constant, no pull
        huber64(pp.gate_grav * pp.gate_grav, pp.huber_grav, &rho, &drho);
        E[27] += pp.w_grav * rho;
        return;
    }
    huber64(s, pp.huber_grav, &rho, &drho);
    const double w = pp.w_grav * drho;
    // rotation block: w [a]x^T [a]x = w (|a|^2 I - a a^T); gradient: w [a]x r = w (a x r)
    const double aa = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
    for (int i = 0; i < 3; ++i)
        for (int k = i; k < 3; ++k) E[tri_index(3 + i, 3 + k)] += w * ((i == k ? aa : 0.0) - a[i] * a[k]);
    E[21 + 3] += w * (a[1] * r[2] - a[2] * r[1]);
    E[21 + 4] += w * (a[2] * r[0] - a[0] * r[2]);
    E[21 + 5] += w * (a[0] * r[1] - a[1] * r[0]);
    E[27] += pp.w_grav * rho;
}

// Laser range prior (Eq. 4-6) at pose T; dropped when the range point leaves the DSM.
__device__ inline void add_range(const PriorParams& pp, const double* T, double* E) {
    const double d[3] = {pp.q[0] - T[3], pp.q[1] - T[7], pp.q[2] - T[11]};
    double P[3];
    for (int i = 0; i < 3; ++i) P[i] = T[i] * d[0] + T[4 + i] * d[1] + T[8 + i] * d[2];  // R^T d
    const double inv_gsd = 1.0 / pp.dsm_gsd;
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
    // dr/dP = e = (-Dx, -Dy, 1); dP/ddelta = R^T [-I | [q]x]  =>  J = [-(R e) | (R e) x q]
    const double e[3] = {-Dx, -Dy, 1.0};
    double n[3];
    for (int i = 0; i < 3; ++i) n[i] = T[4 * i] * e[0] + T[4 * i + 1] * e[1] + T[4 * i + 2] * e[2];
    const double J[6] = {-n[0], -n[1], -n[2],
                         n[1] * pp.q[2] - n[2] * pp.q[1],
                         n[2] * pp.q[0] - n[0] * pp.q[2],
                         n[0] * pp.q[1] - n[1] * pp.q[0]};
    double rho, drho;
    if (pp.gate_range > 0.0 && fabs(r) > pp.gate_range) {          // gated: constant, no pull
        huber64(pp.gate_range * pp.gate_range, pp.huber_range, &rho, &drho);
        E[27] += pp.w_range * rho;
        return;
    }
    huber64(r * r, pp.huber_range, &rho, &drho);
    const double w = pp.w_range * drho;
    int k = 0;
    for (int a = 0; a < 6; ++a)
        for (int b = a; b < 6; ++b) E[k++] += w * J[a] * J[b];
    for (int a = 0; a < 6; ++a) E[21 + a] += w * J[a] * r;
    E[27] += pp.w_range * rho;
}

// (H + damping) x = -g by Cholesky (reciprocal pivots); false if not positive definite.
__device__ inline bool damped_solve(const double* H21, const double* g, double lambda, int mode,
                                    double* x) {
    double L[6][6], inv[6];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j <= i; ++j) {
            double a = H21[tri_index(j, i)];
            if (i == j) a += (mode == 1) ? lambda * H21[tri_index(i, i)] : lambda;
            for (int k = 0; k < j; ++k) a -= L[i][k] * L[j][k];
            if (i == j) {
                if (!(a > 0.0)) return false;
                L[i][i] = sqrt(a);
                inv[i] = 1.0 / L[i][i];
            } else {
                L[i][j] = a * inv[j];
            }
        }
    double y[6];
    for (int i = 0; i < 6; ++i) {
        double s = -g[i];
        for (int k = 0; k < i; ++k) s -= L[i][k] * y[k];
        y[i] = s * inv[i];
    }
    for (int i = 5; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < 6; ++k) s -= L[k][i] * x[k];
        x[i] = s * inv[i];
    }
    return true;
}

// Coefficients of Exp and V: A = sin(th)/th, B = (1 - cos th)/th^2, C = (th - sin th)/th^3.
// For th <= 0.25 rad (every LM step in practice) their Maclaurin series in x = th^2,
//   A = sum_k (-x)^k / (2k+1)!,  B = sum_k (-x)^k / (2k+2)!,  C = sum_k (-x)^k / (2k+3)!,
// are summed for k = 0..8 by Horner (the first omitted term is below 1e-27); larger
// angles use sin and cos.
__device__ inline void exp_coefficients(double x, double* A, double* B, double* C) {
    if (x <= 0.0625) {
        // reciprocal factorials 1/n!, n = 1..19
        constexpr double f[20] = {1.0, 1.0, 1.0 / 2, 1.0 / 6, 1.0 / 24, 1.0 / 120, 1.0 / 720, 1.0 / 5040,
                                  1.0 / 40320, 1.0 / 362880, 1.0 / 3628800, 1.0 / 39916800,
                                  1.0 / 479001600, 1.0 / 6227020800.0, 1.0 / 87178291200.0,
                                  1.0 / 1307674368000.0, 1.0 / 20922789888000.0,
                                  1.0 / 355687428096000.0, 1.0 / 6402373705728000.0,
                                  1.0 / 121645100408832000.0};
        double a = f[17], b = f[18], c = f[19];
        for (int k = 7; k >= 0; --k) {
            a = f[2 * k + 1] - x * a;
            b = f[2 * k + 2] - x * b;
            c = f[2 * k + 3] - x * c;
        }
        *A = a;
        *B = b;
        *C = c;
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
// V = I + B K + C K^2, K = [w]x, K^2 = w w^T - th^2 I.
__device__ inline void pose_update(const double* xi, const double* T, double* Tn) {
    const double w0 = xi[3], w1 = xi[4], w2 = xi[5];
    const double th2 = w0 * w0 + w1 * w1 + w2 * w2;
    double A, B, Cc;
    exp_coefficients(th2, &A, &B, &Cc);
    const double w[3] = {w0, w1, w2};
    const double K[3][3] = {{0.0, -w2, w1}, {w2, 0.0, -w0}, {-w1, w0, 0.0}};
    double Re[3][3], V[3][3];
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) {
            const double K2 = w[i] * w[k] - (i == k ? th2 : 0.0);
            const double I = (i == k) ? 1.0 : 0.0;
            Re[i][k] = I + A * K[i][k] + B * K2;
            V[i][k] = I + B * K[i][k] + Cc * K2;
        }
    for (int i = 0; i < 3; ++i) {
        for (int k = 0; k < 3; ++k)
            Tn[4 * i + k] = Re[i][0] * T[k] + Re[i][1] * T[4 + k] + Re[i][2] * T[8 + k];
        Tn[4 * i + 3] = Re[i][0] * T[3] + Re[i][1] * T[7] + Re[i][2] * T[11] +
                        V[i][0] * xi[0] + V[i][1] * xi[1] + V[i][2] * xi[2];
    }
}

__device__ __forceinline__ void store_pose32(float* dst, const double* T) {
    for (int i = 0; i < 12; ++i) dst[i] = (float)T[i];
}

// One hypothesis' FP64 step after a build pass at its candidate.  E (29 sums, photo term
// only on entry) gets the priors at the evaluated pose; then (init) it becomes the current
// state, or (step) the candidate is accepted or rejected; then the next candidate is
// solved for and, if cand32 is given, written there in FP32.  Single thread.
//
// Not inlined: every kernel of a translation unit (plain fused, batched, served) then runs
// the same compiled instructions, so the compiler cannot contract a * b + c into an FMA in
// one caller and not in another, and the forms stay bitwise equal.
static __device__ __noinline__ void lm_update(HypState& st, int mode, int solve_next, int damping_mode,
                                 const PriorParams& prior, double* E, double min_valid,
                                 float* cand32, double* eval_out) {
    const bool evaluated = (mode == kEpiStep) ? (st.has_cand != 0) : true;
    const double* Tev = (mode == kEpiStep) ? st.Tc : st.T;
    if (evaluated) {
        if (prior.use_gravity) add_gravity(prior, Tev, E);
        if (prior.use_range) add_range(prior, Tev, E);
    }
    if (mode == kEpiEval) {
        for (int i = 0; i < kNumSums; ++i) eval_out[i] = E[i];
        st.has_cand = 0;
        return;
    }
    if (mode == kEpiInit) {
        for (int i = 0; i < 21; ++i) st.H[i] = E[i];
        for (int i = 0; i < 6; ++i) st.g[i] = E[21 + i];
        st.cost = E[27];
        st.n_valid = (int)E[28];
    } else if (evaluated) {
        if (E[27] < st.cost && E[28] >= min_valid) {
            for (int i = 0; i < 12; ++i) st.T[i] = st.Tc[i];
            for (int i = 0; i < 21; ++i) st.H[i] = E[i];
            for (int i = 0; i < 6; ++i) st.g[i] = E[21 + i];
            st.cost = E[27];
            st.n_valid = (int)E[28];
            st.lambda = fmax(st.lambda / 10.0, kLambdaMin);
        } else {
            st.lambda = fmin(st.lambda * 10.0, kLambdaMax);
        }
    }
    st.has_cand = 0;
    if (solve_next) {
        double dxi[6];
        if (!damped_solve(st.H, st.g, st.lambda, damping_mode, dxi)) {
            st.lambda = fmin(st.lambda * 10.0, kLambdaMax);
            st.last_fail = 1;
        } else {
            st.last_fail = 0;
            pose_update(dxi, st.T, st.Tc);
            if (cand32) store_pose32(cand32, st.Tc);
            st.has_cand = 1;
        }
    }
}

// lm_update for slot `slot` of a launch described by p (candidate written to p.pose32).
__device__ inline void lm_step(const EpilogueParams& p, int slot, double* E, double min_valid) {
    const int hyp = p.active_idx[slot];
    lm_update(p.state[hyp], p.mode, p.solve_next, p.damping_mode, p.prior, E, min_valid,
              p.pose32 + 12 * hyp, p.eval_out ? p.eval_out + (size_t)slot * kNumSums : nullptr);
}

}  // namespace pilot
