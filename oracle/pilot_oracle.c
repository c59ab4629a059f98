/*
 * FP64 CPU oracle of the featuremetric multi-hypothesis LM pose solver.
 *
 * TEST INFRASTRUCTURE ONLY: the plain, slow reference the CUDA path is checked
 * against.  Only tests, the smoke check and the benchmark's CPU-baseline leg load it.
 * Nothing here is shared with the CUDA library (no headers, helpers or tables).
 *
 * Everything is double precision and plain loops: the dense C x 6 Jacobian of every
 * anchor is formed explicitly and J^T W J is accumulated entry by entry, exactly as
 * Eq. 8 writes it.  The pieces follow the paper:
 *   Eq. 1  photo residual r = f^q(pi(K_l, T, P_j)) - f^r(p_j)
 *   Eq. 2  photo cost sum_j rho(w_l(j) ||r||^2)           (Huber rho)
 *   Eq. 3  gravity residual R gamma^W - gamma^imu           (R world->camera)
 *   Eq. 4  camera-centre ray v = K^-1 p_c / ||K^-1 p_c||
 *   Eq. 5  range point C + R_wc (d v)
 *   Eq. 6  range residual z - D(x, y)
 *   Eq. 7  total objective photo + lambda_imu rho(.) + lambda_range rho(.)
 *   Eq. 8  damped normal equation (J^T W J + lambda I) dxi = -J^T W r
 *   Eq. 9  left pose update T <- exp(dxi) T
 *   Supp. "Sensor-Prior Fusion in LM": H_total, g_total are sums of the three terms
 *   Sec. IV-E / Supp. "Multi-Hypothesis Refinement": independent hypotheses, optional
 *     top-K after a level, argmin of the final objective.
 *
 * Readings where the paper is silent (pixel convention, Huber on the squared norm,
 * damping schedule, accept/reject rule, world->camera state with a camera-frame left
 * update) are the ones the CUDA library documents; they are restated at each use.
 */
#include "pilot_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Z_NEAR 0.1
#define LAMBDA_MIN 1e-12
#define LAMBDA_MAX 1e12

/* ------------------------------------------------------------------ small helpers */

static void mat3_mul(const double A[9], const double B[9], double C[9]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
            C[3 * i + j] = s;
        }
}

static void hat(const double w[3], double K[9]) {
    /* [w]x such that [w]x v = w x v */
    K[0] = 0.0;   K[1] = -w[2]; K[2] = w[1];
    K[3] = w[2];  K[4] = 0.0;   K[5] = -w[0];
    K[6] = -w[1]; K[7] = w[0];  K[8] = 0.0;
}

static void pose_split(const double T[12], double R[9], double t[3]) {
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) R[3 * i + j] = T[4 * i + j];
        t[i] = T[4 * i + 3];
    }
}

static void pose_join(const double R[9], const double t[3], double T[12]) {
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) T[4 * i + j] = R[3 * i + j];
        T[4 * i + 3] = t[i];
    }
}

/* Upper triangle (row-major) index of H[a][b], a <= b. */
static int tri(int a, int b) {
    int idx = 0;
    for (int r = 0; r < a; ++r) idx += 6 - r;
    return idx + (b - a);
}

static void add_JtJ(double H[36], double g[6], const double* J, const double* r,
                    int rows, double weight) {
    /* H += weight * J^T J, g += weight * J^T r for a rows x 6 Jacobian J */
    for (int a = 0; a < 6; ++a) {
        for (int b = 0; b < 6; ++b) {
            double s = 0.0;
            for (int i = 0; i < rows; ++i) s += J[6 * i + a] * J[6 * i + b];
            H[6 * a + b] += weight * s;
        }
        double s = 0.0;
        for (int i = 0; i < rows; ++i) s += J[6 * i + a] * r[i];
        g[a] += weight * s;
    }
}

/* --------------------------------------------------------------------------- SE(3) */

void or_so3_exp(const double w[3], double R[9]) {
    /* Rodrigues: R = I + (sin th / th) K + ((1 - cos th) / th^2) K^2, K = [w]x;
     * second-order Taylor coefficients below th = 1e-6. */
    double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double th = sqrt(th2);
    double a, b;
    if (th < 1e-6) {
        a = 1.0 - th2 / 6.0;
        b = 0.5 - th2 / 24.0;
    } else {
        a = sin(th) / th;
        b = (1.0 - cos(th)) / th2;
    }
    double K[9], K2[9];
    hat(w, K);
    mat3_mul(K, K, K2);
    for (int i = 0; i < 9; ++i) R[i] = a * K[i] + b * K2[i];
    R[0] += 1.0; R[4] += 1.0; R[8] += 1.0;
}

static void so3_V(const double w[3], double V[9]) {
    /* V = I + ((1 - cos th) / th^2) K + ((th - sin th) / th^3) K^2 */
    double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double th = sqrt(th2);
    double b, c;
    if (th < 1e-6) {
        b = 0.5 - th2 / 24.0;
        c = 1.0 / 6.0 - th2 / 120.0;
    } else {
        b = (1.0 - cos(th)) / th2;
        c = (th - sin(th)) / (th2 * th);
    }
    double K[9], K2[9];
    hat(w, K);
    mat3_mul(K, K, K2);
    for (int i = 0; i < 9; ++i) V[i] = b * K[i] + c * K2[i];
    V[0] += 1.0; V[4] += 1.0; V[8] += 1.0;
}

void or_se3_exp(const double xi[6], double T[12]) {
    /* xi = (nu, omega), translation first: exp(xi) = [Exp(omega) | V(omega) nu] */
    double R[9], V[9], t[3];
    or_so3_exp(xi + 3, R);
    so3_V(xi + 3, V);
    for (int i = 0; i < 3; ++i) t[i] = V[3 * i] * xi[0] + V[3 * i + 1] * xi[1] + V[3 * i + 2] * xi[2];
    pose_join(R, t, T);
}

static int solve3(const double A_in[9], const double b_in[3], double x[3]) {
    /* Gaussian elimination with partial pivoting on a 3x3 system */
    double A[9], b[3];
    memcpy(A, A_in, sizeof A);
    memcpy(b, b_in, sizeof b);
    for (int k = 0; k < 3; ++k) {
        int p = k;
        for (int i = k + 1; i < 3; ++i)
            if (fabs(A[3 * i + k]) > fabs(A[3 * p + k])) p = i;
        if (A[3 * p + k] == 0.0) return 0;
        if (p != k) {
            for (int j = 0; j < 3; ++j) {
                double s = A[3 * k + j]; A[3 * k + j] = A[3 * p + j]; A[3 * p + j] = s;
            }
            double s = b[k]; b[k] = b[p]; b[p] = s;
        }
        for (int i = k + 1; i < 3; ++i) {
            double m = A[3 * i + k] / A[3 * k + k];
            for (int j = k; j < 3; ++j) A[3 * i + j] -= m * A[3 * k + j];
            b[i] -= m * b[k];
        }
    }
    for (int i = 2; i >= 0; --i) {
        double s = b[i];
        for (int j = i + 1; j < 3; ++j) s -= A[3 * i + j] * x[j];
        x[i] = s / A[3 * i + i];
    }
    return 1;
}

void or_se3_log(const double T[12], double xi[6]) {
    /* inverse of or_se3_exp for rotation angles below pi */
    double R[9], t[3];
    pose_split(T, R, t);
    double c = (R[0] + R[4] + R[8] - 1.0) / 2.0;
    if (c > 1.0) c = 1.0;
    if (c < -1.0) c = -1.0;
    double th = acos(c);
    double vee[3] = {R[7] - R[5], R[2] - R[6], R[3] - R[1]};
    double k = (th < 1e-6) ? 0.5 + th * th / 12.0 : th / (2.0 * sin(th));
    for (int i = 0; i < 3; ++i) xi[3 + i] = k * vee[i];
    double V[9];
    so3_V(xi + 3, V);
    solve3(V, t, xi);
}

void or_pose_update(const double xi[6], const double T[12], double Tout[12]) {
    /* Eq. 9 with the camera-frame reading: T' = exp(xi) T for T = T_cw */
    double E[12], Re[9], te[3], R[9], t[3], Rn[9], tn[3];
    or_se3_exp(xi, E);
    pose_split(E, Re, te);
    pose_split(T, R, t);
    mat3_mul(Re, R, Rn);
    for (int i = 0; i < 3; ++i)
        tn[i] = Re[3 * i] * t[0] + Re[3 * i + 1] * t[1] + Re[3 * i + 2] * t[2] + te[i];
    pose_join(Rn, tn, Tout);
}

/* --------------------------------------------------------------------------- Huber */

void or_huber(double s, double delta, double* rho, double* drho) {
    /* Huber applied to a squared argument s = w ||r||^2 (Eq. 2, Eq. 7):
     * rho(s) = s for s <= delta^2, else 2 delta sqrt(s) - delta^2; drho = d rho / d s. */
    double d2 = delta * delta;
    if (s <= d2) {
        *rho = s;
        *drho = 1.0;
    } else {
        double q = sqrt(s);
        *rho = 2.0 * delta * q - d2;
        *drho = delta / q;
    }
}

/* ------------------------------------------------------------------------ bilinear */

int or_bilinear(const float* map, int H, int W, int C, double x, double y,
                double* f, double* dfdx, double* dfdy) {
    /* Array coordinates: sample (r, c) sits at (x, y) = (c, r).  The cell is
     * (floor(x), floor(y)) clamped to (W-2, H-2); the interpolant's derivatives are
     * taken inside that cell. */
    if (!(x >= 0.0 && x <= W - 1.0 && y >= 0.0 && y <= H - 1.0)) return 0;
    int c0 = (int)floor(x), r0 = (int)floor(y);
    if (c0 > W - 2) c0 = W - 2;
    if (r0 > H - 2) r0 = H - 2;
    double ax = x - c0, ay = y - r0;
    const float* p00 = map + ((size_t)r0 * W + c0) * C;
    const float* p01 = map + ((size_t)r0 * W + c0 + 1) * C;
    const float* p10 = map + ((size_t)(r0 + 1) * W + c0) * C;
    const float* p11 = map + ((size_t)(r0 + 1) * W + c0 + 1) * C;
    for (int ch = 0; ch < C; ++ch) {
        double v00 = p00[ch], v01 = p01[ch], v10 = p10[ch], v11 = p11[ch];
        f[ch] = (1 - ax) * (1 - ay) * v00 + ax * (1 - ay) * v01 + (1 - ax) * ay * v10 + ax * ay * v11;
        dfdx[ch] = (1 - ay) * (v01 - v00) + ay * (v11 - v10);
        dfdy[ch] = (1 - ax) * (v10 - v00) + ax * (v11 - v01);
    }
    return 1;
}

/* ------------------------------------------------------------------ photo residual */

static void level_intrinsics(const or_frame* f, int level, double* fx, double* fy,
                             double* cx, double* cy) {
    /* K_l = diag(2^-l, 2^-l, 1) K_0 (Eq. 1: K scaled to level l) */
    double s = ldexp(1.0, -level);
    *fx = f->fx * s; *fy = f->fy * s; *cx = f->cx * s; *cy = f->cy * s;
}

int or_point_residual(const or_frame* f, int level, const double T[12], int j,
                      double* r, double* J) {
    if (f->point_valid && !f->point_valid[j]) return 0;
    const int C = f->C, N = f->N;
    double R[9], t[3];
    pose_split(T, R, t);
    double P[3] = {f->points[j], f->points[N + j], f->points[2 * N + j]};
    double p[3];
    for (int i = 0; i < 3; ++i) p[i] = R[3 * i] * P[0] + R[3 * i + 1] * P[1] + R[3 * i + 2] * P[2] + t[i];
    if (!(p[2] > Z_NEAR)) return 0;                   /* behind or too close: dropped */
    double fx, fy, cx, cy;
    level_intrinsics(f, level, &fx, &fy, &cx, &cy);
    double u = fx * p[0] / p[2] + cx;                   /* pinhole projection pi */
    double v = fy * p[1] / p[2] + cy;
    double fv[3 * C];
    double *df_du = fv + C, *df_dv = fv + 2 * C;
    /* pixel i covers [i, i+1): array coordinate = pixel coordinate - 1/2 */
    int vis = or_bilinear(f->qry_feat[level], f->H[level], f->W[level], C, u - 0.5, v - 0.5,
                          fv, df_du, df_dv);
    if (vis) {
        const float* ref = f->ref_feat[level] + (size_t)j * C;
        for (int ch = 0; ch < C; ++ch) r[ch] = fv[ch] - ref[ch];
        if (J) {
            /* d(u,v)/dp (2x3) times dp/ddelta = [I | -[p]x] (3x6) */
            double Jp[6] = {fx / p[2], 0.0, -fx * p[0] / (p[2] * p[2]),
                            0.0, fy / p[2], -fy * p[1] / (p[2] * p[2])};
            double Ph[9];
            hat(p, Ph);
            double D[18];
            for (int i = 0; i < 3; ++i)
                for (int k = 0; k < 3; ++k) {
                    D[6 * i + k] = (i == k) ? 1.0 : 0.0;
                    D[6 * i + 3 + k] = -Ph[3 * i + k];
                }
            double A[12];
            for (int a = 0; a < 2; ++a)
                for (int k = 0; k < 6; ++k) {
                    double s = 0.0;
                    for (int i = 0; i < 3; ++i) s += Jp[3 * a + i] * D[6 * i + k];
                    A[6 * a + k] = s;
                }
            for (int ch = 0; ch < C; ++ch)
                for (int k = 0; k < 6; ++k)
                    J[6 * ch + k] = df_du[ch] * A[k] + df_dv[ch] * A[6 + k];
        }
    }
    return vis;
}

double or_point_margin(const or_frame* f, int level, const double T[12], int j) {
    const int N = f->N;
    double R[9], t[3];
    pose_split(T, R, t);
    double P[3] = {f->points[j], f->points[N + j], f->points[2 * N + j]};
    double p[3];
    for (int i = 0; i < 3; ++i) p[i] = R[3 * i] * P[0] + R[3 * i + 1] * P[1] + R[3 * i + 2] * P[2] + t[i];
    if (fabs(p[2] - Z_NEAR) < 1e-3) return 0.0;
    if (!(p[2] > Z_NEAR)) return 1e30;
    double fx, fy, cx, cy;
    level_intrinsics(f, level, &fx, &fy, &cx, &cy);
    double x = fx * p[0] / p[2] + cx - 0.5;
    double y = fy * p[1] / p[2] + cy - 0.5;
    double mx = fabs(x - floor(x + 0.5)), my = fabs(y - floor(y + 0.5));
    return mx < my ? mx : my;
}

double or_query_confidence(const or_frame* f, int level, const double T[12], int j) {
    if (f->point_valid && !f->point_valid[j]) return 0.0;
    const int N = f->N;
    double R[9], t[3];
    pose_split(T, R, t);
    double P[3] = {f->points[j], f->points[N + j], f->points[2 * N + j]};
    double p[3];
    for (int i = 0; i < 3; ++i) p[i] = R[3 * i] * P[0] + R[3 * i + 1] * P[1] + R[3 * i + 2] * P[2] + t[i];
    if (!(p[2] > Z_NEAR)) return 0.0;
    double fx, fy, cx, cy;
    level_intrinsics(f, level, &fx, &fy, &cx, &cy);
    const double x = fx * p[0] / p[2] + cx - 0.5, y = fy * p[1] / p[2] + cy - 0.5;   /* array coordinates */
    if (!(x >= 0.0 && x <= f->W[level] - 1.0 && y >= 0.0 && y <= f->H[level] - 1.0)) return 0.0;
    if (!f->qry_conf[level]) return 1.0;
    double w, dwx, dwy;
    or_bilinear(f->qry_conf[level], f->H[level], f->W[level], 1, x, y, &w, &dwx, &dwy);
    return w;
}

void or_photo_terms(const or_frame* f, const or_config* c, int level, const double T[12],
                    double H21[21], double g6[6], double* cost, int* n_valid) {
    const int C = f->C;
    double H[36] = {0}, g[6] = {0}, total = 0.0;
    int n = 0;
    double* r = (double*)malloc(sizeof(double) * 7 * C);
    double* J = r + C;
    for (int j = 0; j < f->N; ++j) {
        if (!or_point_residual(f, level, T, j, r, J)) continue;
        double s = 0.0;
        for (int ch = 0; ch < C; ++ch) s += r[ch] * r[ch];
        double w = f->point_weight ? f->point_weight[j] : 1.0;
        if (f->qry_conf[level]) w *= or_query_confidence(f, level, T, j);
        double rho, drho;
        or_huber(w * s, c->huber_photo, &rho, &drho);
        total += rho;
        /* IRLS weight: d/ddelta rho(w ||r||^2) = 2 w rho' J^T r, so W = w rho' */
        add_JtJ(H, g, J, r, C, w * drho);
        ++n;
    }
    free(r);
    for (int a = 0; a < 6; ++a)
        for (int b = a; b < 6; ++b) H21[tri(a, b)] = H[6 * a + b];
    for (int a = 0; a < 6; ++a) g6[a] = g[a];
    *cost = total;
    *n_valid = n;
}

/* ------------------------------------------------------------------------- priors */

void or_gravity_residual(const or_frame* f, const double T[12], double r[3], double J[18]) {
    /* Eq. 3 with R = R_cw = R(T~)^T: r = R gamma^W - gamma^imu.
     * Under R <- Exp(omega) R, R gamma^W moves by -[R gamma^W]x omega. */
    double R[9], t[3], a[3];
    pose_split(T, R, t);
    for (int i = 0; i < 3; ++i)
        a[i] = R[3 * i] * f->gravity_world[0] + R[3 * i + 1] * f->gravity_world[1] +
               R[3 * i + 2] * f->gravity_world[2];
    for (int i = 0; i < 3; ++i) r[i] = a[i] - f->gravity_cam[i];
    if (J) {
        double Ah[9];
        hat(a, Ah);
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) {
                J[6 * i + k] = 0.0;
                J[6 * i + 3 + k] = -Ah[3 * i + k];
            }
    }
}

int or_gravity_terms(const or_frame* f, const or_config* c, const double T[12],
                     double H21[21], double g6[6], double* cost) {
    double r[3], J[18], H[36] = {0}, g[6] = {0};
    or_gravity_residual(f, T, r, J);
    double s = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    double rho, drho;
    if (c->gate_grav > 0.0 && s > c->gate_grav * c->gate_grav) {
        /* gated: constant cost at the gate, no pull on the pose */
        or_huber(c->gate_grav * c->gate_grav, c->huber_grav, &rho, &drho);
        for (int i = 0; i < 21; ++i) H21[i] = 0.0;
        for (int i = 0; i < 6; ++i) g6[i] = 0.0;
        *cost = f->w_grav * rho;
        return 1;
    }
    or_huber(s, c->huber_grav, &rho, &drho);
    add_JtJ(H, g, J, r, 3, f->w_grav * drho);
    for (int a = 0; a < 6; ++a)
        for (int b = a; b < 6; ++b) H21[tri(a, b)] = H[6 * a + b];
    for (int a = 0; a < 6; ++a) g6[a] = g[a];
    *cost = f->w_grav * rho;
    return 1;
}

int or_range_residual(const or_frame* f, const double T[12], double* r, double J[6]) {
    /* Eq. 4: v = K^-1 p_c / ||K^-1 p_c|| at the level-0 image centre p_c = (W0/2, H0/2).
     * Eq. 5: P_range = C + R_wc (d v) = R^T (d v - t).
     * Eq. 6: r = z_range - D(x_range, y_range), D bilinear on the DSM cell centres.
     * Under T <- exp(delta) T: dP/dnu = -R^T, dP/domega = R^T [q]x with q = d v. */
    double R[9], t[3];
    pose_split(T, R, t);
    double k[3] = {(0.5 * f->W[0] - f->cx) / f->fx, (0.5 * f->H[0] - f->cy) / f->fy, 1.0};
    double nk = sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
    double q[3], d[3], P[3];
    for (int i = 0; i < 3; ++i) q[i] = f->range_m * k[i] / nk;
    for (int i = 0; i < 3; ++i) d[i] = q[i] - t[i];
    for (int i = 0; i < 3; ++i) P[i] = R[i] * d[0] + R[3 + i] * d[1] + R[6 + i] * d[2];
    double gx = (P[0] - f->dsm_x0) / f->dsm_gsd - 0.5;
    double gy = (P[1] - f->dsm_y0) / f->dsm_gsd - 0.5;
    double D, dDx, dDy;
    if (!or_bilinear(f->dsm, f->dsm_H, f->dsm_W, 1, gx, gy, &D, &dDx, &dDy)) return 0;
    *r = P[2] - D;
    if (J) {
        double e[3] = {-dDx / f->dsm_gsd, -dDy / f->dsm_gsd, 1.0};   /* d r / d P */
        double Qh[9], RtQ[9];
        hat(q, Qh);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double s = 0.0;
                for (int l = 0; l < 3; ++l) s += R[3 * l + i] * Qh[3 * l + j];
                RtQ[3 * i + j] = s;
            }
        for (int kk = 0; kk < 6; ++kk) J[kk] = 0.0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                J[j] += e[i] * (-R[3 * j + i]);        /* (-R^T)_{ij} = -R[j][i] */
                J[3 + j] += e[i] * RtQ[3 * i + j];
            }
    }
    return 1;
}

int or_range_terms(const or_frame* f, const or_config* c, const double T[12],
                   double H21[21], double g6[6], double* cost) {
    double r, J[6], H[36] = {0}, g[6] = {0};
    for (int i = 0; i < 21; ++i) H21[i] = 0.0;
    for (int i = 0; i < 6; ++i) g6[i] = 0.0;
    *cost = 0.0;
    if (!or_range_residual(f, T, &r, J)) return 0;   /* off the DSM: term dropped */
    double rho, drho;
    if (c->gate_range > 0.0 && fabs(r) > c->gate_range) {
        /* gated: constant cost at the gate, no pull on the pose */
        or_huber(c->gate_range * c->gate_range, c->huber_range, &rho, &drho);
        *cost = f->w_range * rho;
        return 1;
    }
    or_huber(r * r, c->huber_range, &rho, &drho);
    add_JtJ(H, g, J, &r, 1, f->w_range * drho);
    for (int a = 0; a < 6; ++a)
        for (int b = a; b < 6; ++b) H21[tri(a, b)] = H[6 * a + b];
    for (int a = 0; a < 6; ++a) g6[a] = g[a];
    *cost = f->w_range * rho;
    return 1;
}

void or_evaluate(const or_frame* f, const or_config* c, int level, const double T[12],
                 double out29[29]) {
    /* Eq. 7 and the Supp. fused assembly: H = H_vis + H_range + H_grav (the weights
     * lambda_imu, lambda_range are already inside each prior's terms). */
    double H[21], g[6], cost;
    int n;
    or_photo_terms(f, c, level, T, H, g, &cost, &n);
    for (int i = 0; i < 21; ++i) out29[i] = H[i];
    for (int i = 0; i < 6; ++i) out29[21 + i] = g[i];
    out29[27] = cost;
    out29[28] = n;
    if (f->use_gravity) {
        or_gravity_terms(f, c, T, H, g, &cost);
        for (int i = 0; i < 21; ++i) out29[i] += H[i];
        for (int i = 0; i < 6; ++i) out29[21 + i] += g[i];
        out29[27] += cost;
    }
    if (f->use_range) {
        or_range_terms(f, c, T, H, g, &cost);
        for (int i = 0; i < 21; ++i) out29[i] += H[i];
        for (int i = 0; i < 6; ++i) out29[21 + i] += g[i];
        out29[27] += cost;
    }
}

/* ------------------------------------------------------------------------ Cholesky */

int or_cholesky_solve(const double A[36], const double b[6], double x[6]) {
    double L[36] = {0}, y[6];
    for (int i = 0; i < 6; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = A[6 * i + j];
            for (int k = 0; k < j; ++k) s -= L[6 * i + k] * L[6 * j + k];
            if (i == j) {
                if (!(s > 0.0)) return 0;
                L[6 * i + i] = sqrt(s);
            } else {
                L[6 * i + j] = s / L[6 * j + j];
            }
        }
    }
    for (int i = 0; i < 6; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= L[6 * i + k] * y[k];
        y[i] = s / L[6 * i + i];
    }
    for (int i = 5; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < 6; ++k) s -= L[6 * k + i] * x[k];
        x[i] = s / L[6 * i + i];
    }
    return 1;
}

/* ---------------------------------------------------------------------- LM driver */

static double min_valid_count(const or_frame* f, const or_config* c) {
    int n = 0;
    for (int j = 0; j < f->N; ++j) n += (!f->point_valid || f->point_valid[j]) ? 1 : 0;
    return c->min_valid_frac * n;
}

static void lm_level(const or_frame* f, const or_config* c, int level, double T[12],
                     double E[29], int* last_fail, double min_valid) {
    /* Levenberg-Marquardt at one pyramid level (Eq. 8, Eq. 9).  Each iteration:
     * solve (H + lambda I) dxi = -g; if not positive definite, raise lambda and count
     * the iteration; otherwise evaluate the objective at exp(dxi) T and accept the step
     * only if the cost drops (and enough anchors stay visible).  lambda moves by 10x,
     * clamped to [1e-12, 1e12], and restarts from lambda0 at every level. */
    double lambda = c->lambda0;
    or_evaluate(f, c, level, T, E);
    *last_fail = 0;
    for (int k = 0; k < c->iters[level]; ++k) {
        double A[36], b[6], dxi[6];
        for (int a = 0; a < 6; ++a) {
            for (int bb = a; bb < 6; ++bb) A[6 * a + bb] = A[6 * bb + a] = E[tri(a, bb)];
            b[a] = -E[21 + a];
        }
        for (int a = 0; a < 6; ++a)
            A[7 * a] += (c->damping_mode == 1) ? lambda * E[tri(a, a)] : lambda;
        if (!or_cholesky_solve(A, b, dxi)) {
            lambda = fmin(lambda * 10.0, LAMBDA_MAX);
            *last_fail = 1;
            continue;
        }
        *last_fail = 0;
        double Tn[12], En[29];
        or_pose_update(dxi, T, Tn);
        or_evaluate(f, c, level, Tn, En);
        if (En[27] < E[27] && En[28] >= min_valid) {
            memcpy(T, Tn, sizeof Tn);
            memcpy(E, En, sizeof En);
            lambda = fmax(lambda / 10.0, LAMBDA_MIN);
        } else {
            lambda = fmin(lambda * 10.0, LAMBDA_MAX);
        }
    }
}

void or_lm_level(const or_frame* f, const or_config* c, int level, double T[12],
                 double E29[29], int* last_solve_failed) {
    lm_level(f, c, level, T, E29, last_solve_failed, min_valid_count(f, c));
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

typedef struct { int bad; double cost; int idx; } rank_key;

static int rank_cmp(const void* pa, const void* pb) {
    const rank_key* a = (const rank_key*)pa;
    const rank_key* b = (const rank_key*)pb;
    if (a->bad != b->bad) return a->bad - b->bad;
    if (a->cost < b->cost) return -1;
    if (a->cost > b->cost) return 1;
    return a->idx - b->idx;
}

static int finite_pose(const double T[12]) {
    for (int i = 0; i < 12; ++i)
        if (!isfinite(T[i])) return 0;
    return 1;
}

int or_solve(const or_frame* f, const or_config* c, or_result* out, int n_threads) {
    const int M = f->M;
    if (M <= 0) {
        if (out->best) *out->best = -1;
        if (out->hyp_iters) *out->hyp_iters = 0;
        return 0;
    }
    const double min_valid = min_valid_count(f, c);
    double* T = out->T_cw;
    double* E = (double*)calloc((size_t)M * 29, sizeof(double));
    int* active = (int*)malloc(sizeof(int) * M);
    int* fail = (int*)calloc(M, sizeof(int));
    long long hyp_iters = 0;
    memcpy(T, f->T_cw, sizeof(double) * 12 * M);
    for (int m = 0; m < M; ++m) active[m] = 1;
#ifdef _OPENMP
    int nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#else
    (void)n_threads;
#endif
    for (int level = f->L - 1; level >= 0; --level) {
        int n_active = 0;
        for (int m = 0; m < M; ++m) n_active += active[m];
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
        for (int m = 0; m < M; ++m)
            if (active[m]) lm_level(f, c, level, T + 12 * m, E + 29 * m, fail + m, min_valid);
        hyp_iters += (long long)n_active * c->iters[level];
        int K = c->keep_top_k[level];
        if (level > 0 && K > 0 && K < n_active) {
            /* Supp. "Multi-Hypothesis Refinement": rank by the post-update objective,
             * keep the best K for the finer levels (unusable hypotheses rank last,
             * ties go to the lower index). */
            rank_key* keys = (rank_key*)malloc(sizeof(rank_key) * n_active);
            int n = 0;
            for (int m = 0; m < M; ++m)
                if (active[m]) {
                    double cost = E[29 * m + 27];
                    keys[n].bad = !(isfinite(cost) && E[29 * m + 28] >= min_valid);
                    keys[n].cost = isfinite(cost) ? cost : 0.0;
                    keys[n].idx = m;
                    ++n;
                }
            qsort(keys, n, sizeof(rank_key), rank_cmp);
            for (int i = K; i < n; ++i) {
                active[keys[i].idx] = 0;
                out->status[keys[i].idx] = OR_HYP_PRUNED;
            }
            free(keys);
        }
    }
    int best = -1;
    for (int m = 0; m < M; ++m) {
        out->cost[m] = E[29 * m + 27];
        out->n_valid[m] = (int)E[29 * m + 28];
        if (!active[m]) continue;     /* pruned: status already set */
        int st;
        if (!isfinite(E[29 * m + 27]) || !finite_pose(T + 12 * m)) st = OR_HYP_NONFINITE;
        else if (E[29 * m + 28] < min_valid) st = OR_HYP_FEW_VALID;
        else if (fail[m]) st = OR_HYP_NOT_PD;
        else st = OR_HYP_OK;
        out->status[m] = st;
        if (st == OR_HYP_OK && (best < 0 || E[29 * m + 27] < E[29 * best + 27])) best = m;
    }
    if (out->best) *out->best = best;
    if (out->hyp_iters) *out->hyp_iters = hyp_iters;
    free(E);
    free(active);
    free(fail);
    return 0;
}
