/*
 * FP64 CPU oracle of the featuremetric multi-hypothesis LM pose solver.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, obviously-correct reference
 * that the CUDA path is checked against.  Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it; the product path never does.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * Every quantity is computed in double precision with plain loops, in the order the
 * paper states it:
 *   photo residual       Eq. 1 (r = f^q(pi(K_l, T, P_j)) - f^r(p_j))
 *   photo cost           Eq. 2 (sum_j rho(w_l(j) ||r||^2))
 *   gravity residual     Eq. 3 (r = R gamma^W - gamma^imu, R world->camera)
 *   laser range          Eq. 4-6 (camera ray, range point, height residual)
 *   total objective      Eq. 7
 *   damped normal eq.    Eq. 8 ((J^T W J + lambda I) dxi = -J^T W r)
 *   pose update          Eq. 9 (T <- exp(dxi) T)
 *   fused H/g assembly   Supp. Sec. "Sensor-Prior Fusion in LM"
 *   hypotheses, top-K    Sec. IV-E and Supp. Sec. "Multi-Hypothesis Refinement"
 *
 * Parity status of each function is listed in its comment ("pinned by ...").
 */
#ifndef PILOT_ORACLE_H
#define PILOT_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define OR_MAX_LEVELS 4

/* Per-hypothesis final status. */
enum { OR_HYP_OK = 0, OR_HYP_FEW_VALID = 1, OR_HYP_NOT_PD = 2, OR_HYP_NONFINITE = 3,
       OR_HYP_PRUNED = 4 };

typedef struct {
    int N;                              /* anchors */
    const float* points;                /* 3 x N, SoA (x[], y[], z[]), local metric frame */
    const float* point_weight;          /* N or NULL (= 1): w_l(j) of Eq. 2 */
    const unsigned char* point_valid;   /* N or NULL (= all valid) */
    int C, L;                           /* channels, pyramid levels */
    const float* ref_feat[OR_MAX_LEVELS];   /* per level N x C */
    const float* qry_feat[OR_MAX_LEVELS];   /* per level H_l x W_l x C (NHWC) */
    const float* qry_conf[OR_MAX_LEVELS];   /* per level H_l x W_l query confidence w^q_l, or NULL (= 1) */
    int H[OR_MAX_LEVELS], W[OR_MAX_LEVELS];
    double fx, fy, cx, cy;              /* level-0 intrinsics, corner pixel convention */
    int M;                              /* hypotheses */
    const double* T_cw;                 /* M x 12, [R | t] row-major, world -> camera */
    int use_gravity;
    double gravity_cam[3];              /* gamma^imu */
    double gravity_world[3];            /* gamma^W */
    double w_grav;                      /* lambda_imu */
    int use_range;
    double range_m;                     /* d^range */
    double w_range;                     /* lambda_range */
    const float* dsm;                   /* dsm_H x dsm_W, row = y */
    int dsm_H, dsm_W;
    double dsm_x0, dsm_y0, dsm_gsd;     /* cell (r,c) centre = (x0+(c+.5)gsd, y0+(r+.5)gsd) */
} or_frame;

typedef struct {
    int iters[OR_MAX_LEVELS];           /* LM iterations at level l */
    double lambda0;
    int damping_mode;                   /* 0: + lambda I (Eq. 8); 1: + lambda diag(H) */
    double huber_photo, huber_grav, huber_range;
    int keep_top_k[OR_MAX_LEVELS];      /* applied after level l finishes; 0 = keep all */
    double min_valid_frac;
    /* residual gates of the sensor priors (Supp. "Sensor-Prior Fusion in LM": a prior whose
     * residual becomes excessively large is down-weighted): a residual norm above the gate
     * contributes the constant cost w rho(gate^2) and nothing to H and g (a truncated
     * Huber, continuous at the gate); 0 = no gate */
    double gate_grav, gate_range;
} or_config;

typedef struct {
    double* T_cw;       /* M x 12 final poses */
    double* cost;       /* M final objective (at the last level the hypothesis ran) */
    int* n_valid;       /* M */
    int* status;        /* M */
    int* best;          /* 1: argmin over OK hypotheses, -1 if none */
    long long* hyp_iters;  /* 1: sum over levels of active hypotheses x iterations */
} or_result;

/* ---- SE(3) (pinned by closed forms, scipy expm of the twist, log/exp round trip) ---- */
void or_so3_exp(const double w[3], double R[9]);
void or_se3_exp(const double xi[6], double T[12]);           /* xi = (nu, omega) */
void or_se3_log(const double T[12], double xi[6]);
void or_pose_update(const double xi[6], const double T[12], double Tout[12]);  /* exp(xi) T */

/* ---- Huber on a squared argument (pinned by continuity and finite differences) ---- */
void or_huber(double s, double delta, double* rho, double* drho);

/* ---- bilinear read of an H x W x C map at array coordinates (x, y) with its analytic
 *      derivatives (pinned exact on affine maps).  Returns 0 outside [0,W-1]x[0,H-1]. */
int or_bilinear(const float* map, int H, int W, int C, double x, double y,
                double* f, double* dfdx, double* dfdy);

/* ---- one anchor at one level: residual r (C) and dense Jacobian J (C x 6, row-major)
 *      w.r.t. the left perturbation T <- exp(delta) T.  Returns 1 if visible.
 *      (pinned by central finite differences of the residual) */
int or_point_residual(const or_frame* f, int level, const double T[12], int j,
                      double* r, double* J);

/* distance (pixels) of anchor j's sampling position to the nearest cell or visibility
 * boundary, and of Z to the near plane; used by the parity tests to set aside anchors
 * whose cell or visibility decision is ambiguous in FP32. */
double or_point_margin(const or_frame* f, int level, const double T[12], int j);

/* Query confidence w^q_l at anchor j's projection under T (bilinear in the level's
 * confidence map, the cell the features are read from); 1 without a map, 0 when the anchor
 * is not visible.  Its product with the anchor weight is the w_l(j) of Eq. 2; like the anchor
 * weight it is held constant when linearising (pinned by an affine confidence map and by a
 * constant map equalling a constant anchor weight). */
double or_query_confidence(const or_frame* f, int level, const double T[12], int j);

/* ---- objective pieces at pose T: H (21, upper triangle row-major), g (6), cost.
 *      (pinned: 2g == finite-difference gradient of cost, H == sum of FD Jacobians) */
void or_photo_terms(const or_frame* f, const or_config* c, int level, const double T[12],
                    double H21[21], double g6[6], double* cost, int* n_valid);
int  or_gravity_terms(const or_frame* f, const or_config* c, const double T[12],
                      double H21[21], double g6[6], double* cost);
int  or_range_terms(const or_frame* f, const or_config* c, const double T[12],
                    double H21[21], double g6[6], double* cost);
/* gravity residual (3) and range residual (1) on their own, for finite differences */
void or_gravity_residual(const or_frame* f, const double T[12], double r[3], double J[18]);
int  or_range_residual(const or_frame* f, const double T[12], double* r, double J[6]);

/* total: out29 = H(21) | g(6) | cost | n_valid (as double) */
void or_evaluate(const or_frame* f, const or_config* c, int level, const double T[12],
                 double out29[29]);

/* ---- 6x6 Cholesky solve A x = b.  Returns 0 if A is not positive definite. */
int or_cholesky_solve(const double A[36], const double b[6], double x[6]);

/* ---- the whole multi-hypothesis coarse-to-fine LM solve.  n_threads <= 0: all. */
int or_solve(const or_frame* f, const or_config* c, or_result* out, int n_threads);

/* ---- one level of LM for one hypothesis (exposed for sampled parity checks).
 *      T, lambda are updated in place; E29 receives the final evaluation. */
void or_lm_level(const or_frame* f, const or_config* c, int level, double T[12],
                 double E29[29], int* last_solve_failed);

int or_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
