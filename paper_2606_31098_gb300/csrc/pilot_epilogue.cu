// Per-hypothesis FP64 epilogue of each build pass, and the small bookkeeping kernels.
//
//   tile sums     FP64 sum of the build pass' FP32 partial records, fixed tile order
//   gravity term  Eq. 3: r = R gamma^W - gamma^imu, J = [0 | -[a]x], a = R gamma^W
//   range term    Eq. 4-6: P = R^T (q - t), r = P_z - D(P_x, P_y), J = [-n | n x q]
//                 with n = R (-D_x, -D_y, 1) and q = d v
//   assembly      Supp. "Sensor-Prior Fusion in LM": H, g are sums over the terms
//   LM step       Eq. 8: (H + lambda I) dxi = -g by 6x6 Cholesky, Eq. 9: T' = exp(dxi) T
//   acceptance    keep T' iff its objective is lower and enough anchors stay visible
//   top-K         Supp. "Multi-Hypothesis Refinement": keep the K lowest objectives
//   selection     Sec. IV-E: argmin of the final objective over usable hypotheses
#include <math.h>

#include "pilot_internal.cuh"

namespace pilot {

namespace {

constexpr double kLambdaMin = 1e-12;
constexpr double kLambdaMax = 1e12;

__device__ __forceinline__ int tri_index(int a, int b) {
    // row-major upper triangle of a 6x6 matrix, a <= b
    return a * 6 - (a * (a - 1)) / 2 + (b - a);
}

__device__ void add_outer(double* E, const double* J, double r, double w) {
    int e = 0;
    for (int a = 0; a < 6; ++a)
        for (int b = a; b < 6; ++b) E[e++] += w * J[a] * J[b];
    for (int a = 0; a < 6; ++a) E[21 + a] += w * J[a] * r;
}

__device__ void huber64(double s, double delta, double* rho, double* drho) {
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
__device__ void add_gravity(const PriorParams& pp, const double* T, double* E) {
    double a[3];
    for (int i = 0; i < 3; ++i)
        a[i] = T[4 * i] * pp.g_world[0] + T[4 * i + 1] * pp.g_world[1] + T[4 * i + 2] * pp.g_world[2];
    const double r[3] = {a[0] - pp.g_cam[0], a[1] - pp.g_cam[1], a[2] - pp.g_cam[2]};
    double rho, drho;
    huber64(r[0] * r[0] + r[1] * r[1] + r[2] * r[2], pp.huber_grav, &rho, &drho);
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
__device__ void add_range(const PriorParams& pp, const double* T, double* E) {
    const double d[3] = {pp.q[0] - T[3], pp.q[1] - T[7], pp.q[2] - T[11]};
    double P[3];
    for (int i = 0; i < 3; ++i) P[i] = T[i] * d[0] + T[4 + i] * d[1] + T[8 + i] * d[2];  // R^T d
    const double gx = (P[0] - pp.dsm_x0) / pp.dsm_gsd - 0.5;
    const double gy = (P[1] - pp.dsm_y0) / pp.dsm_gsd - 0.5;
    if (!(gx >= 0.0 && gx <= pp.dsm_W - 1.0 && gy >= 0.0 && gy <= pp.dsm_H - 1.0)) return;
    const int c0 = min((int)gx, pp.dsm_W - 2), r0 = min((int)gy, pp.dsm_H - 2);
    const double ax = gx - c0, ay = gy - r0;
    const float* row0 = pp.dsm + (size_t)r0 * pp.dsm_W + c0;
    const float* row1 = row0 + pp.dsm_W;
    const double h00 = row0[0], h01 = row0[1], h10 = row1[0], h11 = row1[1];
    const double bx = h01 - h00, cy = h10 - h00, dxy = (h11 - h10) - bx;
    const double D = h00 + ax * (bx + dxy * ay) + ay * cy;
    const double Dx = (bx + dxy * ay) / pp.dsm_gsd, Dy = (cy + dxy * ax) / pp.dsm_gsd;
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
    huber64(r * r, pp.huber_range, &rho, &drho);
    add_outer(E, J, r, pp.w_range * drho);
    E[27] += pp.w_range * rho;
}

// (H + damping) x = -g by Cholesky; returns false if not positive definite.
__device__ bool damped_solve(const double* H21, const double* g, double lambda, int mode,
                             double* x) {
    double L[6][6];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j <= i; ++j) {
            double a = H21[tri_index(j, i)];
            if (i == j) a += (mode == 1) ? lambda * H21[tri_index(i, i)] : lambda;
            for (int k = 0; k < j; ++k) a -= L[i][k] * L[j][k];
            if (i == j) {
                if (!(a > 0.0)) return false;
                L[i][i] = sqrt(a);
            } else {
                L[i][j] = a / L[j][j];
            }
        }
    double y[6];
    for (int i = 0; i < 6; ++i) {
        double s = -g[i];
        for (int k = 0; k < i; ++k) s -= L[i][k] * y[k];
        y[i] = s / L[i][i];
    }
    for (int i = 5; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < 6; ++k) s -= L[k][i] * x[k];
        x[i] = s / L[i][i];
    }
    return true;
}

// T' = exp(xi) T with xi = (nu, omega):  Exp(w) = I + A K + B K^2,
// V = I + B K + C K^2, K = [w]x, K^2 = w w^T - th^2 I.
__device__ void pose_update(const double* xi, const double* T, double* Tn) {
    const double w0 = xi[3], w1 = xi[4], w2 = xi[5];
    const double th2 = w0 * w0 + w1 * w1 + w2 * w2;
    double A, B, Cc;
    if (th2 < 1e-12) {
        A = 1.0 - th2 / 6.0;
        B = 0.5 - th2 / 24.0;
        Cc = 1.0 / 6.0 - th2 / 120.0;
    } else {
        const double th = sqrt(th2);
        double sn, cs;
        sincos(th, &sn, &cs);
        A = sn / th;
        B = (1.0 - cs) / th2;
        Cc = (th - sn) / (th2 * th);
    }
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

__device__ void store_pose32(float* dst, const double* T) {
    for (int i = 0; i < 12; ++i) dst[i] = (float)T[i];
}

__global__ void epilogue_kernel(const EpilogueParams p, const double* min_valid_ptr) {
    const int slot = blockIdx.x;
    const int hyp = p.active_idx[slot];
    HypState& st = p.state[hyp];
    __shared__ double E[kNumSums];
    const bool evaluated = (p.mode == kEpiStep) ? (st.has_cand != 0) : true;
    const int lane = threadIdx.x;
    if (evaluated && lane < kNumSums) {
        const float* src = p.partial + (size_t)slot * p.n_tiles * kAcc + lane;
        double v = 0.0;
        for (int t = 0; t < p.n_tiles; ++t) v += (double)src[(size_t)t * kAcc];
        E[lane] = v;
    }
    __syncwarp();
    if (lane != 0) return;

    const double* Tev = (p.mode == kEpiStep) ? st.Tc : st.T;
    if (evaluated) {
        if (p.prior.use_gravity) add_gravity(p.prior, Tev, E);
        if (p.prior.use_range) add_range(p.prior, Tev, E);
    }
    if (p.mode == kEpiEval) {
        for (int i = 0; i < kNumSums; ++i) p.eval_out[(size_t)slot * kNumSums + i] = E[i];
        st.has_cand = 0;
        return;
    }
    const double min_valid = *min_valid_ptr;
    if (p.mode == kEpiInit) {
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
    if (p.solve_next) {
        double dxi[6];
        if (!damped_solve(st.H, st.g, st.lambda, p.damping_mode, dxi)) {
            st.lambda = fmin(st.lambda * 10.0, kLambdaMax);
            st.last_fail = 1;
        } else {
            st.last_fail = 0;
            pose_update(dxi, st.T, st.Tc);
            store_pose32(p.pose32 + 12 * hyp, st.Tc);
            st.has_cand = 1;
        }
    }
}

__global__ void hyp_init_kernel(HypState* st, const double* T_cw, int* active_idx, int M) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    HypState& s = st[m];
    for (int i = 0; i < 12; ++i) s.T[i] = s.Tc[i] = T_cw[12 * m + i];
    for (int i = 0; i < 21; ++i) s.H[i] = 0.0;
    for (int i = 0; i < 6; ++i) s.g[i] = 0.0;
    s.cost = 0.0;
    s.lambda = 0.0;
    s.n_valid = 0;
    s.has_cand = 0;
    s.last_fail = 0;
    s.active = 1;
    s.status = PILOT_HYP_OK;
    active_idx[m] = m;
}

__global__ void set_poses_kernel(HypState* st, float* pose32, const double* T_cw, int* active_idx,
                                 int M) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    for (int i = 0; i < 12; ++i) st[m].T[i] = T_cw[12 * m + i];
    store_pose32(pose32 + 12 * m, st[m].T);
    st[m].has_cand = 1;
    active_idx[m] = m;
}

__global__ void level_init_kernel(HypState* st, float* pose32, const int* active_idx, int n_active,
                                  double lambda0) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_active) return;
    const int m = active_idx[s];
    st[m].lambda = lambda0;
    st[m].last_fail = 0;
    st[m].has_cand = 1;
    store_pose32(pose32 + 12 * m, st[m].T);
}

__device__ __forceinline__ bool ranks_before(const HypState& a, int ia, const HypState& b, int ib,
                                             double min_valid) {
    // ordering key (unusable, cost, index); unusable = non-finite or too few visible
    const bool bad_a = !(isfinite(a.cost) && a.n_valid >= min_valid);
    const bool bad_b = !(isfinite(b.cost) && b.n_valid >= min_valid);
    if (bad_a != bad_b) return !bad_a;
    const double ca = isfinite(a.cost) ? a.cost : 0.0;
    const double cb = isfinite(b.cost) ? b.cost : 0.0;
    if (ca != cb) return ca < cb;
    return ia < ib;
}

// One block.  Ranks the active hypotheses, marks all but the K first as pruned, and
// writes the surviving indices, in increasing order, to active_out.
__global__ void prune_kernel(HypState* st, const int* active_in, int* active_out, int n, int K,
                             const double* min_valid_ptr) {
    const double min_valid = *min_valid_ptr;
    for (int s = threadIdx.x; s < n; s += blockDim.x) {
        const int m = active_in[s];
        int rank = 0;
        for (int s2 = 0; s2 < n; ++s2) {
            const int m2 = active_in[s2];
            rank += ranks_before(st[m2], m2, st[m], m, min_valid) ? 1 : 0;
        }
        if (rank >= K) {
            st[m].active = 0;
            st[m].status = PILOT_HYP_PRUNED;
        }
    }
    __syncthreads();
    for (int s = threadIdx.x; s < n; s += blockDim.x) {
        const int m = active_in[s];
        if (!st[m].active) continue;
        int pos = 0;
        for (int s2 = 0; s2 < s; ++s2) pos += st[active_in[s2]].active;
        active_out[pos] = m;
    }
}

// One block of 1024 threads: number of valid anchors (4 flags per load when aligned).
__global__ void count_valid_kernel(const uint8_t* valid, int N, double frac, double* min_valid) {
    __shared__ int part[32];
    int c = 0;
    if (!valid) {
        c = (threadIdx.x == 0) ? N : 0;
    } else if (((uintptr_t)valid & 3) == 0) {
        const uint32_t* w = reinterpret_cast<const uint32_t*>(valid);
        for (int k = threadIdx.x; k < N / 4; k += blockDim.x) {
            const uint32_t v = w[k];
            c += ((v & 0xffu) != 0) + ((v & 0xff00u) != 0) + ((v & 0xff0000u) != 0) + ((v >> 24) != 0);
        }
        for (int j = (N / 4) * 4 + threadIdx.x; j < N; j += blockDim.x) c += valid[j] != 0;
    } else {
        for (int j = threadIdx.x; j < N; j += blockDim.x) c += valid[j] != 0;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x < 32) {
        int v = (threadIdx.x < (blockDim.x >> 5)) ? part[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) *min_valid = frac * (double)v;
    }
}

// One block of 256 threads: final statuses, result block, argmin (ties -> lowest index).
__global__ void finalize_kernel(HypState* st, int M, const double* min_valid_ptr,
                                unsigned char* res, ResultLayout lay) {
    const double min_valid = *min_valid_ptr;
    double* T = reinterpret_cast<double*>(res + lay.off_T);
    double* cost = reinterpret_cast<double*>(res + lay.off_cost);
    int* nv = reinterpret_cast<int*>(res + lay.off_nvalid);
    int* status = reinterpret_cast<int*>(res + lay.off_status);
    int* best = reinterpret_cast<int*>(res + lay.off_best);
    __shared__ double bc[256];
    __shared__ int bi[256];
    double my_c = 0.0;
    int my_i = -1;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        HypState& s = st[m];
        if (s.active) {
            bool finite = isfinite(s.cost);
            for (int i = 0; i < 12; ++i) finite = finite && isfinite(s.T[i]);
            int code;
            if (!finite) code = PILOT_HYP_NONFINITE;
            else if (s.n_valid < min_valid) code = PILOT_HYP_FEW_VALID;
            else if (s.last_fail) code = PILOT_HYP_NOT_PD;
            else code = PILOT_HYP_OK;
            s.status = code;
        }
        for (int i = 0; i < 12; ++i) T[12 * m + i] = s.T[i];
        cost[m] = s.cost;
        nv[m] = s.n_valid;
        status[m] = s.status;
        if (s.status == PILOT_HYP_OK && (my_i < 0 || s.cost < my_c)) {
            my_c = s.cost;
            my_i = m;
        }
    }
    bc[threadIdx.x] = my_c;
    bi[threadIdx.x] = my_i;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const int j = threadIdx.x + s;
            const bool take = bi[j] >= 0 &&
                              (bi[threadIdx.x] < 0 || bc[j] < bc[threadIdx.x] ||
                               (bc[j] == bc[threadIdx.x] && bi[j] < bi[threadIdx.x]));
            if (take) {
                bc[threadIdx.x] = bc[j];
                bi[threadIdx.x] = bi[j];
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *best = bi[0];
}

}  // namespace

cudaError_t launch_epilogue(const EpilogueParams& p, const double* min_valid, cudaStream_t s) {
    if (p.n_active <= 0) return cudaSuccess;
    epilogue_kernel<<<p.n_active, 32, 0, s>>>(p, min_valid);
    return cudaGetLastError();
}

cudaError_t launch_hyp_init(HypState* st, const double* T_cw, int* active_idx, int M,
                            cudaStream_t s) {
    if (M <= 0) return cudaSuccess;
    hyp_init_kernel<<<(M + 127) / 128, 128, 0, s>>>(st, T_cw, active_idx, M);
    return cudaGetLastError();
}

cudaError_t launch_set_poses(HypState* st, float* pose32, const double* T_cw, int* active_idx,
                             int M, cudaStream_t s) {
    if (M <= 0) return cudaSuccess;
    set_poses_kernel<<<(M + 127) / 128, 128, 0, s>>>(st, pose32, T_cw, active_idx, M);
    return cudaGetLastError();
}

cudaError_t launch_level_init(HypState* st, float* pose32, const int* active_idx, int n_active,
                              double lambda0, cudaStream_t s) {
    if (n_active <= 0) return cudaSuccess;
    level_init_kernel<<<(n_active + 127) / 128, 128, 0, s>>>(st, pose32, active_idx, n_active, lambda0);
    return cudaGetLastError();
}

cudaError_t launch_prune(HypState* st, const int* active_in, int* active_out, int n_active,
                         int keep, const double* min_valid, cudaStream_t s) {
    prune_kernel<<<1, 1024, 0, s>>>(st, active_in, active_out, n_active, keep, min_valid);
    return cudaGetLastError();
}

cudaError_t launch_count_valid(const uint8_t* valid, int N, double frac, double* min_valid,
                               cudaStream_t s) {
    count_valid_kernel<<<1, 1024, 0, s>>>(valid, N, frac, min_valid);
    return cudaGetLastError();
}

cudaError_t launch_finalize(HypState* st, int M, const double* min_valid, unsigned char* result,
                            ResultLayout lay, cudaStream_t s) {
    finalize_kernel<<<1, 256, 0, s>>>(st, M, min_valid, result, lay);
    return cudaGetLastError();
}

}  // namespace pilot
