// Sequential tracking pieces (Supp. "Runtime Analysis"; Sec. IV-E seeds).
//
// pilot_pose_predict   constant-velocity prior of the next frame from the last two
//                      estimates (host, FP64): T_{k+s} = (T_k T_{k-1}^-1)^s T_k
// pilot_pose_reorigin  a pose re-expressed for points given relative to (dx, dy, 0):
//                      t' = t + R (dx, dy, 0) (crop-local <-> world)
// pilot_seed_hypotheses  the (x, y, psi) grid around a prior, written straight into device
//                      memory as the solver's T_cw array (one thread per hypothesis, FP64):
//                      camera centre C + (x, y, 0), camera turned about world +z through its
//                      centre by psi (R_wc' = Rz(psi) R_wc), then re-origined to the crop.
#include <cuda_runtime.h>

#include <math.h>
#include <stdint.h>
#include <string.h>

#include "pilot_internal.cuh"

namespace pilot {
namespace {

constexpr double kDegToRad = 0.017453292519943295;   // pi / 180

struct SeedArgs {
    double R[9];      // prior R_cw
    double C[3];      // prior camera centre (world)
    double ox, oy;    // crop origin
    double xy[PILOT_MAX_SEED_XY];
    double yaw[PILOT_MAX_SEED_YAW];   // radians
    int n_xy, n_yaw;
};

__global__ void seed_kernel(const SeedArgs a, double* __restrict__ out) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int M = a.n_xy * a.n_xy * a.n_yaw;
    if (m >= M) return;
    const int k = m % a.n_yaw;
    const int iy = (m / a.n_yaw) % a.n_xy;
    const int ix = m / (a.n_yaw * a.n_xy);
    double s, c;
    sincos(a.yaw[k], &s, &c);
    // R' = R Rz^T: column j of R' mixes columns 0 and 1 of R; column 2 is unchanged
    double Rn[9];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const double r0 = a.R[3 * i], r1 = a.R[3 * i + 1];
        Rn[3 * i] = r0 * c - r1 * s;
        Rn[3 * i + 1] = r0 * s + r1 * c;
        Rn[3 * i + 2] = a.R[3 * i + 2];
    }
    // centre moved by (x, y, 0); the crop-local centre is that minus the origin
    const double Cl[3] = {a.C[0] + a.xy[ix] - a.ox, a.C[1] + a.xy[iy] - a.oy, a.C[2]};
    double* o = out + 12 * (size_t)m;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        o[4 * i] = Rn[3 * i];
        o[4 * i + 1] = Rn[3 * i + 1];
        o[4 * i + 2] = Rn[3 * i + 2];
        o[4 * i + 3] = -(Rn[3 * i] * Cl[0] + Rn[3 * i + 1] * Cl[1] + Rn[3 * i + 2] * Cl[2]);
    }
}

pilot_status track_fail(pilot_status st, const char* m) {
    record_error(m);
    return st;
}

// 4x4 helpers on 12-value [R | t] poses
void compose(const double* A, const double* B, double* out) {   // out = A B
    double r[12];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j)
            r[4 * i + j] = A[4 * i] * B[j] + A[4 * i + 1] * B[4 + j] + A[4 * i + 2] * B[8 + j];
        r[4 * i + 3] = A[4 * i] * B[3] + A[4 * i + 1] * B[7] + A[4 * i + 2] * B[11] + A[4 * i + 3];
    }
    memcpy(out, r, sizeof r);
}

void invert(const double* A, double* out) {                     // [R^T | -R^T t]
    double r[12];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) r[4 * i + j] = A[4 * j + i];
        r[4 * i + 3] = -(A[i] * A[3] + A[4 + i] * A[7] + A[8 + i] * A[11]);
    }
    memcpy(out, r, sizeof r);
}

bool finite12(const double* T) {
    for (int i = 0; i < 12; ++i)
        if (!isfinite(T[i])) return false;
    return true;
}

}  // namespace
}  // namespace pilot

using namespace pilot;

extern "C" pilot_status pilot_pose_predict(const double* T_prev, const double* T_prev2, int steps, double* T_out) {
    if (!T_prev || !T_out) return track_fail(PILOT_EINVAL, "T_prev or T_out is NULL");
    if (steps < 0) return track_fail(PILOT_EINVAL, "steps must be >= 0");
    if (!finite12(T_prev) || (T_prev2 && !finite12(T_prev2))) return track_fail(PILOT_EINVAL, "non-finite pose");
    double P[12];
    memcpy(P, T_prev, sizeof P);
    if (T_prev2) {
        double D[12], inv2[12];
        invert(T_prev2, inv2);
        compose(T_prev, inv2, D);
        for (int s = 0; s < steps; ++s) compose(D, P, P);
    }
    memcpy(T_out, P, sizeof P);
    return PILOT_OK;
}

extern "C" pilot_status pilot_pose_reorigin(const double* T, double dx, double dy, double* T_out) {
    if (!T || !T_out) return track_fail(PILOT_EINVAL, "T or T_out is NULL");
    double r[12];
    memcpy(r, T, sizeof r);
    for (int i = 0; i < 3; ++i) r[4 * i + 3] = T[4 * i + 3] + T[4 * i] * dx + T[4 * i + 1] * dy;
    memcpy(T_out, r, sizeof r);
    return PILOT_OK;
}

extern "C" pilot_status pilot_seed_hypotheses(const pilot_seed_params* p, double* T_out, void* stream) {
    if (!p || !T_out) return track_fail(PILOT_EINVAL, "params or T_out is NULL");
    if (p->n_xy < 1 || p->n_xy > PILOT_MAX_SEED_XY || p->n_yaw < 1 || p->n_yaw > PILOT_MAX_SEED_YAW)
        return track_fail(PILOT_EINVAL, "n_xy must be in [1, 32] and n_yaw in [1, 64]");
    if (((uintptr_t)T_out & 7) != 0) return track_fail(PILOT_EINVAL, "T_out must be 8-byte aligned");
    if (!finite12(p->T_prior) || !isfinite(p->origin_x) || !isfinite(p->origin_y))
        return track_fail(PILOT_EINVAL, "non-finite prior or origin");
    SeedArgs a{};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) a.R[3 * i + j] = p->T_prior[4 * i + j];
    for (int i = 0; i < 3; ++i)   // C = -R^T t
        a.C[i] = -(p->T_prior[i] * p->T_prior[3] + p->T_prior[4 + i] * p->T_prior[7] + p->T_prior[8 + i] * p->T_prior[11]);
    a.ox = p->origin_x;
    a.oy = p->origin_y;
    for (int i = 0; i < p->n_xy; ++i) a.xy[i] = p->grid_xy[i];
    for (int i = 0; i < p->n_yaw; ++i) a.yaw[i] = p->grid_yaw_deg[i] * kDegToRad;
    a.n_xy = p->n_xy;
    a.n_yaw = p->n_yaw;
    const int M = p->n_xy * p->n_xy * p->n_yaw;
    seed_kernel<<<(M + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(a, T_out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return track_fail(PILOT_ECUDA, cudaGetErrorString(e));
    return PILOT_OK;
}
