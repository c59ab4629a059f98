"""FP64 oracle of sequential tracking (TEST INFRASTRUCTURE ONLY: only tests/ and the
benchmark's CPU-baseline leg use it; the CUDA library never calls it).

What it computes, in the order of the online system (Supp. "Runtime Analysis"; Sec. V-A's
Failure Recovery Count protocol; Sec. IV-E and Supp. "Multi-Hypothesis Refinement" for the
seeds):

* ``predict``: the pose prior of a frame by constant-velocity propagation of the last two
  estimates, T_{k+s} = (T_k T_{k-1}^-1)^s T_k (world->camera poses; a body-frame constant
  velocity), or the last estimate held when only one exists;
* ``seed_grid``: the (x, y, psi) hypothesis grid around a prior: the camera centre moved by
  (x, y, 0) in the world and the camera turned about the world z axis through its centre by
  psi; x outermost, psi innermost;
* ``to_local`` / ``to_world``: poses in the metric frame of a reference crop, whose anchors
  are offsets from the crop origin o = (o_x, o_y, 0): t_local = t + R o;
* ``track``: the sequential loop.  Frame t's prior is ground truth at t = 0 and after a
  failure, else predict(est[t-1], est[t-2], 1).  Its reference crop is made around the same
  prior ("serial"), or, when the map preparation runs one frame ahead ("lookahead"), around
  the prior predicted two frames ahead from est[t-2] and est[t-3] (the estimates known
  before frame t-1 is localised).  A frame whose estimate is more than 20 m or 20 deg from
  ground truth counts one recovery; the next frame then starts from its ground truth pose
  (prior and crop), and the failed estimate is replaced by ground truth in the history.

Readings where the paper is silent: the propagation model (constant velocity), the
initial prior (ground truth), what the history holds after a recovery (ground truth),
and the map preparation's one-frame lead.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def _h(T) -> np.ndarray:
    """3x4 (or 12-vector) pose -> 4x4 homogeneous matrix."""
    M = np.eye(4)
    M[:3, :] = np.asarray(T, np.float64).reshape(3, 4)
    return M


def _inv(M: np.ndarray) -> np.ndarray:
    R, t = M[:3, :3], M[:3, 3]
    out = np.eye(4)
    out[:3, :3] = R.T
    out[:3, 3] = -R.T @ t
    return out


def predict(T_prev, T_prev2=None, steps: int = 1) -> np.ndarray:
    """Constant-velocity prediction `steps` frames after T_prev (12 values, world->camera).
    With T_prev2 (the estimate one frame before T_prev) the per-frame motion
    D = T_prev T_prev2^-1 is applied `steps` times on the left; without it T_prev is held."""
    if steps < 0:
        raise ValueError("steps must be >= 0")
    P = _h(T_prev)
    if T_prev2 is None:
        return P[:3, :].ravel().copy()
    D = P @ _inv(_h(T_prev2))
    out = P
    for _ in range(steps):
        out = D @ out
    return out[:3, :].ravel().copy()


def seed_grid(T_prior, grid_xy, grid_yaw_deg) -> np.ndarray:
    """The (x, y, psi) grid around a prior: (len(grid_xy)^2 * len(grid_yaw_deg), 12)."""
    P = _h(T_prior)
    R_cw = P[:3, :3]
    C = -R_cw.T @ P[:3, 3]
    out = []
    for gx in grid_xy:
        for gy in grid_xy:
            for gp in grid_yaw_deg:
                a = np.deg2rad(gp)
                Rz = np.array([[np.cos(a), -np.sin(a), 0.0], [np.sin(a), np.cos(a), 0.0], [0.0, 0.0, 1.0]])
                R_new = R_cw @ Rz.T                 # R_wc' = Rz R_wc
                C_new = C + np.array([gx, gy, 0.0])
                out.append(np.hstack([R_new, (-R_new @ C_new)[:, None]]).ravel())
    return np.array(out)


def to_local(T, origin) -> np.ndarray:
    """World->camera pose expressed for points given as offsets from (o_x, o_y, 0)."""
    P = _h(T)
    o = np.array([origin[0], origin[1], 0.0])
    P[:3, 3] = P[:3, 3] + P[:3, :3] @ o
    return P[:3, :].ravel()


def to_world(T_local, origin) -> np.ndarray:
    P = _h(T_local)
    o = np.array([origin[0], origin[1], 0.0])
    P[:3, 3] = P[:3, 3] - P[:3, :3] @ o
    return P[:3, :].ravel()


def pose_error(T_est, T_gt) -> tuple[float, float]:
    """(camera-centre distance in metres, rotation angle in degrees)."""
    A, B = _h(T_est), _h(T_gt)
    Ca = -A[:3, :3].T @ A[:3, 3]
    Cb = -B[:3, :3].T @ B[:3, 3]
    c = (np.trace(A[:3, :3].T @ B[:3, :3]) - 1.0) / 2.0
    return float(np.linalg.norm(Ca - Cb)), float(np.rad2deg(np.arccos(np.clip(c, -1.0, 1.0))))


@dataclass
class TrackLog:
    estimates: np.ndarray            # (n, 12) world->camera estimate of every frame
    priors: np.ndarray               # (n, 12) the prior the frame's seeds were made around
    crop_priors: np.ndarray          # (n, 12) the pose its reference crop was made around
    err_t: np.ndarray                # (n,) metres
    err_R: np.ndarray                # (n,) degrees
    failed: np.ndarray               # (n,) bool: error above the thresholds
    frc: int                         # failures counted (recoveries made)
    extra: list = field(default_factory=list)   # whatever localise() returned per frame


def crop_prior_lookahead(t: int, hist: list, T0) -> np.ndarray:
    """The crop pose for frame t when the map preparation runs one frame ahead: predicted
    two frames on from est[t-2] (and est[t-3]); frames 0 and 1 use the initial pose."""
    if t <= 1:
        return np.asarray(T0, np.float64).ravel().copy()
    return predict(hist[t - 2], hist[t - 3] if t >= 3 else None, 2)


def track(gt_poses, localise, mode: str = "serial", t_fail: float = 20.0, r_fail: float = 20.0) -> TrackLog:
    """Run the sequential loop over the ground-truth poses `gt_poses` (n, 12).

    ``localise(t, T_prior, T_crop)`` makes frame t's crop around T_crop, seeds hypotheses
    around T_prior, solves, and returns (T_estimate_world, extra).  `mode` is "serial" or
    "lookahead" (see the module docstring)."""
    if mode not in ("serial", "lookahead"):
        raise ValueError(mode)
    gt = np.asarray(gt_poses, np.float64).reshape(-1, 12)
    n = gt.shape[0]
    hist: list = []
    priors, crops, ests, et, er, failed, extra = [], [], [], [], [], [], []
    frc, reinit = 0, True
    for t in range(n):
        if reinit:
            prior = gt[t].copy()
        else:
            prior = predict(hist[t - 1], hist[t - 2] if t >= 2 else None, 1)
        if reinit or mode == "serial":
            crop = prior.copy()
        else:
            crop = crop_prior_lookahead(t, hist, gt[0])
        T_est, x = localise(t, prior, crop)
        T_est = np.asarray(T_est, np.float64).ravel()
        e_t, e_R = pose_error(T_est, gt[t])
        fail = e_t > t_fail or e_R > r_fail
        frc += int(fail)
        reinit = fail
        hist.append(gt[t].copy() if fail else T_est.copy())
        priors.append(prior)
        crops.append(crop)
        ests.append(T_est)
        et.append(e_t)
        er.append(e_R)
        failed.append(fail)
        extra.append(x)
    return TrackLog(np.array(ests), np.array(priors), np.array(crops), np.array(et), np.array(er),
                    np.array(failed), frc, extra)
