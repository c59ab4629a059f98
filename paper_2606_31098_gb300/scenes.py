"""Seeded synthetic scenes: the inputs both the CUDA solver and the CPU oracle read.

The paper evaluates on TDOM/DSM benchmarks and learned feature pyramids that are not
available here (Sec. III-B, Sec. V-A).  This module stands in for them with seeded
synthetic frames of the same structure:

* a DSM crop (sum of Gaussian hills plus box buildings) lifted to 3D geo-anchors
  P_j = (x_j, y_j, D(x_j, y_j)), one per crop cell (Supp. "Geo-anchor Construction");
* a 3-level query feature pyramid with C channels, L2-normalised per pixel
  (Supp. "Network Architecture": descriptors are L2-normalised along channels);
* reference descriptors f_l^r(p_j) obtained by reading the query pyramid at the
  ground-truth projection of each anchor, plus Gaussian noise;
* pose hypotheses in (x, y, yaw) around the ground truth (Sec. IV-E), an IMU gravity
  measurement (Eq. 3) and a single-point laser range along the optical axis (Eq. 4-6).

This module only *synthesises data*.  It contains none of the solver: no residual,
Jacobian, robust weight, normal equation or pose update.  The ground-truth rendering
of reference descriptors uses a 3x4 projection matrix and scipy's
``ndimage.map_coordinates`` (order 1), i.e. an implementation independent of both the
oracle and the CUDA path, so that "the oracle's cost vanishes at the ground truth" is
a real check of the oracle's projection and sampling conventions.

Conventions (shared by every consumer of these arrays):
  * world frame ENU (x east, y north, z up), gravity direction gamma^W = (0, 0, -1);
  * camera frame x right, y down, z forward; a pose is T_cw = [R | t] (world->camera),
    stored row-major as 12 float64 values;
  * pixel i covers [i, i+1) (corner convention); the principal point of level 0 is
    (W0/2, H0/2) and level l uses K scaled by 2^-l;
  * DSM cell (r, c) is centred at (x0 + (c + 1/2) gsd, y0 + (r + 1/2) gsd);
  * every coordinate is expressed in the frame's local metric frame whose origin is the
    crop centre (the map origin is not needed by the solver).
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field

import numpy as np
from scipy import ndimage
from scipy.spatial.transform import Rotation


GRAVITY_WORLD = np.array([0.0, 0.0, -1.0])


@dataclass
class SceneConfig:
    """Recipe of one synthetic frame.  Defaults follow the 256^2-crop, C=32 workload."""

    crop_side: int = 256                  # anchors per crop side (N = crop_side^2)
    gsd: float = 0.5                      # metres per DSM cell
    n_hills: int = 8
    hill_sigma: float = 10.0              # metres
    hill_amp: tuple = (0.0, 15.0)         # metres
    n_boxes: int = 4
    box_height: tuple = (5.0, 40.0)       # metres
    box_side: tuple = (6.0, 16.0)         # metres
    channels: int = 32
    levels: tuple = ((480, 640), (240, 320), (120, 160))   # (H, W), level 0 finest
    f0: float = 600.0                     # level-0 focal length in pixels (fx = fy)
    blur_sigma: float = 2.0               # pixels, at each level's own resolution
    n_blobs: int = 8                      # Gaussian blobs per channel
    blob_sigma: tuple = (6.0, 20.0)       # pixels
    blob_amp: tuple = (-2.0, 2.0)
    altitude: tuple = (120.0, 300.0)      # camera height above the datum, metres
    pitch_deg: tuple = (30.0, 70.0)       # depression of the optical axis below horizon
    ref_noise: float = 0.01               # std of the noise added to reference descriptors
    n_hyps: int = 64
    hyp_mode: str = "xy_yaw"              # "xy_yaw": U(+-dxy, +-dxy, +-dyaw); "rot_trans": exact angle/offset;
                                          # "grid": grid_xy^2 x grid_yaw_deg around a perturbed prior
    hyp_xy: float = 10.0                  # metres
    hyp_yaw_deg: float = 5.0              # degrees
    hyp_rot_deg: float = 3.0              # rot_trans mode: rotation angle about a random axis
    hyp_trans: float = 5.0                # rot_trans mode: translation length
    # grid mode: the (x, y, yaw) grid of Supp. "Multi-Hypothesis Refinement" around a prior
    grid_xy: tuple = tuple(float(v) for v in range(-10, 11, 2))      # metres, x and y
    grid_yaw_deg: tuple = (-9.0, -7.0, -5.0, -3.0, -1.0, 1.0, 3.0, 5.0, 7.0, 9.0)
    prior_xy: float = 4.0                 # prior = GT shifted by U(+-prior_xy) in x and y
    prior_yaw_deg: float = 4.0            # ... and rotated by U(+-prior_yaw_deg) in yaw
    prior_ring: tuple | None = None       # (lo, hi): instead, |dxy| ~ U(lo, hi) m in a uniform
                                          # direction and |dyaw| ~ U(lo, hi) deg with a random sign
    n_anchors: int = 0                    # > 0: sample this many valid anchors of the crop
    use_gravity: bool = True
    gravity_noise_deg: float = 0.2
    w_grav: float = 1e2
    use_range: bool = True
    range_noise: float = 0.1              # metres
    w_range: float = 1e1


def config_small_plain() -> SceneConfig:
    """Plain single frame: 64x64 DSM at 1 m, C=16, one 120x160 level, 1 hypothesis
    perturbed by exactly 3 deg / 5 m, no priors (the small parity workload)."""
    return SceneConfig(crop_side=64, gsd=1.0, box_height=(5.0, 30.0), channels=16,
                       levels=((120, 160),), f0=150.0, altitude=(150.0, 150.0),
                       pitch_deg=(45.0, 45.0), n_hyps=1, hyp_mode="rot_trans",
                       use_gravity=False, use_range=False)


def config_full_frame(n_hyps: int = 64) -> SceneConfig:
    """Full single frame: 256x256 crop at 0.5 m, C=32, 3 levels 480x640/240x320/120x160,
    fx=600, 64 hypotheses within +-10 m / +-5 deg, gravity and range priors on."""
    return SceneConfig(n_hyps=n_hyps)


def config_paper_schedule(n_anchors: int = 500, crop_side: int = 256) -> SceneConfig:
    """The paper's own refinement schedule (Sec. V-A "Implementation Details", Supp.
    "Multi-Hypothesis Refinement"): 500 geo-anchors sampled from the crop, the 1210
    hypotheses of the 11 x 11 (x, y) grid (+-10 m, 2 m steps) times 10 yaw offsets
    (+-1, 3, 5, 7, 9 deg) around a prior pose, images resized to 512 px (levels 384x512 /
    192x256 / 96x128, focal length scaled so the field of view stays that of the full
    frame).  The solve keeps the best 128 after the coarse level and runs 2 / 3 / 4
    iterations from coarse to fine."""
    return SceneConfig(crop_side=crop_side, levels=((384, 512), (192, 256), (96, 128)),
                       f0=600.0 * 512.0 / 640.0, hyp_mode="grid", n_anchors=n_anchors)


def config_seeding_ablation() -> SceneConfig:
    """The paper's schedule with the prior drawn at 5-15 m horizontal offset and 5-15 deg
    yaw offset (the pose-prior uncertainty of Sec. V-A's data: 5-15 m, 5-15 deg), for the
    synthetic analogue of the seeding ablation (Supp. "Effect of Multi-hypothesis
    Sampling"; hypotheses from seeding_hypotheses)."""
    cfg = config_paper_schedule()
    cfg.prior_ring = (5.0, 15.0)
    return cfg


def config_reduced_frame(crop_side: int = 90, n_hyps: int = 6, channels: int = 32,
                         levels=((240, 320), (120, 160), (60, 80)), f0: float = 600.0,
                         gsd: float = 1.0) -> SceneConfig:
    """The full-frame recipe shrunk so that the FP64 oracle finishes in seconds, while
    still spanning several point tiles and a ragged tail (90^2 = 8100 anchors).  The
    focal length stays that of the full frame (600 px at the finest level), so a pixel
    subtends the same angle and the pose is as well conditioned per anchor; with fewer
    anchors the weakest direction of the FP32 objective flattens toward the 1 mm parity
    tolerance, which 90^2 anchors keep well clear of."""
    return SceneConfig(crop_side=crop_side, gsd=gsd, channels=channels, levels=levels,
                       f0=f0, n_hyps=n_hyps)


@dataclass
class Frame:
    """One synthetic frame.  Arrays are C-contiguous numpy arrays."""

    points: np.ndarray            # (3, N) float32, SoA: x, y, z in the local frame
    point_valid: np.ndarray       # (N,) uint8
    point_weight: np.ndarray      # (N,) float32 (ones)
    ref_feat: list                # L arrays (N, C) float32
    qry_feat: list                # L arrays (H_l, W_l, C) float32, NHWC
    fx: float
    fy: float
    cx: float
    cy: float
    T_hyps: np.ndarray            # (M, 12) float64, rows [R | t] row-major
    T_gt: np.ndarray              # (12,) float64
    use_gravity: bool
    gravity_cam: np.ndarray       # (3,)
    gravity_world: np.ndarray     # (3,)
    w_grav: float
    use_range: bool
    range_m: float
    w_range: float
    dsm: np.ndarray               # (H_D, W_D) float32
    dsm_x0: float
    dsm_y0: float
    dsm_gsd: float
    seed: int = 0
    meta: dict = field(default_factory=dict)
    qry_conf: list | None = None  # L arrays (H_l, W_l) float32 query confidence w^q_l, or None

    @property
    def N(self) -> int:
        return self.points.shape[1]

    @property
    def M(self) -> int:
        return self.T_hyps.shape[0]

    @property
    def C(self) -> int:
        return self.qry_feat[0].shape[2]

    @property
    def L(self) -> int:
        return len(self.qry_feat)

    def replace(self, **kw) -> "Frame":
        return dataclasses.replace(self, **kw)


# ----------------------------------------------------------------------------- DSM

def _make_dsm(cfg: SceneConfig, rng: np.random.Generator):
    S, gsd = cfg.crop_side, cfg.gsd
    half = 0.5 * S * gsd
    x0 = y0 = -half
    xs = x0 + (np.arange(S) + 0.5) * gsd
    ys = y0 + (np.arange(S) + 0.5) * gsd
    X, Y = np.meshgrid(xs, ys)                       # row = y, column = x
    Z = np.zeros((S, S))
    for _ in range(cfg.n_hills):
        cx_, cy_ = rng.uniform(-half, half, 2)
        amp = rng.uniform(*cfg.hill_amp)
        Z += amp * np.exp(-((X - cx_) ** 2 + (Y - cy_) ** 2) / (2 * cfg.hill_sigma ** 2))
    for _ in range(cfg.n_boxes):
        cx_, cy_ = rng.uniform(-half, half, 2)
        sx, sy = rng.uniform(*cfg.box_side, 2)
        h = rng.uniform(*cfg.box_height)
        inside = (np.abs(X - cx_) <= sx / 2) & (np.abs(Y - cy_) <= sy / 2)
        Z = np.where(inside, np.maximum(Z, h), Z)
    return Z.astype(np.float32), x0, y0, X, Y


def dsm_height(dsm: np.ndarray, x0: float, y0: float, gsd: float, x, y):
    """Bilinear DSM height at world (x, y) via scipy (cell centres at x0 + (c+1/2) gsd).
    Outside the raster the nearest edge value is used (only for ground-truth synthesis)."""
    cc = (np.asarray(x, float) - x0) / gsd - 0.5
    rr = (np.asarray(y, float) - y0) / gsd - 0.5
    return ndimage.map_coordinates(dsm.astype(np.float64), [np.atleast_1d(rr), np.atleast_1d(cc)],
                                   order=1, mode="nearest")


# ------------------------------------------------------------------------ features

def _make_feature_map(H: int, W: int, C: int, cfg: SceneConfig, rng: np.random.Generator):
    maps = np.empty((H, W, C), np.float64)
    yy = np.arange(H) + 0.5
    xx = np.arange(W) + 0.5
    for c in range(C):
        m = ndimage.gaussian_filter(rng.standard_normal((H, W)), cfg.blur_sigma, mode="reflect")
        for _ in range(cfg.n_blobs):
            bx, by = rng.uniform(0, W), rng.uniform(0, H)
            s = rng.uniform(*cfg.blob_sigma)
            a = rng.uniform(*cfg.blob_amp)
            m += a * np.outer(np.exp(-(yy - by) ** 2 / (2 * s * s)),
                              np.exp(-(xx - bx) ** 2 / (2 * s * s)))
        maps[:, :, c] = m
    maps /= np.linalg.norm(maps, axis=2, keepdims=True) + 1e-12
    return maps.astype(np.float32)


# ---------------------------------------------------------------------------- pose

def look_pose(C_world: np.ndarray, yaw: float, pitch: float) -> np.ndarray:
    """World->camera pose (12 values) of a camera at C_world heading `yaw` (radians from
    east, counter-clockwise) with its optical axis `pitch` radians below the horizon."""
    h = np.array([np.cos(yaw), np.sin(yaw), 0.0])
    d = np.cos(pitch) * h + np.sin(pitch) * np.array([0.0, 0.0, -1.0])
    right = np.array([np.sin(yaw), -np.cos(yaw), 0.0])
    down = np.cross(d, right)
    R_wc = np.stack([right, down, d], axis=1)        # columns: camera axes in world
    R_cw = R_wc.T
    t = -R_cw @ C_world
    return np.concatenate([np.hstack([R_cw, t[:, None]]).ravel()])


def pose_parts(T: np.ndarray):
    T = np.asarray(T, float).reshape(3, 4)
    return T[:, :3], T[:, 3]


def camera_centre(T: np.ndarray) -> np.ndarray:
    R, t = pose_parts(T)
    return -R.T @ t


def compose_pose(R_cw: np.ndarray, C_world: np.ndarray) -> np.ndarray:
    t = -R_cw @ C_world
    return np.hstack([R_cw, t[:, None]]).ravel()


def _perturb_xy_yaw(T_gt, dx, dy, dyaw):
    """Shift the camera centre by (dx, dy, 0) and rotate it about the world z axis
    through the camera centre by dyaw (the (x, y, psi) hypothesis space, Sec. IV-E)."""
    R, _ = pose_parts(T_gt)
    C = camera_centre(T_gt)
    Rz = Rotation.from_rotvec([0.0, 0.0, dyaw]).as_matrix()
    R_wc = Rz @ R.T
    return compose_pose(R_wc.T, C + np.array([dx, dy, 0.0]))


def _perturb_rot_trans(T_gt, axis, angle, direction, length):
    R, _ = pose_parts(T_gt)
    C = camera_centre(T_gt)
    Rw = Rotation.from_rotvec(axis * angle).as_matrix()
    R_wc = Rw @ R.T
    return compose_pose(R_wc.T, C + direction * length)


def _unit(rng):
    v = rng.standard_normal(3)
    return v / np.linalg.norm(v)


# -------------------------------------------------------------------- ground truth

def project_gt(points_xyz: np.ndarray, T: np.ndarray, f: float, cx: float, cy: float):
    """Ground-truth pixel coordinates of world points via the 3x4 matrix K [R | t]."""
    P = np.array([[f, 0.0, cx], [0.0, f, cy], [0.0, 0.0, 1.0]]) @ np.asarray(T, float).reshape(3, 4)
    Xh = np.vstack([points_xyz.astype(np.float64), np.ones((1, points_xyz.shape[1]))])
    uvw = P @ Xh
    return uvw[0] / uvw[2], uvw[1] / uvw[2], uvw[2]


def read_map(fmap: np.ndarray, u: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Read an (H, W, C) map at continuous pixel coordinates (corner convention) with
    scipy's linear interpolation.  Returns (len(u), C) float64."""
    coords = [v - 0.5, u - 0.5]
    out = np.empty((u.size, fmap.shape[2]))
    for c in range(fmap.shape[2]):
        out[:, c] = ndimage.map_coordinates(fmap[:, :, c].astype(np.float64), coords,
                                            order=1, mode="nearest")
    return out


def _point_height(dsm: np.ndarray, x0: float, y0: float, gsd: float, x: float, y: float) -> float:
    """Bilinear DSM height at one world point (cell centres at x0 + (c+1/2) gsd), clamped to
    the raster like dsm_height; reads only the four cells it needs."""
    H, W = dsm.shape
    c = min(max((x - x0) / gsd - 0.5, 0.0), W - 1.0)
    r = min(max((y - y0) / gsd - 0.5, 0.0), H - 1.0)
    c0, r0 = min(int(c), W - 2), min(int(r), H - 2)
    ax, ay = c - c0, r - r0
    t = dsm[r0:r0 + 2, c0:c0 + 2].astype(np.float64)
    return float((1 - ay) * ((1 - ax) * t[0, 0] + ax * t[0, 1]) + ay * ((1 - ax) * t[1, 0] + ax * t[1, 1]))


def _ray_to_dsm(C, d, dsm, x0, y0, gsd, step=0.05, s_max=5000.0, pointwise=False):
    """Distance along the ray C + s d to its first crossing of the bilinear DSM surface
    (march, then bisection to 1e-9 m).  pointwise=True reads four cells per sample (for
    large maps) instead of scipy's interpolation of the whole raster."""
    def above(s):
        p = C + s * d
        if pointwise:
            return p[2] - _point_height(dsm, x0, y0, gsd, p[0], p[1])
        return p[2] - dsm_height(dsm, x0, y0, gsd, p[0], p[1])[0]

    s_lo, s = 0.0, step
    f_lo = above(0.0)
    if f_lo <= 0:
        raise ValueError("camera below the surface")
    while s < s_max:
        if above(s) <= 0:
            break
        s_lo, s = s, s + step
    else:
        raise ValueError("ray does not reach the surface")
    lo, hi = s_lo, s
    while hi - lo > 1e-9:
        mid = 0.5 * (lo + hi)
        if above(mid) > 0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def _rays_to_dsm(Cs, ds, dsm, x0, y0, gsd, step=0.25, s_max=5000.0):
    """_ray_to_dsm for many rays at once (Cs, ds: (K, 3)): each ray starts where it drops
    below the map's highest cell (no crossing before that), marches in lockstep with the
    others, then bisects to 1e-9 m.  Bilinear DSM between cell centres, clamped to the raster."""
    Cs, ds = np.asarray(Cs, np.float64), np.asarray(ds, np.float64)
    H, W = dsm.shape
    D = dsm.astype(np.float64)

    def above(idx, s_arr):
        p = Cs[idx] + s_arr[:, None] * ds[idx]
        c = np.clip((p[:, 0] - x0) / gsd - 0.5, 0.0, W - 1.0)
        r = np.clip((p[:, 1] - y0) / gsd - 0.5, 0.0, H - 1.0)
        c0 = np.minimum(c.astype(np.int64), W - 2)
        r0 = np.minimum(r.astype(np.int64), H - 2)
        ax, ay = c - c0, r - r0
        h = ((1 - ay) * ((1 - ax) * D[r0, c0] + ax * D[r0, c0 + 1]) + ay * ((1 - ax) * D[r0 + 1, c0] + ax * D[r0 + 1, c0 + 1]))
        return p[:, 2] - h

    K = Cs.shape[0]
    lo = np.maximum((Cs[:, 2] - float(D.max()) - 1.0) / np.maximum(-ds[:, 2], 1e-12), 0.0)
    hi = np.full(K, np.nan)
    todo = np.arange(K)
    while todo.size:
        s_new = lo[todo] + step
        f = above(todo, s_new)
        hit = f <= 0
        hi[todo[hit]] = s_new[hit]
        lo[todo[~hit]] = s_new[~hit]
        todo = todo[~hit & (s_new < s_max)]
    if np.isnan(hi).any():
        raise ValueError("a ray does not reach the surface")
    lo = hi - step
    idx = np.arange(K)
    while np.max(hi - lo) > 1e-9:
        mid = 0.5 * (lo + hi)
        up = above(idx, mid) > 0
        lo = np.where(up, mid, lo)
        hi = np.where(up, hi, mid)
    return 0.5 * (lo + hi)


# ------------------------------------------------------------------------- frames

def make_frame(cfg: SceneConfig, seed: int) -> Frame:
    """Build one seeded frame from `cfg`.  Independent sub-streams (SeedSequence children)
    drive the DSM, each pyramid level, the pose, the noise and the hypotheses."""
    ss = np.random.SeedSequence(seed)
    kids = ss.spawn(8 + len(cfg.levels))
    r_dsm, r_pose, r_ref, r_hyp, r_grav, r_rng = (np.random.default_rng(k) for k in kids[:6])
    r_lev = [np.random.default_rng(k) for k in kids[8:]]

    dsm, x0, y0, X, Y = _make_dsm(cfg, r_dsm)
    S, gsd = cfg.crop_side, cfg.gsd
    points = np.stack([X.ravel(), Y.ravel(), dsm.astype(np.float64).ravel()]).astype(np.float32)

    H0, W0 = cfg.levels[0]
    cx0, cy0 = W0 / 2.0, H0 / 2.0

    # ground-truth pose: optical axis through the crop centre's surface point
    alt = r_pose.uniform(*cfg.altitude)
    pitch = np.deg2rad(r_pose.uniform(*cfg.pitch_deg))
    yaw = r_pose.uniform(0.0, 2.0 * np.pi)
    target = np.array([0.0, 0.0, dsm_height(dsm, x0, y0, gsd, 0.0, 0.0)[0]])
    d = np.cos(pitch) * np.array([np.cos(yaw), np.sin(yaw), 0.0]) + np.sin(pitch) * np.array([0, 0, -1.0])
    dist = (alt - target[2]) / np.sin(pitch)
    C_gt = target - dist * d
    T_gt = look_pose(C_gt, yaw, pitch)

    qry, refs, seen = [], [], []
    valid = np.ones(points.shape[1], bool)
    for lvl, (H, W) in enumerate(cfg.levels):
        qry.append(_make_feature_map(H, W, cfg.channels, cfg, r_lev[lvl]))
    for lvl, (H, W) in enumerate(cfg.levels):
        s = 2.0 ** -lvl
        u, v, z = project_gt(points, T_gt, cfg.f0 * s, cx0 * s, cy0 * s)
        vis = (z > 0.1) & (u - 0.5 >= 0) & (u - 0.5 <= W - 1) & (v - 0.5 >= 0) & (v - 0.5 <= H - 1)
        valid &= vis
        seen.append(vis)
        f = read_map(qry[lvl], u, v)
        f += cfg.ref_noise * r_ref.standard_normal(f.shape)
        refs.append(f.astype(np.float32))
    if cfg.n_anchors > 0:
        # geo-anchors drawn from the whole crop, blind to the ground truth (Sec. V-A: the
        # refinement runs on a fixed number of anchors drawn from the crop's valid pixels --
        # every cell of a synthetic crop is one): an anchor the query does not see at a level
        # gets a random unit descriptor there, as a real network's reference descriptor of a
        # pixel outside the query view would match nothing
        r_anc = np.random.default_rng(kids[6])
        keep = np.sort(r_anc.choice(points.shape[1], cfg.n_anchors, replace=False))
        points = np.ascontiguousarray(points[:, keep])
        valid = np.ones(keep.size, bool)
        out = []
        for f, vis in zip(refs, seen):
            f = np.ascontiguousarray(f[keep])
            unseen = ~vis[keep]
            rnd = r_anc.standard_normal((int(unseen.sum()), f.shape[1]))
            f[unseen] = (rnd / np.linalg.norm(rnd, axis=1, keepdims=True)).astype(np.float32)
            out.append(f)
        refs = out
        n_seen_all = int(np.logical_and.reduce([vis[keep] for vis in seen]).sum())
    else:
        for f in refs:
            f[~valid] = 0.0
        n_seen_all = int(valid.sum())

    # hypotheses
    M = cfg.n_hyps
    if cfg.hyp_mode == "grid":
        r_prior = np.random.default_rng(kids[7])
        if cfg.prior_ring is None:
            pdx, pdy = r_prior.uniform(-cfg.prior_xy, cfg.prior_xy, 2)
            pyaw = r_prior.uniform(-cfg.prior_yaw_deg, cfg.prior_yaw_deg)
        else:
            lo, hi = cfg.prior_ring
            rad, ang = r_prior.uniform(lo, hi), r_prior.uniform(0.0, 2.0 * np.pi)
            pdx, pdy = rad * np.cos(ang), rad * np.sin(ang)
            pyaw = r_prior.choice([-1.0, 1.0]) * r_prior.uniform(lo, hi)
        prior = _perturb_xy_yaw(T_gt, pdx, pdy, np.deg2rad(pyaw))
        grid = [(gx, gy, gp) for gx in cfg.grid_xy for gy in cfg.grid_xy for gp in cfg.grid_yaw_deg]
        M = len(grid)
    hyps = np.empty((M, 12))
    for m in range(M):
        if cfg.hyp_mode == "grid":
            gx, gy, gp = grid[m]
            hyps[m] = _perturb_xy_yaw(prior, gx, gy, np.deg2rad(gp))
        elif cfg.hyp_mode == "xy_yaw":
            dx, dy = r_hyp.uniform(-cfg.hyp_xy, cfg.hyp_xy, 2)
            dpsi = np.deg2rad(r_hyp.uniform(-cfg.hyp_yaw_deg, cfg.hyp_yaw_deg))
            hyps[m] = _perturb_xy_yaw(T_gt, dx, dy, dpsi)
        elif cfg.hyp_mode == "rot_trans":
            hyps[m] = _perturb_rot_trans(T_gt, _unit(r_hyp), np.deg2rad(cfg.hyp_rot_deg),
                                         _unit(r_hyp), cfg.hyp_trans)
        else:
            raise ValueError(cfg.hyp_mode)

    # IMU gravity in the camera frame, tilted by a small angle about a perpendicular axis
    R_gt, _ = pose_parts(T_gt)
    g_cam = R_gt @ GRAVITY_WORLD
    a = np.cross(g_cam, _unit(r_grav))
    a /= np.linalg.norm(a)
    g_meas = Rotation.from_rotvec(a * np.deg2rad(cfg.gravity_noise_deg)).as_matrix() @ g_cam

    # laser range along the optical axis (the principal point is the image centre)
    rng_true = _ray_to_dsm(C_gt, d, dsm, x0, y0, gsd)
    rng_meas = rng_true + cfg.range_noise * r_rng.standard_normal()

    return Frame(points=np.ascontiguousarray(points), point_valid=valid.astype(np.uint8),
                 point_weight=np.ones(points.shape[1], np.float32), ref_feat=refs,
                 qry_feat=qry, fx=cfg.f0, fy=cfg.f0, cx=cx0, cy=cy0,
                 T_hyps=hyps, T_gt=T_gt, use_gravity=cfg.use_gravity,
                 gravity_cam=g_meas, gravity_world=GRAVITY_WORLD.copy(), w_grav=cfg.w_grav,
                 use_range=cfg.use_range, range_m=float(rng_meas), w_range=cfg.w_range,
                 dsm=dsm, dsm_x0=x0, dsm_y0=y0, dsm_gsd=gsd, seed=seed,
                 meta=dict(alt=alt, pitch_deg=float(np.rad2deg(pitch)), yaw_deg=float(np.rad2deg(yaw)),
                           range_true=float(rng_true), crop_side=S, n_seen_all_levels=n_seen_all,
                           T_prior=prior if cfg.hyp_mode == "grid" else None))


SEEDING_STRATEGIES = ("none", "yaw", "xy", "joint")


def seeding_hypotheses(T_prior: np.ndarray, strategy: str, cfg: SceneConfig | None = None) -> np.ndarray:
    """Initial hypotheses around a prior pose for the four seeding strategies of the
    multi-hypothesis ablation (Supp. "Effect of Multi-hypothesis Sampling"): "none" is the
    prior alone, "yaw" the yaw offsets of the grid at the prior's position, "xy" the (x, y)
    grid at the prior's yaw, "joint" the full (x, y, psi) grid (cfg's grid_xy x grid_xy x
    grid_yaw_deg; the paper's 11 x 11 x 10 by default).  Returns (M, 12) world->camera poses,
    x outermost and psi innermost as in the grid mode of make_frame."""
    cfg = cfg or SceneConfig()
    xy = cfg.grid_xy if strategy in ("xy", "joint") else (0.0,)
    yaw = cfg.grid_yaw_deg if strategy in ("yaw", "joint") else (0.0,)
    if strategy not in SEEDING_STRATEGIES:
        raise ValueError(strategy)
    return np.stack([_perturb_xy_yaw(T_prior, gx, gy, np.deg2rad(gp)).ravel()
                     for gx in xy for gy in xy for gp in yaw])


# ------------------------------------------------------------------ global TDOM/DSM map

@dataclass
class GlobalMap:
    """A georeferenced TDOM/DSM pair: cell (r, c) is centred at (x0 + (c + 1/2) gsd,
    y0 + (r + 1/2) gsd); the map's origin is its centre (x0 = y0 = -side gsd / 2)."""

    dsm: np.ndarray               # (side, side) float32 heights, metres
    tdom: np.ndarray              # (side, side, 3) uint8 RGB
    x0: float
    y0: float
    gsd: float


def make_global_map(side: int = 4096, gsd: float = 0.5, n_hills: int = 2048, n_boxes: int = 4096,
                    seed: int = 0) -> GlobalMap:
    """The crop-recipe terrain scaled to a whole map (Gaussian hills of sigma 10 m and
    amplitude U(0, 15) m, box buildings of U(5, 40) m on U(6, 16) m footprints), each added on
    its own window; the TDOM is a seeded colour texture (blurred noise at several scales,
    shaded by height) so that every map layer varies pixel to pixel."""
    rng = np.random.default_rng(seed)
    dsm = np.zeros((side, side), np.float32)
    half = side * gsd / 2.0
    x0 = y0 = -half
    sig = 10.0 / gsd                                   # hill sigma in cells
    rad = int(np.ceil(4 * sig))
    ax = np.arange(-rad, rad + 1, dtype=np.float32)
    for _ in range(n_hills):
        cr, cc = rng.uniform(0, side, 2)
        amp = rng.uniform(0.0, 15.0)
        r0, c0 = int(cr), int(cc)
        rs, cs = slice(max(r0 - rad, 0), min(r0 + rad + 1, side)), slice(max(c0 - rad, 0), min(c0 + rad + 1, side))
        gr = np.exp(-((np.arange(rs.start, rs.stop) + 0.5 - cr) ** 2) / (2 * sig * sig))
        gc = np.exp(-((np.arange(cs.start, cs.stop) + 0.5 - cc) ** 2) / (2 * sig * sig))
        dsm[rs, cs] += (amp * np.outer(gr, gc)).astype(np.float32)
    del ax
    for _ in range(n_boxes):
        cr, cc = rng.uniform(0, side, 2)
        sr, sc = rng.uniform(6.0, 16.0, 2) / gsd
        h = np.float32(rng.uniform(5.0, 40.0))
        rs = slice(max(int(cr - sr / 2), 0), min(int(cr + sr / 2) + 1, side))
        cs = slice(max(int(cc - sc / 2), 0), min(int(cc + sc / 2) + 1, side))
        np.maximum(dsm[rs, cs], h, out=dsm[rs, cs])
    tex = np.zeros((side, side, 3), np.float32)
    for k in range(3):
        for scale, w in ((2.0, 0.5), (8.0, 1.0), (32.0, 1.0)):
            small = max(side // int(scale), 8)
            noise = ndimage.gaussian_filter(rng.standard_normal((small, small)), 1.0, mode="wrap")
            tex[:, :, k] += w * ndimage.zoom(noise, side / small, order=1)[:side, :side]
    tex = (tex - tex.mean()) / (tex.std() + 1e-6)
    shade = (dsm - dsm.mean()) / (dsm.std() + 1e-6)
    rgb = 128.0 + 40.0 * tex + 20.0 * shade[:, :, None]
    return GlobalMap(dsm=dsm, tdom=np.clip(rgb, 0, 255).astype(np.uint8), x0=x0, y0=y0, gsd=gsd)


def crop_prior(gmap: GlobalMap, seed: int, img_w: int = 640, img_h: int = 480, f: float = 600.0,
               altitude=(120.0, 300.0), pitch_deg=(30.0, 70.0), margin: float = 400.0):
    """A seeded pose prior over the map (altitude, pitch and yaw as the frame recipe, optical
    axis through a surface point at least `margin` metres inside the map edge) and the
    intrinsics of its image (principal point at the image centre)."""
    rng = np.random.default_rng(seed)
    half = gmap.dsm.shape[0] * gmap.gsd / 2.0
    tx, ty = rng.uniform(-half + margin, half - margin, 2)
    c = int(np.clip((tx - gmap.x0) / gmap.gsd, 0, gmap.dsm.shape[1] - 1))
    r = int(np.clip((ty - gmap.y0) / gmap.gsd, 0, gmap.dsm.shape[0] - 1))
    target = np.array([tx, ty, float(gmap.dsm[r, c])])
    alt = rng.uniform(*altitude)
    pitch = np.deg2rad(rng.uniform(*pitch_deg))
    yaw = rng.uniform(0.0, 2.0 * np.pi)
    d = np.cos(pitch) * np.array([np.cos(yaw), np.sin(yaw), 0.0]) + np.sin(pitch) * np.array([0, 0, -1.0])
    C = target - (alt - target[2]) / np.sin(pitch) * d
    return dict(T_cw=look_pose(C, yaw, pitch), fx=f, fy=f, cx=img_w / 2.0, cy=img_h / 2.0,
                img_w=img_w, img_h=img_h, altitude=alt)


def with_query_confidence(frame: Frame, seed: int, low: float = 0.2) -> Frame:
    """The frame with seeded per-level query confidence maps in [low, 1] (a smooth random
    field: blurred noise through a logistic), standing in for the network's uncertainty
    output w^q_l."""
    rng = np.random.default_rng(seed)
    confs = []
    for q in frame.qry_feat:
        H, W = q.shape[:2]
        z = ndimage.gaussian_filter(rng.standard_normal((H, W)), max(H, W) / 40.0, mode="reflect")
        z /= z.std() + 1e-12
        confs.append((low + (1.0 - low) / (1.0 + np.exp(-2.0 * z))).astype(np.float32))
    return frame.replace(qry_conf=confs)


def frame_seed(workload: int, index: int) -> int:
    """Seed of frame `index` of workload number `workload` (1_000_000 * workload + index)."""
    return 1_000_000 * workload + index


# ------------------------------------------------------------------- error metrics

def rotation_error_deg(Ta, Tb) -> float:
    """Angle of R_a^T R_b in degrees (arccos of the clamped trace formula)."""
    Ra, _ = pose_parts(Ta)
    Rb, _ = pose_parts(Tb)
    c = (np.trace(Ra.T @ Rb) - 1.0) / 2.0
    return float(np.rad2deg(np.arccos(np.clip(c, -1.0, 1.0))))


def translation_error_m(Ta, Tb) -> float:
    """Distance between camera centres in metres."""
    return float(np.linalg.norm(camera_centre(Ta) - camera_centre(Tb)))


# ------------------------------------------------------------------ sequential tracking

@dataclass
class TrackConfig:
    """Recipe of a synthetic UAV sequence over a global TDOM/DSM map: a smooth flight
    (speed and heading rate varying as sums of sinusoids), the paper's 512-px pyramid and
    refinement schedule, and a reference crop per frame."""

    n_frames: int = 60
    rate_hz: float = 5.0
    speed: tuple = (10.0, 18.0)                      # m/s
    turn_rate_deg_s: float = 8.0                     # amplitude of the heading rate
    altitude: tuple = (110.0, 140.0)                 # camera height above the datum, m
    pitch_deg: tuple = (45.0, 60.0)                  # optical axis below the horizon
    levels: tuple = ((384, 512), (192, 256), (96, 128))
    f0: float = 480.0                                # level-0 focal length (600 px at 640 wide)
    channels: int = 32
    crop_side: int = 256
    ray_step: float = 0.25                           # footprint ray samples, metres
    ray_samples: int = 8000
    n_anchors: int = 500
    query_bank: int = 4                              # distinct query pyramids, used in turn
    ref_noise: float = 0.01
    degrade_prob: float = 0.05                       # frames whose reference descriptors are noise
    degraded_frames: tuple = ()                      # ... and frames that always are
    gravity_noise_deg: float = 0.2
    range_noise: float = 0.1
    w_grav: float = 1e2
    w_range: float = 1e1


def make_trajectory(gmap: GlobalMap, tc: TrackConfig, seed: int) -> np.ndarray:
    """(n_frames, 12) ground-truth world->camera poses of a seeded smooth flight that starts
    near the map centre; the camera looks forward along the heading."""
    rng = np.random.default_rng(seed)
    dt = 1.0 / tc.rate_hz
    n = tc.n_frames
    tt = np.arange(n) * dt
    ph = rng.uniform(0, 2 * np.pi, 6)
    w = rng.uniform(0.05, 0.2, 3)
    v = 0.5 * (tc.speed[0] + tc.speed[1]) + 0.5 * (tc.speed[1] - tc.speed[0]) * np.sin(w[0] * tt + ph[0])
    rate = np.deg2rad(tc.turn_rate_deg_s) * (0.6 * np.sin(w[1] * tt + ph[1]) + 0.4 * np.sin(3.1 * w[1] * tt + ph[2]))
    yaw = rng.uniform(0, 2 * np.pi) + np.concatenate([[0.0], np.cumsum(rate[:-1] * dt)])
    xy = np.zeros((n, 2))
    xy[0] = rng.uniform(-100.0, 100.0, 2)
    for k in range(1, n):
        xy[k] = xy[k - 1] + v[k - 1] * dt * np.array([np.cos(yaw[k - 1]), np.sin(yaw[k - 1])])
    alt = 0.5 * (tc.altitude[0] + tc.altitude[1]) + 0.5 * (tc.altitude[1] - tc.altitude[0]) * np.sin(w[2] * tt + ph[3])
    pitch = np.deg2rad(0.5 * (tc.pitch_deg[0] + tc.pitch_deg[1])
                       + 0.5 * (tc.pitch_deg[1] - tc.pitch_deg[0]) * np.sin(0.7 * w[2] * tt + ph[4]))
    return np.array([look_pose(np.array([xy[k, 0], xy[k, 1], alt[k]]), yaw[k], pitch[k]) for k in range(n)])


def query_bank(tc: TrackConfig, seed: int) -> list:
    """tc.query_bank query pyramids (lists of (H_l, W_l, C) maps), the stand-in for the
    feature network's query output; frame t uses pyramid t mod the bank size."""
    cfg = SceneConfig(levels=tc.levels, channels=tc.channels)
    ss = np.random.SeedSequence(seed).spawn(tc.query_bank * len(tc.levels))
    out = []
    for b in range(tc.query_bank):
        out.append([_make_feature_map(H, W, tc.channels, cfg, np.random.default_rng(ss[b * len(tc.levels) + l]))
                    for l, (H, W) in enumerate(tc.levels)])
    return out


def track_inputs(gmap: GlobalMap, tc: TrackConfig, bank: list, t: int, T_gt_world: np.ndarray,
                 crop_points: np.ndarray, crop_valid: np.ndarray, origin, seed: int, anchor_idx) -> Frame:
    """Frame t of a sequence from its reference crop (the stand-in for the feature network:
    reference descriptors are the query features at the anchors' ground-truth projections).

    crop_points (3, S^2) are the crop's anchors as offsets from `origin` (ox, oy);
    anchor_idx are the crop pixels drawn as geo-anchors (by the geo-anchor sampler, from the
    crop's valid mask, blind to the ground truth).  An anchor the query sees at a level under
    the ground truth (1-pixel margin) gets the query feature there plus noise; any other gets
    a random unit descriptor at that level (a real network's descriptor of a pixel outside
    the query view matches nothing).  With probability tc.degrade_prob the frame's reference
    descriptors are all random unit vectors (a visual failure).  Poses and the DSM are
    crop-local; T_hyps is a placeholder the tracker replaces by its seeds."""
    ss = np.random.SeedSequence([seed, t]).spawn(4)
    r_key, r_ref, r_sens, r_deg = (np.random.default_rng(k) for k in ss)
    ox, oy = float(origin[0]), float(origin[1])
    R, tw = pose_parts(T_gt_world)
    T_loc = np.hstack([R, (tw + R @ np.array([ox, oy, 0.0]))[:, None]]).ravel()
    qry = bank[t % len(bank)]
    keep = np.asarray(anchor_idx, np.int64)
    if keep.size == 0:
        raise ValueError(f"frame {t}: no geo-anchor drawn from the crop")
    pts = np.asarray(crop_points, np.float32)[:, keep]
    H0, W0 = tc.levels[0]
    cx0, cy0 = W0 / 2.0, H0 / 2.0
    refs = []
    degraded = bool(r_deg.random() < tc.degrade_prob) or t in tc.degraded_frames
    seen_all = np.ones(keep.size, bool)
    for lvl, (H, W) in enumerate(tc.levels):
        s = 2.0 ** -lvl
        u, v, z = project_gt(pts, T_loc, tc.f0 * s, cx0 * s, cy0 * s)
        seen = (z > 0.1) & (u - 0.5 >= 1.0) & (u - 0.5 <= W - 2.0) & (v - 0.5 >= 1.0) & (v - 0.5 <= H - 2.0)
        seen_all &= seen
        f = np.empty((keep.size, tc.channels))
        if seen.any():
            f[seen] = read_map(qry[lvl], u[seen], v[seen]) + tc.ref_noise * r_ref.standard_normal((int(seen.sum()), tc.channels))
        rnd_rows = ~seen if not degraded else np.ones(keep.size, bool)
        rnd = r_ref.standard_normal((int(rnd_rows.sum()), tc.channels))
        f[rnd_rows] = rnd / np.linalg.norm(rnd, axis=1, keepdims=True)
        refs.append(f.astype(np.float32))
    g_cam = R @ GRAVITY_WORLD
    a = np.cross(g_cam, _unit(r_sens))
    a /= np.linalg.norm(a)
    g_meas = Rotation.from_rotvec(a * np.deg2rad(tc.gravity_noise_deg)).as_matrix() @ g_cam
    C_loc = -R.T @ T_loc.reshape(3, 4)[:, 3]
    d = R[2]                                         # optical axis in the world
    rng_true = _ray_to_dsm(C_loc, d, gmap.dsm, gmap.x0 - ox, gmap.y0 - oy, gmap.gsd, step=tc.ray_step, pointwise=True)
    rng_meas = rng_true + tc.range_noise * r_sens.standard_normal()
    sub = np.ascontiguousarray(pts)
    return Frame(points=sub, point_valid=np.ones(keep.size, np.uint8),
                 point_weight=np.ones(keep.size, np.float32), ref_feat=refs, qry_feat=qry,
                 fx=tc.f0, fy=tc.f0, cx=cx0, cy=cy0, T_hyps=T_loc.reshape(1, 12).copy(), T_gt=T_loc,
                 use_gravity=True, gravity_cam=g_meas, gravity_world=GRAVITY_WORLD.copy(), w_grav=tc.w_grav,
                 use_range=True, range_m=float(rng_meas), w_range=tc.w_range,
                 dsm=gmap.dsm, dsm_x0=gmap.x0 - ox, dsm_y0=gmap.y0 - oy, dsm_gsd=gmap.gsd,
                 seed=seed, meta=dict(t=t, degraded=degraded, origin=(ox, oy), n_seen_all_levels=int(seen_all.sum())))


class SyntheticNetwork:
    """The feature extractor's place in a tracked sequence: frame t's crop -> (Frame, device
    arrays without T_cw).  Query pyramids of the bank are uploaded once and shared; the
    per-frame anchors and reference descriptors come from track_inputs."""

    def __init__(self, gmap: GlobalMap, tc: TrackConfig, bank: list, gt_poses: np.ndarray, seed: int,
                 device: str = "cuda"):
        self.gmap, self.tc, self.bank, self.gt, self.seed, self.device = gmap, tc, bank, gt_poses, seed, device
        self._qdev = {}
        self.frames = {}

    def frame(self, t: int, crop: dict) -> Frame:
        return track_inputs(self.gmap, self.tc, self.bank, t, self.gt[t], crop["points"], crop["valid"],
                            crop["origin"], self.seed, crop["anchor_idx"])

    def __call__(self, t: int, crop: dict):
        import torch
        f = self.frame(t, crop)
        self.frames[t] = f
        b = t % len(self.bank)
        if b not in self._qdev:
            self._qdev[b] = [torch.from_numpy(np.ascontiguousarray(q)).to(self.device) for q in self.bank[b]]
        to = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(self.device)
        arrays = dict(points=to(f.points), point_weight=to(f.point_weight), point_valid=to(f.point_valid),
                      ref_feat=[to(r) for r in f.ref_feat], qry_feat=self._qdev[b])
        return f, arrays


# ------------------------------------------------------------- serving workload (streams)

@dataclass
class StreamConfig:
    """Recipe of the serving workload: UAV streams over one global map, each a smooth
    trajectory at `rate_hz` (Poisson jitter on arrival, mean 1 / rate_hz), altitude and pitch
    drawn per stream, heading rate at most `yaw_rate_deg_s`, ground speed `speed`; per frame
    a reference crop of side U{crop_sides} around the previous estimate (every valid crop
    pixel a geo-anchor), hypotheses on a grid around it, BF16 features (the query pyramids of
    a bank, used in turn; reference descriptors the query features at the anchors'
    ground-truth projections plus noise, random unit vectors for anchors the query does not
    see), gravity and range priors as the frame recipe."""

    n_frames: int = 300
    rate_hz: float = 30.0
    speed: float = 10.0                              # m/s
    yaw_rate_deg_s: float = 10.0                     # largest heading rate
    altitude: tuple = (100.0, 300.0)
    pitch_deg: tuple = (30.0, 70.0)
    crop_sides: tuple = (128, 192, 256, 320, 384)
    grids: tuple = ((2, 4), (3, 4), (2, 9), (3, 7), (4, 5), (3, 9), (4, 7), (4, 9))   # (n_xy, n_yaw): M = 16 .. 144
    xy_span: float = 10.0                            # grid half-width, metres
    yaw_span_deg: float = 5.0                        # grid half-width, degrees
    levels: tuple = ((480, 640), (240, 320), (120, 160))
    f0: float = 600.0
    channels: int = 32
    query_bank: int = 4
    ref_noise: float = 0.01
    gravity_noise_deg: float = 0.2
    range_noise: float = 0.1
    w_grav: float = 1e2
    w_range: float = 1e1


def stream_trajectory(gmap: GlobalMap, sc: StreamConfig, seed: int) -> np.ndarray:
    """(n_frames, 12) ground-truth world->camera poses of one seeded stream: constant
    altitude U(altitude) and pitch U(pitch), heading rate a sinusoid of amplitude up to
    yaw_rate_deg_s, ground speed `speed`, starting well inside the map."""
    rng = np.random.default_rng(seed)
    n, dt = sc.n_frames, 1.0 / sc.rate_hz
    tt = np.arange(n) * dt
    alt = rng.uniform(*sc.altitude)
    pitch = np.deg2rad(rng.uniform(*sc.pitch_deg))
    amp = np.deg2rad(rng.uniform(0.3, 1.0) * sc.yaw_rate_deg_s)
    w, ph = rng.uniform(0.2, 1.0), rng.uniform(0, 2 * np.pi)
    yaw = rng.uniform(0, 2 * np.pi) + np.concatenate([[0.0], np.cumsum(amp * np.sin(w * tt[:-1] + ph) * dt)])
    half = gmap.dsm.shape[0] * gmap.gsd / 2.0
    xy = np.zeros((n, 2))
    margin = min(900.0, 0.5 * half)                  # the crops stay on the map
    xy[0] = rng.uniform(-half + margin, half - margin, 2)
    for k in range(1, n):
        xy[k] = xy[k - 1] + sc.speed * dt * np.array([np.cos(yaw[k - 1]), np.sin(yaw[k - 1])])
    return np.array([look_pose(np.array([xy[k, 0], xy[k, 1], alt]), yaw[k], pitch) for k in range(n)])


def stream_sensors(gmap: GlobalMap, sc: StreamConfig, gt: np.ndarray, seed: int) -> list:
    """Per frame of a stream: (measured gravity in the camera frame, measured laser range
    along the optical axis), from the ground truth with the recipe's noise."""
    rng = np.random.default_rng(seed)
    Cs = np.array([camera_centre(T) for T in gt])
    ds = np.array([pose_parts(T)[0][2] for T in gt])            # optical axes in the world
    rng_true = _rays_to_dsm(Cs, ds, gmap.dsm, gmap.x0, gmap.y0, gmap.gsd)
    out = []
    for T, r_t in zip(gt, rng_true):
        R, _ = pose_parts(T)
        g_cam = R @ GRAVITY_WORLD
        a = np.cross(g_cam, _unit(rng))
        a /= np.linalg.norm(a)
        g_meas = Rotation.from_rotvec(a * np.deg2rad(sc.gravity_noise_deg)).as_matrix() @ g_cam
        out.append((g_meas, float(r_t + sc.range_noise * rng.standard_normal())))
    return out


def stream_frame_shape(sc: StreamConfig, stream: int, t: int) -> tuple:
    """(crop side, n_xy, n_yaw) of frame t of a stream, seeded by (stream, t)."""
    rng = np.random.default_rng([9_000_000 + stream, t])
    side = int(sc.crop_sides[rng.integers(0, len(sc.crop_sides))])
    n_xy, n_yaw = sc.grids[rng.integers(0, len(sc.grids))]
    return side, int(n_xy), int(n_yaw)


class StreamNetwork:
    """The feature network's stand-in for the serving workload, on the device: a bank of
    query pyramids (FP32 for sampling, BF16 for the solver) and, for a crop, the reference
    descriptors of every anchor at every level -- the bank pyramid read bilinearly at the
    anchor's ground-truth projection (pixel i covers [i, i + 1), read at array coordinate
    pixel - 1/2) plus N(0, ref_noise) noise where the query sees it (1-pixel margin), a random
    unit vector elsewhere.  The noise and the unit vectors are rows of two fixed device banks
    read from an offset drawn per frame and level from the frame's seed, so a frame's
    descriptors are the same whether it is described alone or with others."""

    BANK_ROWS = 1 << 18              # at least the largest crop (384^2 anchors) + offsets

    def __init__(self, sc: StreamConfig, seed: int, device: str = "cuda"):
        import torch
        self.torch, self.sc, self.device = torch, sc, device
        cfg = SceneConfig(levels=sc.levels, channels=sc.channels)
        ss = np.random.SeedSequence(seed).spawn(sc.query_bank * len(sc.levels) + 1)
        self.bank32, self.bank_nchw = [], []
        for b in range(sc.query_bank):
            lv, lc = [], []
            for l, (H, W) in enumerate(sc.levels):
                m = _make_feature_map(H, W, sc.channels, cfg, np.random.default_rng(ss[b * len(sc.levels) + l]))
                t = torch.from_numpy(np.ascontiguousarray(m, np.float32)).to(device)
                lv.append(t)
                lc.append(t.permute(2, 0, 1).unsqueeze(0).contiguous())
            self.bank32.append(lv)
            self.bank_nchw.append(lc)
        g = torch.Generator(device=device)
        g.manual_seed(int(ss[-1].generate_state(1)[0]))
        self.noise = torch.randn((self.BANK_ROWS, sc.channels), generator=g, device=device)
        u = torch.randn((self.BANK_ROWS, sc.channels), generator=g, device=device)
        self.unit = u / u.norm(dim=1, keepdim=True)

    def _offsets(self, seed: int, n: int) -> np.ndarray:
        """Per level the (noise, unit) bank rows where a frame of n anchors starts."""
        r = np.random.default_rng(int(seed) & 0x7FFFFFFFFFFFFFFF)
        return r.integers(0, self.BANK_ROWS - n + 1, size=(len(self.sc.levels), 2))

    def descriptors(self, b: int, points, T_local: np.ndarray, seed: int) -> list:
        """Per level (N, C) FP32 device reference descriptors of the anchors `points` (3, N)
        (device, crop-local) under the crop-local ground truth T_local, with pyramid b."""
        return self.descriptors_batch([(b, points, T_local, seed)])[0]

    def descriptors_batch(self, items: list) -> list:
        """descriptors() for several (b, points, T_local, seed) at once: the frames of one
        pyramid are concatenated and described by one sequence of device operations per
        level; the results equal descriptors() frame by frame, bitwise (every operation is
        per anchor).  Returns, per item, its per-level (N, C) tensors (views of one tensor per
        pyramid and level)."""
        torch = self.torch
        sc = self.sc
        H0, W0 = sc.levels[0]
        out = [None] * len(items)
        for b in sorted({it[0] for it in items}):
            idx = [i for i, it in enumerate(items) if it[0] == b]
            counts = [int(items[i][1].shape[1]) for i in idx]
            n_all = sum(counts)
            P = torch.cat([items[i][1] for i in idx], dim=1).double()
            # per-frame pose rows and bank offsets in pinned host blocks, copied without waiting
            # for the stream (a pageable copy would wait for the server's running round)
            L = len(sc.levels)
            hT = torch.empty((len(idx), 12), dtype=torch.float64, pin_memory=True)
            hO = torch.empty((len(idx), 2 * L), dtype=torch.int64, pin_memory=True)
            hN = torch.empty(len(idx), dtype=torch.int64, pin_memory=True)
            start = 0
            for k, i in enumerate(idx):
                hT[k] = torch.from_numpy(np.asarray(items[i][2], np.float64).ravel())
                hO[k] = torch.from_numpy((self._offsets(items[i][3], counts[k]) - start).ravel())
                hN[k] = counts[k]
                start += counts[k]
            fi = torch.repeat_interleave(torch.arange(len(idx), device=self.device),
                                         hN.to(self.device, non_blocking=True), output_size=n_all)
            T = hT.to(self.device, non_blocking=True)[fi]          # (n_all, 12): the anchor's frame pose
            O = hO.to(self.device, non_blocking=True)[fi]          # (n_all, 2L): its bank row shifts
            x, y, z = (T[:, 4 * r] * P[0] + T[:, 4 * r + 1] * P[1] + T[:, 4 * r + 2] * P[2] + T[:, 4 * r + 3]
                       for r in range(3))
            pos = torch.arange(n_all, device=self.device)
            per_level = []
            for l, (H, W) in enumerate(sc.levels):
                s = 2.0 ** -l
                zz = torch.where(z > 0.1, z, torch.ones_like(z))
                u = sc.f0 * s * x / zz + W0 / 2.0 * s
                v = sc.f0 * s * y / zz + H0 / 2.0 * s
                seen = (z > 0.1) & (u - 0.5 >= 1.0) & (u - 0.5 <= W - 2.0) & (v - 0.5 >= 1.0) & (v - 0.5 <= H - 2.0)
                gx = (2.0 * (u - 0.5) / (W - 1) - 1.0).float()
                gy = (2.0 * (v - 0.5) / (H - 1) - 1.0).float()
                grid = torch.stack([gx, gy], dim=-1).view(1, 1, -1, 2)
                f = torch.nn.functional.grid_sample(self.bank_nchw[b][l], grid, mode="bilinear", align_corners=True)
                f = f.view(sc.channels, -1).t()
                rn = pos + O[:, 2 * l]
                ru = pos + O[:, 2 * l + 1]
                f = f + sc.ref_noise * self.noise[rn]
                per_level.append(torch.where(seen[:, None], f, self.unit[ru]).contiguous())
            parts = [torch.split(t, counts) for t in per_level]
            for k, i in enumerate(idx):
                out[i] = [parts[l][k] for l in range(L)]
        return out
