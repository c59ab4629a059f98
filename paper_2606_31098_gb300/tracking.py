"""Sequential localisation over the C-ABI (Supp. "Runtime Analysis"; Sec. V-A's Failure
Recovery Count).

Every numeric step runs in the library: the constant-velocity prior (pilot_pose_predict),
the reference crop around it (pilot_crop_reference, on the map-preparation stream), the
(x, y, psi) seeds written into device memory (pilot_seed_hypotheses), the solve
(pilot_align_solve) and the return to world coordinates (pilot_pose_reorigin).  This
module only orders the calls and keeps the history of estimates.

Frame t's prior is the initial pose for t = 0 and the given pose after a recovery, else
the prediction one frame on from the last two estimates.  In "serial" mode its crop is made
around that prior just before it is localised.  In "lookahead" mode a map-preparation
thread makes frame t+1's crop while frame t is localised, around the prediction two frames
on from the estimates known then (frames up to t-1); a recovery discards that crop and the
next frame is cropped around the pose it restarts from.  The caller's `network` turns a
crop into the frame to solve (the feature extractor's place in the online system).
"""
from __future__ import annotations

import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import binding as B


def frame_prior(t: int, history: list, given=None) -> np.ndarray:
    """Frame t's prior: `given` (the initial pose, or the pose a recovery restarts from) when
    set, else the prediction one frame on from the estimates of frames t-1 and t-2 (the last
    one held when it is the only one)."""
    if given is not None:
        return np.asarray(given, np.float64).ravel().copy()
    return B.pose_predict(history[t - 1], history[t - 2] if t >= 2 else None, 1)


def lookahead_crop_pose(t: int, history: list, initial) -> np.ndarray:
    """Crop pose of frame t made while frame t-1 is localised: predicted two frames on from
    the estimates of frames t-2 and t-3 (frames 0 and 1: the initial pose)."""
    if t <= 1:
        return np.asarray(initial, np.float64).ravel().copy()
    return B.pose_predict(history[t - 2], history[t - 3] if t >= 3 else None, 2)


class CropFailure(RuntimeError):
    """The reference crop around a prior failed (a corner ray never met the DSM)."""


@dataclass
class Camera:
    fx: float
    fy: float
    cx: float
    cy: float
    img_w: int
    img_h: int


@dataclass
class CropSettings:
    side: int = 256
    s_min: float = 0.0
    s_step: float = 0.25
    n_samples: int = 8000
    n_anchors: int = 500          # geo-anchors drawn from each crop's valid pixels
    anchor_seed: int = 0          # base seed of the draws (frame t: frame_anchor_seed(anchor_seed, t))


def frame_anchor_seed(base: int, t: int) -> int:
    """Seed of frame t's geo-anchor draw (a distinct SplitMix64 stream per frame)."""
    return (int(base) * 1000003 + int(t) + 1) & 0xFFFFFFFFFFFFFFFF


@dataclass
class FrameTiming:
    crop_ms: float            # device time of the crop (map-preparation stream)
    solve_ms: float           # device time of seeding + solve (localisation stream)
    wall_ms: float            # host time of localise(), network included
    prepared_ahead: bool      # the crop came from the map-preparation thread


@dataclass
class TrackerState:
    history: list = field(default_factory=list)      # world estimates (after recovery: given poses)
    priors: list = field(default_factory=list)
    crop_poses: list = field(default_factory=list)
    timings: list = field(default_factory=list)


class SequentialTracker:
    """Localises a sequence frame by frame on one GPU with two CUDA streams."""

    def __init__(self, dsm, tdom, x0: float, y0: float, gsd: float, camera: Camera, crop: CropSettings,
                 opts: B.Options, grid_xy, grid_yaw_deg, mode: str = "serial"):
        import torch
        if mode not in ("serial", "lookahead"):
            raise ValueError(mode)
        self.torch = torch
        self.mode = mode
        self.cam, self.crop_cfg = camera, crop
        self.grid_xy, self.grid_yaw = tuple(grid_xy), tuple(grid_yaw_deg)
        self.M = len(self.grid_xy) ** 2 * len(self.grid_yaw)
        dev = torch.device("cuda")
        self.dsm_dev = dsm if isinstance(dsm, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(dsm, np.float32)).to(dev)
        self.tdom_dev = None if tdom is None else (
            tdom if isinstance(tdom, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(tdom, np.uint8)).to(dev))
        self.map = B.MapArgs(self.dsm_dev, self.tdom_dev, x0, y0, gsd)
        self.solver = B.Solver(opts)
        self.loc_stream = torch.cuda.Stream()
        self.map_stream = torch.cuda.Stream()
        S = crop.side
        # two crop slots (the one being localised and the one being prepared), each with a
        # page-locked host copy for the network
        self.slots = []
        n = crop.n_anchors
        for _ in range(2):
            d = dict(points=torch.empty((3, S * S), dtype=torch.float32, device=dev),
                     valid=torch.empty(S * S, dtype=torch.uint8, device=dev), rgb=None,
                     geometry=torch.empty(28, dtype=torch.float64, device=dev),
                     idx=torch.empty(n, dtype=torch.int32, device=dev),
                     anchors=torch.empty((3, n), dtype=torch.float32, device=dev),
                     count=torch.empty(1, dtype=torch.int32, device=dev))
            h = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in d.items() if v is not None}
            self.slots.append((d, h))
        self.seeds = torch.empty((self.M, 12), dtype=torch.float64, device=dev)
        self.state = TrackerState()
        self._next_given = None
        self._pending = None          # (thread, result holder) of the crop being prepared
        self._slot = 0

    # ------------------------------------------------------------------ poses
    def _prior(self, t: int) -> np.ndarray:
        return frame_prior(t, self.state.history, self._next_given)

    def _lookahead_pose(self, t: int) -> np.ndarray:
        return lookahead_crop_pose(t, self.state.history, self._initial)

    # ------------------------------------------------------------------ crops
    def _crop(self, T, slot: int, t: int) -> dict:
        """Crop around T into `slot` on the map-preparation stream and draw frame t's
        geo-anchors from its valid pixels (pilot_sample_anchors); waits for it and returns
        the host copies with the device time."""
        torch = self.torch
        d, h = self.slots[slot]
        c = self.crop_cfg
        p = B.crop_params(T, self.cam.fx, self.cam.fy, self.cam.cx, self.cam.cy, self.cam.img_w, self.cam.img_h,
                          c.s_min, c.s_step, c.n_samples, c.side)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(self.map_stream):
            e0.record(self.map_stream)
            B.crop_reference(self.map, p, with_rgb=False, out=d, stream=self.map_stream)
            B.sample_anchors(d["valid"], d["points"], c.n_anchors, frame_anchor_seed(c.anchor_seed, t),
                             out=dict(idx=d["idx"], points=d["anchors"], count=d["count"]), stream=self.map_stream)
            for k in h:
                h[k].copy_(d[k], non_blocking=True)
            e1.record(self.map_stream)
        e1.synchronize()
        g = h["geometry"].numpy()
        if g[27] != 1.0:
            raise CropFailure("the reference crop failed (a corner ray never met the DSM)")
        n = int(h["count"].numpy()[0])
        return dict(points=h["points"].numpy(), valid=h["valid"].numpy(), origin=(float(g[9]), float(g[10])),
                    anchor_idx=h["idx"].numpy()[:n].astype(np.int64).copy(), geometry=g.copy(),
                    crop_ms=e0.elapsed_time(e1), slot=slot)

    def _start_prepare(self, t_next: int):
        T = self._lookahead_pose(t_next)
        slot = 1 - self._slot
        box = {}

        def work():
            try:
                box["crop"] = self._crop(T, slot, t_next)
            except Exception as ex:      # surfaced when the crop is taken
                box["error"] = ex
        th = threading.Thread(target=work, daemon=True)
        th.start()
        self._pending = (t_next, T, th, box)

    def _take_prepared(self, t: int):
        if self._pending is None:
            return None
        t_next, T, th, box = self._pending
        th.join()
        self._pending = None
        if t_next != t or self._next_given is not None:
            return None
        if "error" in box:
            raise box["error"]
        return T, box["crop"]

    # ------------------------------------------------------------------ API
    def reset(self, T0):
        """Start a sequence at pose T0 (world -> camera)."""
        if self._pending is not None:
            self._pending[2].join()
            self._pending = None
        self._initial = np.asarray(T0, np.float64).ravel().copy()
        self.state = TrackerState()
        self._next_given = self._initial.copy()

    def localise(self, t: int, network):
        """Localise frame t (frames are given in order).  `network(t, crop)` returns
        (frame, device_arrays): a scenes.Frame in the crop's local frame and its device
        arrays (no T_cw).  Returns (world estimate, Result); when the crop around the prior
        fails, the prior is the estimate and the Result is None."""
        torch = self.torch
        if t != len(self.state.history):
            raise ValueError(f"frame {t} out of order (expected {len(self.state.history)})")
        w0 = time.perf_counter()
        prior = self._prior(t)
        prepared = None
        try:
            prepared = self._take_prepared(t) if self.mode == "lookahead" else None
            if prepared is not None:
                crop_pose, crop = prepared
                self._slot = crop["slot"]
            else:
                crop_pose = prior.copy()
                crop = self._crop(crop_pose, self._slot, t)
        except CropFailure:
            # no reference for this frame: the prior stands as its estimate
            self._next_given = None
            st = self.state
            st.history.append(prior.copy())
            st.priors.append(prior)
            st.crop_poses.append(prior.copy())
            st.timings.append(FrameTiming(0.0, 0.0, 1e3 * (time.perf_counter() - w0), False))
            return prior.copy(), None
        self._next_given = None
        if self.mode == "lookahead":
            self._start_prepare(t + 1)     # map preparation of frame t+1 runs meanwhile
        frame, arrays = network(t, crop)
        ox, oy = crop["origin"]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        arrays = dict(arrays)
        arrays["T_cw"] = self.seeds
        arrays["dsm"] = self.dsm_dev
        fa = B.FrameArgs(frame, arrays, is_device=True)
        with torch.cuda.stream(self.loc_stream):
            e0.record(self.loc_stream)
            B.seed_hypotheses(B.seed_params(prior, self.grid_xy, self.grid_yaw, (ox, oy)), out=self.seeds,
                              stream=self.loc_stream)
            r = self.solver.solve(fa, self.loc_stream)
            e1.record(self.loc_stream)
        e1.synchronize()
        if r.best < 0:
            T_world = prior.copy()         # nothing usable: the prior stands
        else:
            T_world = B.pose_reorigin(r.T_cw[r.best], -ox, -oy)
        st = self.state
        st.history.append(T_world.copy())
        st.priors.append(prior)
        st.crop_poses.append(crop_pose)
        st.timings.append(FrameTiming(crop["crop_ms"], e0.elapsed_time(e1), 1e3 * (time.perf_counter() - w0),
                                      prepared is not None))
        return T_world, r

    def recover(self, T_frame, T_next):
        """After a failure: frame t's estimate is replaced by T_frame in the history and frame
        t+1 restarts from T_next (prior and crop)."""
        self.state.history[-1] = np.asarray(T_frame, np.float64).ravel().copy()
        self._next_given = np.asarray(T_next, np.float64).ravel().copy()

    def close(self):
        if self._pending is not None:
            self._pending[2].join()
            self._pending = None
        self.solver.close()


def pose_error(T_est, T_gt) -> tuple[float, float]:
    """(camera-centre distance in metres, rotation angle in degrees)."""
    A, G = np.asarray(T_est, np.float64).reshape(3, 4), np.asarray(T_gt, np.float64).reshape(3, 4)
    Ca, Cg = -A[:, :3].T @ A[:, 3], -G[:, :3].T @ G[:, 3]
    c = (np.trace(A[:, :3].T @ G[:, :3]) - 1.0) / 2.0
    return float(np.linalg.norm(Ca - Cg)), float(np.rad2deg(np.arccos(np.clip(c, -1.0, 1.0))))


def run_sequence(tracker: SequentialTracker, gt_poses, network, t_fail: float = 20.0, r_fail: float = 20.0) -> dict:
    """The evaluation protocol of Sec. V-A over ground truth `gt_poses` (n, 12): start at the
    first ground-truth pose; a frame more than t_fail metres or r_fail degrees off counts one
    recovery and the next frame restarts from its ground truth."""
    gt = np.asarray(gt_poses, np.float64).reshape(-1, 12)
    tracker.reset(gt[0])
    est, err, failed = [], [], []
    for t in range(gt.shape[0]):
        T, _ = tracker.localise(t, network)
        e = pose_error(T, gt[t])
        fail = e[0] > t_fail or e[1] > r_fail
        if fail and t + 1 < gt.shape[0]:
            tracker.recover(gt[t], gt[t + 1])
        est.append(T)
        err.append(e)
        failed.append(fail)
    st = tracker.state
    return dict(estimates=np.array(est), err=np.array(err), failed=np.array(failed), frc=int(sum(failed)),
                priors=np.array(st.priors), crop_poses=np.array(st.crop_poses), timings=list(st.timings))
