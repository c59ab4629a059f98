"""ctypes binding of include/pilot_align.h (argument marshalling only).

Every step of the solve runs in the CUDA library libpilot_align.so; this module only
fills the C structures.  PyTorch serves as the owner of device memory and streams.
There is no fallback: if the library is missing, loading raises.
"""
from __future__ import annotations

import ctypes as ct
import os
from dataclasses import dataclass

import numpy as np

MAX_LEVELS = 4
PILOT_OK, PILOT_EINVAL, PILOT_ENOMEM, PILOT_ECUDA, PILOT_ETIMEOUT, PILOT_EBUSY = 0, -1, -2, -3, -4, -5
F32, BF16, F16, FP8E4M3 = 0, 1, 2, 3
HYP_OK, HYP_FEW_VALID, HYP_NOT_PD, HYP_NONFINITE, HYP_PRUNED = range(5)
DTYPE_NAMES = {F32: "f32", BF16: "bf16", F16: "f16", FP8E4M3: "fp8e4m3"}

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libpilot_align.so")

_vp = ct.c_void_p


class pilot_align_config(ct.Structure):
    _fields_ = [
        ("iters_per_level", ct.c_int * MAX_LEVELS), ("lambda0", ct.c_double),
        ("damping_mode", ct.c_int), ("huber_photo", ct.c_double), ("huber_grav", ct.c_double),
        ("huber_range", ct.c_double), ("keep_top_k", ct.c_int * MAX_LEVELS),
        ("min_valid_frac", ct.c_double), ("max_points", ct.c_int), ("max_hyps", ct.c_int),
        ("max_channels", ct.c_int), ("profile", ct.c_int), ("max_frames", ct.c_int),
        ("gate_grav", ct.c_double), ("gate_range", ct.c_double),
    ]


class pilot_frame(ct.Structure):
    _fields_ = [
        ("is_device", ct.c_int), ("N", ct.c_int), ("points", _vp), ("point_weight", _vp),
        ("point_valid", _vp), ("C", ct.c_int), ("L", ct.c_int), ("feat_dtype", ct.c_int),
        ("ref_feat", _vp * MAX_LEVELS), ("ref_scale", _vp * MAX_LEVELS),
        ("qry_feat", _vp * MAX_LEVELS), ("qry_scale", _vp * MAX_LEVELS), ("qry_conf", _vp * MAX_LEVELS),
        ("H", ct.c_int * MAX_LEVELS), ("W", ct.c_int * MAX_LEVELS),
        ("fx", ct.c_double), ("fy", ct.c_double), ("cx", ct.c_double), ("cy", ct.c_double),
        ("M", ct.c_int), ("T_cw", _vp),
        ("use_gravity", ct.c_int), ("gravity_cam", ct.c_double * 3), ("gravity_world", ct.c_double * 3),
        ("w_grav", ct.c_double), ("use_range", ct.c_int), ("range_m", ct.c_double),
        ("w_range", ct.c_double), ("dsm", _vp), ("dsm_H", ct.c_int), ("dsm_W", ct.c_int),
        ("dsm_x0", ct.c_double), ("dsm_y0", ct.c_double), ("dsm_gsd", ct.c_double),
    ]


class pilot_result(ct.Structure):
    _fields_ = [("T_cw", _vp), ("cost", _vp), ("n_valid", _vp), ("hyp_status", _vp),
                ("best", _vp), ("hyp_iters", _vp)]


_lib = None

# name -> (restype, argtypes), in the order include/pilot_align.h declares them
SIGNATURES = {
    "pilot_align_create": (ct.c_int, [ct.POINTER(pilot_align_config), ct.POINTER(_vp)]),
    "pilot_align_validate": (ct.c_int, [ct.POINTER(pilot_align_config), ct.POINTER(pilot_frame)]),
    "pilot_align_solve": (ct.c_int, [_vp, ct.POINTER(pilot_frame), ct.POINTER(pilot_result), _vp]),
    "pilot_align_solve_batch": (ct.c_int, [_vp, _vp, ct.c_int, _vp, _vp]),
    "pilot_align_autotune": (ct.c_int, [_vp, _vp, ct.c_int, ct.c_int, ct.c_int, _vp, ct.POINTER(ct.c_double), _vp]),
    "pilot_align_get_schedule": (ct.c_int, [_vp, _vp, ct.c_int, ct.c_int, _vp]),
    "pilot_align_set_schedule": (ct.c_int, [_vp, _vp, ct.c_int, ct.c_int, _vp]),
    "pilot_align_selftest_barrier_timeout": (ct.c_int, [_vp, ct.c_double, ct.POINTER(ct.c_double), _vp]),
    "pilot_align_selftest_flag_timeout": (ct.c_int, [_vp, _vp, ct.c_int, ct.c_double, ct.POINTER(ct.c_double), _vp]),
    "pilot_crop_reference": (ct.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "pilot_sample_anchors": (ct.c_int, [_vp, _vp, ct.c_int, ct.c_int, ct.c_ulonglong, _vp, _vp, _vp, _vp]),
    "pilot_pose_predict": (ct.c_int, [_vp, _vp, ct.c_int, _vp]),
    "pilot_pose_reorigin": (ct.c_int, [_vp, ct.c_double, ct.c_double, _vp]),
    "pilot_seed_hypotheses": (ct.c_int, [_vp, _vp, _vp]),
    "pilot_probe_fma": (ct.c_int, [ct.POINTER(ct.c_double), _vp]),
    "pilot_probe_gather": (ct.c_int, [_vp, ct.c_int, ct.c_int, ct.c_int, ct.c_int, ct.c_longlong,
                                      ct.POINTER(ct.c_double), _vp]),
    "pilot_probe_gather_frame": (ct.c_int, [_vp, ct.c_int, _vp, _vp, ct.c_int, ct.c_int, ct.c_int, ct.c_int,
                                            ct.c_double, ct.c_double, ct.c_double, ct.c_double, _vp, ct.c_int,
                                            ct.c_int, ct.POINTER(ct.c_double), _vp]),
    "pilot_align_debug_normal_eq": (ct.c_int, [_vp, ct.POINTER(pilot_frame), ct.c_int, _vp, _vp, _vp]),
    "pilot_align_profile": (ct.c_int, [_vp, ct.POINTER(ct.c_double), ct.POINTER(ct.c_int), ct.POINTER(ct.c_int)]),
    "pilot_align_normal_eq_noalloc": (ct.c_int, [ct.POINTER(pilot_align_config), ct.POINTER(pilot_frame), ct.c_int,
                                                  _vp, _vp, _vp]),
    "pilot_quantize_features": (ct.c_int, [_vp, ct.c_longlong, ct.c_int, ct.c_int, ct.c_int, _vp, _vp, _vp]),
    "pilot_align_destroy": (None, [_vp]),
    "pilot_align_last_error": (ct.c_char_p, []),
    "pilot_serve_create": (ct.c_int, [ct.POINTER(pilot_align_config), ct.c_size_t, ct.c_int, ct.POINTER(_vp)]),
    "pilot_serve_submit": (ct.c_int, [_vp, ct.POINTER(pilot_frame), ct.POINTER(ct.c_uint64)]),
    "pilot_serve_poll": (ct.c_int, [_vp, ct.c_uint64, ct.POINTER(pilot_result), ct.POINTER(ct.c_int),
                                    ct.POINTER(ct.c_double)]),
    "pilot_serve_wait": (ct.c_int, [_vp, ct.c_uint64, ct.POINTER(pilot_result), ct.POINTER(ct.c_double), ct.c_int]),
    "pilot_serve_set_levels_per_round": (ct.c_int, [_vp, ct.c_int]),
    "pilot_serve_set_reserved_sms": (ct.c_int, [_vp, ct.c_int]),
    "pilot_serve_get_stats": (ct.c_int, [_vp, _vp]),
    "pilot_serve_destroy": (None, [_vp]),
}


class pilot_map(ct.Structure):
    _fields_ = [("dsm", _vp), ("tdom", _vp), ("H", ct.c_int), ("W", ct.c_int),
                ("x0", ct.c_double), ("y0", ct.c_double), ("gsd", ct.c_double)]


class pilot_crop_params(ct.Structure):
    _fields_ = [("T_cw", ct.c_double * 12), ("fx", ct.c_double), ("fy", ct.c_double), ("cx", ct.c_double),
                ("cy", ct.c_double), ("img_w", ct.c_int), ("img_h", ct.c_int), ("s_min", ct.c_double),
                ("s_step", ct.c_double), ("n_samples", ct.c_int), ("S", ct.c_int)]


class pilot_schedule(ct.Structure):
    _fields_ = [("tile", ct.c_int), ("ctas_per_sm", ct.c_int), ("job_order", ct.c_int), ("streams", ct.c_int)]


def _schedule_dict(sc: pilot_schedule) -> dict:
    return {"tile": sc.tile, "ctas_per_sm": sc.ctas_per_sm, "job_order": sc.job_order, "streams": sc.streams}


class pilot_serve_stats(ct.Structure):
    _fields_ = [(n, ct.c_longlong) for n in ("rounds", "admitted", "completed", "pending", "active",
                                             "peak_active", "arena_bytes_in_use", "arena_bytes_peak")] + \
               [(n, ct.c_double) for n in ("round_device_ms", "round_wall_ms")]


def load(path: str = LIB_PATH):
    """Load the CUDA library (build it first with build_ext.build()).  Raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} is missing (run build_ext.build())")
        L = ct.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class PilotError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"status {status}: {msg}")
        self.status = status


def check(status: int):
    if status != PILOT_OK:
        raise PilotError(status, load().pilot_align_last_error().decode())
    return status


def pilot_align_last_error() -> str:
    return load().pilot_align_last_error().decode()


@dataclass
class Options:
    iters: tuple = (10, 10, 10, 0)
    lambda0: float = 1e-3
    damping_mode: int = 0
    huber_photo: float = 0.1
    huber_grav: float = 0.1
    huber_range: float = 1.0
    keep_top_k: tuple = (0, 0, 0, 0)
    min_valid_frac: float = 0.05
    max_points: int = 1 << 18
    max_hyps: int = 256
    max_channels: int = 32
    profile: int = 0
    max_frames: int = 64
    gate_grav: float = 0.0         # sensor-prior residual gates; 0 = off
    gate_range: float = 0.0

    def to_c(self) -> pilot_align_config:
        c = pilot_align_config()
        c.iters_per_level[:] = list(self.iters) + [0] * (MAX_LEVELS - len(self.iters))
        c.lambda0 = self.lambda0
        c.damping_mode = self.damping_mode
        c.huber_photo, c.huber_grav, c.huber_range = self.huber_photo, self.huber_grav, self.huber_range
        c.keep_top_k[:] = list(self.keep_top_k) + [0] * (MAX_LEVELS - len(self.keep_top_k))
        c.min_valid_frac = self.min_valid_frac
        c.max_points, c.max_hyps, c.max_channels = self.max_points, self.max_hyps, self.max_channels
        c.profile = self.profile
        c.max_frames = self.max_frames
        c.gate_grav, c.gate_range = self.gate_grav, self.gate_range
        return c


def _ptr(x) -> int | None:
    """Address of a torch tensor or numpy array (None for None)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


class FrameArgs:
    """A pilot_frame over arrays that stay alive as long as this object.

    `arrays` maps field names to numpy arrays (host frame, is_device = 0) or torch CUDA
    tensors (device frame, is_device = 1): points (3, N) f32, point_weight (N,) f32,
    point_valid (N,) u8, ref_feat / qry_feat lists, optional ref_scale / qry_scale / qry_conf lists,
    T_cw (M, 12) f64, dsm (H_D, W_D) f32.  Scalars come from `frame` (a scenes.Frame).
    """

    def __init__(self, frame, arrays: dict, is_device: bool, dtype: int = F32):
        self.arrays = arrays
        f = pilot_frame()
        f.is_device = int(is_device)
        pts = arrays["points"]
        f.N = int(pts.shape[1])
        f.points = _ptr(pts)
        f.point_weight = _ptr(arrays.get("point_weight"))
        f.point_valid = _ptr(arrays.get("point_valid"))
        qry = arrays["qry_feat"]
        ref = arrays["ref_feat"]
        f.L = len(qry)
        f.C = int(qry[0].shape[2])
        f.feat_dtype = dtype
        qs = arrays.get("qry_scale") or [None] * f.L
        rs = arrays.get("ref_scale") or [None] * f.L
        qc = arrays.get("qry_conf") or [None] * f.L
        for l in range(f.L):
            f.qry_feat[l] = _ptr(qry[l])
            f.ref_feat[l] = _ptr(ref[l])
            f.qry_scale[l] = _ptr(qs[l])
            f.ref_scale[l] = _ptr(rs[l])
            f.qry_conf[l] = _ptr(qc[l])
            f.H[l], f.W[l] = int(qry[l].shape[0]), int(qry[l].shape[1])
        f.fx, f.fy, f.cx, f.cy = frame.fx, frame.fy, frame.cx, frame.cy
        T = arrays["T_cw"]
        f.M = int(T.shape[0])
        f.T_cw = _ptr(T)
        f.use_gravity = int(frame.use_gravity)
        f.gravity_cam[:] = [float(v) for v in frame.gravity_cam]
        f.gravity_world[:] = [float(v) for v in frame.gravity_world]
        f.w_grav = frame.w_grav
        f.use_range = int(frame.use_range)
        f.range_m = frame.range_m
        f.w_range = frame.w_range
        dsm = arrays["dsm"]
        f.dsm = _ptr(dsm)
        f.dsm_H, f.dsm_W = int(dsm.shape[0]), int(dsm.shape[1])
        f.dsm_x0, f.dsm_y0, f.dsm_gsd = frame.dsm_x0, frame.dsm_y0, frame.dsm_gsd
        self.c = f

    @property
    def M(self) -> int:
        return self.c.M


def host_arrays(frame, T_hyps=None, pinned: bool = False) -> dict:
    """Host (numpy, optionally page-locked torch CPU) arrays of an FP32 frame."""
    T = np.ascontiguousarray(frame.T_hyps if T_hyps is None else T_hyps, np.float64).reshape(-1, 12)
    arrs = dict(points=np.ascontiguousarray(frame.points, np.float32),
                point_weight=np.ascontiguousarray(frame.point_weight, np.float32),
                point_valid=np.ascontiguousarray(frame.point_valid, np.uint8),
                ref_feat=[np.ascontiguousarray(r, np.float32) for r in frame.ref_feat],
                qry_feat=[np.ascontiguousarray(q, np.float32) for q in frame.qry_feat],
                T_cw=T, dsm=np.ascontiguousarray(frame.dsm, np.float32))
    if getattr(frame, "qry_conf", None) is not None:
        arrs["qry_conf"] = [None if c is None else np.ascontiguousarray(c, np.float32) for c in frame.qry_conf]
    if pinned:
        import torch
        pin = lambda a: None if a is None else torch.from_numpy(a).pin_memory()
        arrs = {k: ([pin(x) for x in v] if isinstance(v, list) else pin(v)) for k, v in arrs.items()}
    return arrs


def device_arrays(frame, T_hyps=None, device="cuda") -> dict:
    """Device (torch CUDA) copies of an FP32 frame's arrays."""
    import torch
    h = host_arrays(frame, T_hyps)
    to = lambda a: None if a is None else torch.from_numpy(a).to(device)
    return {k: ([to(x) for x in v] if isinstance(v, list) else to(v)) for k, v in h.items()}


@dataclass
class Result:
    T_cw: np.ndarray
    cost: np.ndarray
    n_valid: np.ndarray
    status: np.ndarray
    best: int
    hyp_iters: int


class Solver:
    """Owns one pilot_align_handle."""

    def __init__(self, opts: Options | None = None):
        self.opts = opts or Options()
        lib = load()
        self._cfg = self.opts.to_c()
        h = _vp()
        check(lib.pilot_align_create(ct.byref(self._cfg), ct.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            load().pilot_align_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _stream(stream) -> int | None:
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    return torch.cuda.current_stream().cuda_stream
            except Exception:
                pass
            return None
        return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)

    def solve(self, fa: FrameArgs, stream=None) -> Result:
        M = fa.M
        T = np.zeros((M, 12))
        cost = np.zeros(M)
        nv = np.zeros(M, np.int32)
        st = np.zeros(M, np.int32)
        best = np.zeros(1, np.int32)
        hi = np.zeros(1, np.int64)
        r = pilot_result(T.ctypes.data, cost.ctypes.data, nv.ctypes.data, st.ctypes.data,
                         best.ctypes.data, hi.ctypes.data)
        check(load().pilot_align_solve(self.h, ct.byref(fa.c), ct.byref(r), self._stream(stream)))
        return Result(T, cost, nv, st, int(best[0]), int(hi[0]))

    def solve_batch(self, fas: list, stream=None) -> list:
        """pilot_align_solve_batch over a list of device FrameArgs."""
        n = len(fas)
        frames = (pilot_frame * max(n, 1))()
        for i, fa in enumerate(fas):
            frames[i] = fa.c
        outs, res = [], (pilot_result * max(n, 1))()
        for i, fa in enumerate(fas):
            M = fa.M
            o = dict(T=np.zeros((M, 12)), cost=np.zeros(M), nv=np.zeros(M, np.int32), st=np.zeros(M, np.int32),
                     best=np.zeros(1, np.int32), hi=np.zeros(1, np.int64))
            res[i] = pilot_result(o["T"].ctypes.data, o["cost"].ctypes.data, o["nv"].ctypes.data,
                                  o["st"].ctypes.data, o["best"].ctypes.data, o["hi"].ctypes.data)
            outs.append(o)
        check(load().pilot_align_solve_batch(self.h, ct.cast(frames, _vp), n, ct.cast(res, _vp),
                                             self._stream(stream)))
        return [Result(o["T"], o["cost"], o["nv"], o["st"], int(o["best"][0]), int(o["hi"][0])) for o in outs]

    @staticmethod
    def _frame_array(fas):
        frames = (pilot_frame * len(fas))()
        for i, fa in enumerate(fas):
            frames[i] = fa.c
        return frames

    def autotune(self, fas: list, batched: bool, reps: int = 2, stream=None) -> tuple[dict, float]:
        """pilot_align_autotune: returns the chosen schedule and its mean time (ms)."""
        frames = self._frame_array(fas)
        sc = pilot_schedule()
        ms = ct.c_double()
        check(load().pilot_align_autotune(self.h, ct.cast(frames, _vp), len(fas), int(batched), int(reps),
                                          ct.cast(ct.byref(sc), _vp), ct.byref(ms), self._stream(stream)))
        return _schedule_dict(sc), ms.value

    def schedule(self, fas: list, batched: bool) -> dict:
        frames = self._frame_array(fas)
        sc = pilot_schedule()
        check(load().pilot_align_get_schedule(self.h, ct.cast(frames, _vp), len(fas), int(batched),
                                              ct.cast(ct.byref(sc), _vp)))
        return _schedule_dict(sc)

    def selftest_barrier_timeout(self, timeout_ms: float, stream=None) -> float:
        """pilot_align_selftest_barrier_timeout: returns the launch's device time (ms)."""
        ms = ct.c_double()
        check(load().pilot_align_selftest_barrier_timeout(self.h, float(timeout_ms), ct.byref(ms),
                                                          self._stream(stream)))
        return ms.value

    def selftest_flag_timeout(self, fas: list, timeout_ms: float, stream=None) -> float:
        """pilot_align_selftest_flag_timeout on device frames: returns the solve's wall time (ms)."""
        frames = self._frame_array(fas)
        ms = ct.c_double()
        check(load().pilot_align_selftest_flag_timeout(self.h, ct.cast(frames, _vp), len(fas), float(timeout_ms),
                                                       ct.byref(ms), self._stream(stream)))
        return ms.value

    def set_schedule(self, fas: list, batched: bool, tile: int = 1024, ctas_per_sm: int = 0,
                     job_order: int = 0, streams: int = 0) -> None:
        """pilot_align_set_schedule: pin the schedule for frames of this shape."""
        frames = self._frame_array(fas)
        sc = pilot_schedule(tile, ctas_per_sm, job_order, streams)
        check(load().pilot_align_set_schedule(self.h, ct.cast(frames, _vp), len(fas), int(batched),
                                              ct.cast(ct.byref(sc), _vp)))

    def normal_eq(self, fa: FrameArgs, level: int, T_cw, stream=None) -> np.ndarray:
        T = np.ascontiguousarray(T_cw, np.float64).reshape(-1, 12)
        assert T.shape[0] == fa.M
        out = np.zeros((fa.M, 29))
        check(load().pilot_align_debug_normal_eq(self.h, ct.byref(fa.c), int(level), T.ctypes.data,
                                                 out.ctypes.data, self._stream(stream)))
        return out

    def profile(self):
        ms = ct.c_double()
        nb = ct.c_int()
        nt = ct.c_int()
        check(load().pilot_align_profile(self.h, ct.byref(ms), ct.byref(nb), ct.byref(nt)))
        return ms.value, nb.value, nt.value


def normal_eq_noalloc(opts: Options, fa: FrameArgs, level: int, T_cw_dev, out29_dev, stream=None) -> int:
    """pilot_align_normal_eq_noalloc: device poses in, device M x 29 out, no allocation.
    Returns the status (the work is only enqueued on `stream`)."""
    cfg = opts.to_c()
    return load().pilot_align_normal_eq_noalloc(ct.byref(cfg), ct.byref(fa.c), int(level), _ptr(T_cw_dev),
                                                 _ptr(out29_dev), Solver._stream(stream))


class MapArgs:
    """A pilot_map over device tensors (dsm (H, W) float32, tdom (H, W, 3) uint8 or None)."""

    def __init__(self, dsm, tdom, x0: float, y0: float, gsd: float):
        self.dsm, self.tdom = dsm, tdom
        self.c = pilot_map(_ptr(dsm), _ptr(tdom), int(dsm.shape[0]), int(dsm.shape[1]), float(x0), float(y0),
                           float(gsd))


def crop_params(T_cw, fx, fy, cx, cy, img_w, img_h, s_min, s_step, n_samples, S) -> pilot_crop_params:
    p = pilot_crop_params()
    p.T_cw[:] = [float(v) for v in np.asarray(T_cw, np.float64).ravel()]
    p.fx, p.fy, p.cx, p.cy = float(fx), float(fy), float(cx), float(cy)
    p.img_w, p.img_h = int(img_w), int(img_h)
    p.s_min, p.s_step, p.n_samples, p.S = float(s_min), float(s_step), int(n_samples), int(S)
    return p


def crop_reference(m: MapArgs, p: pilot_crop_params, with_rgb: bool = True, out: dict | None = None,
                   stream=None) -> dict:
    """pilot_crop_reference into device tensors (allocated here unless `out` is given):
    points (3, S*S) f32, valid (S*S,) u8, rgb (S*S, 3) f32 or None, geometry (28,) f64.
    Asynchronous on `stream`."""
    import torch
    S = p.S
    if out is None:
        dev = m.dsm.device
        out = dict(points=torch.empty((3, S * S), dtype=torch.float32, device=dev),
                   valid=torch.empty(S * S, dtype=torch.uint8, device=dev),
                   rgb=torch.empty((S * S, 3), dtype=torch.float32, device=dev) if with_rgb else None,
                   geometry=torch.empty(28, dtype=torch.float64, device=dev))
    check(load().pilot_crop_reference(ct.byref(m.c), ct.byref(p), _ptr(out["points"]), _ptr(out["valid"]),
                                      _ptr(out["rgb"]), _ptr(out["geometry"]), Solver._stream(stream)))
    return out


def sample_anchors(valid_dev, points_dev, n_select: int, seed: int, out: dict | None = None, stream=None) -> dict:
    """pilot_sample_anchors on a crop's device valid mask (n,) u8 and geo-anchors (3, n) f32:
    returns device tensors idx (n_select,) i32, points (3, n_select) f32 and count (1,) i32
    (allocated here unless `out` is given).  Asynchronous on `stream`."""
    import torch
    n = int(valid_dev.numel())
    if out is None:
        dev = valid_dev.device
        out = dict(idx=torch.full((n_select,), -1, dtype=torch.int32, device=dev),
                   points=torch.zeros((3, n_select), dtype=torch.float32, device=dev),
                   count=torch.zeros(1, dtype=torch.int32, device=dev))
    check(load().pilot_sample_anchors(_ptr(valid_dev), _ptr(points_dev), n, int(n_select),
                                      ct.c_ulonglong(int(seed) & 0xFFFFFFFFFFFFFFFF), _ptr(out["idx"]),
                                      _ptr(out["points"]) if points_dev is not None else None, _ptr(out["count"]),
                                      Solver._stream(stream)))
    return out


MAX_SEED_XY, MAX_SEED_YAW = 32, 64


class pilot_seed_params(ct.Structure):
    _fields_ = [("T_prior", ct.c_double * 12), ("origin_x", ct.c_double), ("origin_y", ct.c_double),
                ("n_xy", ct.c_int), ("n_yaw", ct.c_int), ("grid_xy", ct.c_double * MAX_SEED_XY),
                ("grid_yaw_deg", ct.c_double * MAX_SEED_YAW)]


def _pose12(T) -> np.ndarray:
    a = np.ascontiguousarray(T, np.float64).ravel()
    if a.size != 12:
        raise ValueError("a pose is 12 values [R | t]")
    return a


def pose_predict(T_prev, T_prev2=None, steps: int = 1) -> np.ndarray:
    """pilot_pose_predict: constant-velocity prior `steps` frames after T_prev."""
    a = _pose12(T_prev)
    b = None if T_prev2 is None else _pose12(T_prev2)
    out = np.empty(12)
    check(load().pilot_pose_predict(a.ctypes.data, None if b is None else b.ctypes.data, int(steps),
                                    out.ctypes.data))
    return out


def pose_reorigin(T, dx: float, dy: float) -> np.ndarray:
    """pilot_pose_reorigin: the pose for points given relative to (dx, dy, 0)."""
    a = _pose12(T)
    out = np.empty(12)
    check(load().pilot_pose_reorigin(a.ctypes.data, float(dx), float(dy), out.ctypes.data))
    return out


def seed_params(T_prior, grid_xy, grid_yaw_deg, origin=(0.0, 0.0)) -> pilot_seed_params:
    p = pilot_seed_params()
    p.T_prior[:] = [float(v) for v in _pose12(T_prior)]
    p.origin_x, p.origin_y = float(origin[0]), float(origin[1])
    p.n_xy, p.n_yaw = len(grid_xy), len(grid_yaw_deg)
    if not (1 <= p.n_xy <= MAX_SEED_XY and 1 <= p.n_yaw <= MAX_SEED_YAW):
        raise ValueError("grid sizes outside [1, 32] x [1, 64]")
    p.grid_xy[:p.n_xy] = [float(v) for v in grid_xy]
    p.grid_yaw_deg[:p.n_yaw] = [float(v) for v in grid_yaw_deg]
    return p


def seed_hypotheses(p: pilot_seed_params, out=None, stream=None):
    """pilot_seed_hypotheses into a device tensor (M, 12) f64 (allocated here unless given)."""
    import torch
    M = p.n_xy * p.n_xy * p.n_yaw
    if out is None:
        out = torch.empty((M, 12), dtype=torch.float64, device="cuda")
    check(load().pilot_seed_hypotheses(ct.byref(p), _ptr(out), Solver._stream(stream)))
    return out


def probe_fma(stream=None) -> float:
    """pilot_probe_fma: measured FP32 FMA throughput (TFLOP/s)."""
    v = ct.c_double()
    check(load().pilot_probe_fma(ct.byref(v), Solver._stream(stream)))
    return v.value


def probe_gather(map_dev, dtype: int, samples: int = 1 << 24, stream=None) -> float:
    """pilot_probe_gather on a device H x W x C map: 4-tap gathers at random pixels (GB/s)."""
    H, W, C = map_dev.shape
    v = ct.c_double()
    check(load().pilot_probe_gather(ct.c_void_p(map_dev.data_ptr()), int(H), int(W), int(C), int(dtype),
                                    int(samples), ct.byref(v), Solver._stream(stream)))
    return v.value


def probe_gather_frame(points_dev, map_dev, ref_dev, dtype: int, fx: float, fy: float, cx: float, cy: float,
                       poses32_dev, tile: int, stream=None) -> float:
    """pilot_probe_gather_frame: the build pass' loads on a real frame at one level, no
    arithmetic; returns (anchor, pose) units per second."""
    H, W, C = map_dev.shape
    N = points_dev.shape[-1]
    M = poses32_dev.shape[0]
    v = ct.c_double()
    check(load().pilot_probe_gather_frame(_ptr(points_dev), int(N), _ptr(map_dev), _ptr(ref_dev), int(H), int(W),
                                          int(C), int(dtype), float(fx), float(fy), float(cx), float(cy),
                                          _ptr(poses32_dev), int(M), int(tile), ct.byref(v), Solver._stream(stream)))
    return v.value


def quantize_features(src, dtype: int, per_channel: bool = False, stream=None):
    """pilot_quantize_features on a contiguous FP32 CUDA tensor (..., C): returns the
    quantised tensor (torch bfloat16 / float16 / uint8 bytes for E4M3) and the C scales."""
    import torch
    src = src.contiguous()
    C = int(src.shape[-1])
    rows = src.numel() // C
    tdt = {BF16: torch.bfloat16, F16: torch.float16, FP8E4M3: torch.uint8}[dtype]
    dst = torch.empty(src.shape, dtype=tdt, device=src.device)
    scale = torch.empty(C, dtype=torch.float32, device=src.device)
    check(load().pilot_quantize_features(src.data_ptr(), rows, C, dtype, int(per_channel), dst.data_ptr(),
                                         scale.data_ptr(), Solver._stream(stream)))
    return dst, scale


def quantized_device_arrays(frame, dtype: int, per_channel: bool = False, T_hyps=None, device="cuda") -> dict:
    """Device arrays of a frame with the query maps and reference descriptors quantised on
    the GPU (each map and each reference block with its own per-channel scales).  BF16 and
    FP16 without per-channel scaling store the values themselves (every scale is exactly 1),
    so no scale arrays are passed and the solver takes its unscaled path (the same values)."""
    arrs = device_arrays(frame, T_hyps, device)
    if dtype == F32:
        return arrs
    qf, qs, rf, rs = [], [], [], []
    for q, r in zip(arrs["qry_feat"], arrs["ref_feat"]):
        a, sa = quantize_features(q, dtype, per_channel)
        b, sb = quantize_features(r, dtype, per_channel) if r.numel() else (r.to(a.dtype), sa.clone())
        qf.append(a); qs.append(sa); rf.append(b); rs.append(sb)
    arrs.update(qry_feat=qf, ref_feat=rf)
    if dtype == FP8E4M3 or per_channel:
        arrs.update(qry_scale=qs, ref_scale=rs)
    return arrs


def validate(opts: Options, fa: FrameArgs) -> tuple[int, str]:
    cfg = opts.to_c()
    st = load().pilot_align_validate(ct.byref(cfg), ct.byref(fa.c))
    return st, pilot_align_last_error()


class Server:
    """pilot_serve_*: continuous-batching server over one CUDA device."""

    def __init__(self, opts: Options, hbm_budget: int, max_slots: int):
        lib = load()
        self._cfg = opts.to_c()
        h = _vp()
        check(lib.pilot_serve_create(ct.byref(self._cfg), int(hbm_budget), int(max_slots), ct.byref(h)))
        self.h = h
        self._frames = {}

    def set_levels_per_round(self, levels: int):
        """pilot_serve_set_levels_per_round (before the first submit; 0 = chosen per frame by size)."""
        check(load().pilot_serve_set_levels_per_round(self.h, int(levels)))

    def set_reserved_sms(self, n_sms: int):
        """pilot_serve_set_reserved_sms (before the first submit): CTA slots of n_sms SMs left
        free of the rounds, for client work on other streams."""
        check(load().pilot_serve_set_reserved_sms(self.h, int(n_sms)))

    def submit(self, fa: FrameArgs) -> int:
        """Queue a frame; returns its ticket (raises PilotError, status PILOT_EBUSY, when the
        pending queue is full).  `fa` is kept alive until the ticket is collected."""
        t = ct.c_uint64()
        check(load().pilot_serve_submit(self.h, ct.byref(fa.c), ct.byref(t)))
        self._frames[t.value] = fa
        return t.value

    def _result_bufs(self, M):
        o = dict(T=np.zeros((M, 12)), cost=np.zeros(M), nv=np.zeros(M, np.int32), st=np.zeros(M, np.int32),
                 best=np.zeros(1, np.int32), hi=np.zeros(1, np.int64))
        r = pilot_result(o["T"].ctypes.data, o["cost"].ctypes.data, o["nv"].ctypes.data, o["st"].ctypes.data,
                         o["best"].ctypes.data, o["hi"].ctypes.data)
        return o, r

    def poll(self, ticket: int):
        """(done, Result or None, latency_ms)."""
        fa = self._frames[ticket]
        o, r = self._result_bufs(fa.M)
        done = ct.c_int()
        lat = ct.c_double()
        check(load().pilot_serve_poll(self.h, ct.c_uint64(ticket), ct.byref(r), ct.byref(done), ct.byref(lat)))
        if not done.value:
            return False, None, None
        del self._frames[ticket]
        return True, Result(o["T"], o["cost"], o["nv"], o["st"], int(o["best"][0]), int(o["hi"][0])), lat.value

    def wait(self, ticket: int, timeout_ms: int = 600000):
        fa = self._frames[ticket]
        o, r = self._result_bufs(fa.M)
        lat = ct.c_double()
        check(load().pilot_serve_wait(self.h, ct.c_uint64(ticket), ct.byref(r), ct.byref(lat), int(timeout_ms)))
        del self._frames[ticket]
        return Result(o["T"], o["cost"], o["nv"], o["st"], int(o["best"][0]), int(o["hi"][0])), lat.value

    def stats(self) -> dict:
        st = pilot_serve_stats()
        check(load().pilot_serve_get_stats(self.h, ct.cast(ct.byref(st), _vp)))
        return {n: getattr(st, n) for n, _ in pilot_serve_stats._fields_}

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            load().pilot_serve_destroy(self.h)
            self.h = None
            self._frames.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
