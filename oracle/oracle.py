"""ctypes binding of the FP64 CPU oracle (test infrastructure only).

Only the test suite, the smoke check and the benchmark's CPU-baseline leg import this
module.  It loads oracle/_lib/libpilot_oracle.so (built by oracle/build_oracle.py) and
marshals a synthetic frame (numpy arrays) into the oracle's own C structures, which are
declared in oracle/pilot_oracle.h and share nothing with the CUDA library.
"""
from __future__ import annotations

import ctypes as ct
import os
from dataclasses import dataclass, field

import numpy as np

from . import build_oracle

MAX_LEVELS = 4
HYP_OK, HYP_FEW_VALID, HYP_NOT_PD, HYP_NONFINITE, HYP_PRUNED = range(5)

_f32p = ct.POINTER(ct.c_float)
_f64p = ct.POINTER(ct.c_double)
_u8p = ct.POINTER(ct.c_ubyte)
_i32p = ct.POINTER(ct.c_int)
_i64p = ct.POINTER(ct.c_longlong)


class OrFrame(ct.Structure):
    _fields_ = [
        ("N", ct.c_int), ("points", _f32p), ("point_weight", _f32p), ("point_valid", _u8p),
        ("C", ct.c_int), ("L", ct.c_int),
        ("ref_feat", _f32p * MAX_LEVELS), ("qry_feat", _f32p * MAX_LEVELS), ("qry_conf", _f32p * MAX_LEVELS),
        ("H", ct.c_int * MAX_LEVELS), ("W", ct.c_int * MAX_LEVELS),
        ("fx", ct.c_double), ("fy", ct.c_double), ("cx", ct.c_double), ("cy", ct.c_double),
        ("M", ct.c_int), ("T_cw", _f64p),
        ("use_gravity", ct.c_int), ("gravity_cam", ct.c_double * 3),
        ("gravity_world", ct.c_double * 3), ("w_grav", ct.c_double),
        ("use_range", ct.c_int), ("range_m", ct.c_double), ("w_range", ct.c_double),
        ("dsm", _f32p), ("dsm_H", ct.c_int), ("dsm_W", ct.c_int),
        ("dsm_x0", ct.c_double), ("dsm_y0", ct.c_double), ("dsm_gsd", ct.c_double),
    ]


class OrConfig(ct.Structure):
    _fields_ = [
        ("iters", ct.c_int * MAX_LEVELS), ("lambda0", ct.c_double), ("damping_mode", ct.c_int),
        ("huber_photo", ct.c_double), ("huber_grav", ct.c_double), ("huber_range", ct.c_double),
        ("keep_top_k", ct.c_int * MAX_LEVELS), ("min_valid_frac", ct.c_double),
        ("gate_grav", ct.c_double), ("gate_range", ct.c_double),
    ]


class OrResult(ct.Structure):
    _fields_ = [("T_cw", _f64p), ("cost", _f64p), ("n_valid", _i32p), ("status", _i32p),
                ("best", _i32p), ("hyp_iters", _i64p)]


@dataclass
class SolverOptions:
    """Solver options, identical in meaning to the CUDA library's configuration."""

    iters: tuple = (10, 10, 10, 0)
    lambda0: float = 1e-3
    damping_mode: int = 0
    huber_photo: float = 0.1
    huber_grav: float = 0.1
    huber_range: float = 1.0
    keep_top_k: tuple = (0, 0, 0, 0)
    min_valid_frac: float = 0.05
    gate_grav: float = 0.0            # prior residual gates; 0 = off
    gate_range: float = 0.0


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build_oracle.build()
        L = ct.CDLL(path)
        L.or_so3_exp.argtypes = [_f64p, _f64p]
        L.or_se3_exp.argtypes = [_f64p, _f64p]
        L.or_se3_log.argtypes = [_f64p, _f64p]
        L.or_pose_update.argtypes = [_f64p, _f64p, _f64p]
        L.or_huber.argtypes = [ct.c_double, ct.c_double, _f64p, _f64p]
        L.or_bilinear.argtypes = [_f32p, ct.c_int, ct.c_int, ct.c_int, ct.c_double, ct.c_double,
                                  _f64p, _f64p, _f64p]
        L.or_bilinear.restype = ct.c_int
        L.or_point_residual.argtypes = [ct.POINTER(OrFrame), ct.c_int, _f64p, ct.c_int, _f64p, _f64p]
        L.or_point_residual.restype = ct.c_int
        L.or_point_margin.argtypes = [ct.POINTER(OrFrame), ct.c_int, _f64p, ct.c_int]
        L.or_point_margin.restype = ct.c_double
        L.or_query_confidence.argtypes = [ct.POINTER(OrFrame), ct.c_int, _f64p, ct.c_int]
        L.or_query_confidence.restype = ct.c_double
        L.or_photo_terms.argtypes = [ct.POINTER(OrFrame), ct.POINTER(OrConfig), ct.c_int, _f64p,
                                     _f64p, _f64p, _f64p, _i32p]
        L.or_gravity_terms.argtypes = [ct.POINTER(OrFrame), ct.POINTER(OrConfig), _f64p, _f64p, _f64p, _f64p]
        L.or_range_terms.argtypes = [ct.POINTER(OrFrame), ct.POINTER(OrConfig), _f64p, _f64p, _f64p, _f64p]
        L.or_range_terms.restype = ct.c_int
        L.or_gravity_residual.argtypes = [ct.POINTER(OrFrame), _f64p, _f64p, _f64p]
        L.or_range_residual.argtypes = [ct.POINTER(OrFrame), _f64p, _f64p, _f64p]
        L.or_range_residual.restype = ct.c_int
        L.or_evaluate.argtypes = [ct.POINTER(OrFrame), ct.POINTER(OrConfig), ct.c_int, _f64p, _f64p]
        L.or_cholesky_solve.argtypes = [_f64p, _f64p, _f64p]
        L.or_cholesky_solve.restype = ct.c_int
        L.or_solve.argtypes = [ct.POINTER(OrFrame), ct.POINTER(OrConfig), ct.POINTER(OrResult), ct.c_int]
        L.or_lm_level.argtypes = [ct.POINTER(OrFrame), ct.POINTER(OrConfig), ct.c_int, _f64p, _f64p, _i32p]
        L.or_num_threads.restype = ct.c_int
        _lib = L
    return _lib


def _p(a, typ):
    return a.ctypes.data_as(typ)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleFrame:
    """Holds the numpy arrays alive and the OrFrame that points into them."""

    def __init__(self, frame, T_hyps=None, ref_feat=None, qry_feat=None):
        self.keep = []
        f = OrFrame()
        pts = np.ascontiguousarray(frame.points, np.float32)
        N = pts.shape[1]
        f.N = N
        f.points = self._k(pts, _f32p)
        f.point_weight = self._k(np.ascontiguousarray(frame.point_weight, np.float32), _f32p) \
            if frame.point_weight is not None else None
        f.point_valid = self._k(np.ascontiguousarray(frame.point_valid, np.uint8), _u8p) \
            if frame.point_valid is not None else None
        refs = ref_feat if ref_feat is not None else frame.ref_feat
        qrys = qry_feat if qry_feat is not None else frame.qry_feat
        f.L = len(qrys)
        f.C = qrys[0].shape[2]
        confs = getattr(frame, "qry_conf", None)
        for l in range(f.L):
            f.ref_feat[l] = self._k(np.ascontiguousarray(refs[l], np.float32), _f32p)
            f.qry_feat[l] = self._k(np.ascontiguousarray(qrys[l], np.float32), _f32p)
            c = None if confs is None else confs[l]
            f.qry_conf[l] = None if c is None else self._k(np.ascontiguousarray(c, np.float32), _f32p)
            f.H[l], f.W[l] = qrys[l].shape[0], qrys[l].shape[1]
        f.fx, f.fy, f.cx, f.cy = frame.fx, frame.fy, frame.cx, frame.cy
        T = _f64(frame.T_hyps if T_hyps is None else T_hyps).reshape(-1, 12)
        f.M = T.shape[0]
        f.T_cw = self._k(T, _f64p)
        f.use_gravity = int(frame.use_gravity)
        f.gravity_cam[:] = list(frame.gravity_cam)
        f.gravity_world[:] = list(frame.gravity_world)
        f.w_grav = frame.w_grav
        f.use_range = int(frame.use_range)
        f.range_m = frame.range_m
        f.w_range = frame.w_range
        f.dsm = self._k(np.ascontiguousarray(frame.dsm, np.float32), _f32p)
        f.dsm_H, f.dsm_W = frame.dsm.shape
        f.dsm_x0, f.dsm_y0, f.dsm_gsd = frame.dsm_x0, frame.dsm_y0, frame.dsm_gsd
        self.c = f
        self.M = f.M

    def _k(self, a, typ):
        self.keep.append(a)
        return _p(a, typ)


def make_config(opts: SolverOptions) -> OrConfig:
    c = OrConfig()
    c.iters[:] = list(opts.iters) + [0] * (MAX_LEVELS - len(opts.iters))
    c.lambda0 = opts.lambda0
    c.damping_mode = opts.damping_mode
    c.huber_photo, c.huber_grav, c.huber_range = opts.huber_photo, opts.huber_grav, opts.huber_range
    c.keep_top_k[:] = list(opts.keep_top_k) + [0] * (MAX_LEVELS - len(opts.keep_top_k))
    c.min_valid_frac = opts.min_valid_frac
    c.gate_grav, c.gate_range = opts.gate_grav, opts.gate_range
    return c


@dataclass
class SolveResult:
    T_cw: np.ndarray
    cost: np.ndarray
    n_valid: np.ndarray
    status: np.ndarray
    best: int
    hyp_iters: int
    extra: dict = field(default_factory=dict)


def solve(frame, opts: SolverOptions, T_hyps=None, n_threads: int = 0, ref_feat=None,
          qry_feat=None) -> SolveResult:
    """Run the whole multi-hypothesis coarse-to-fine LM solve on the CPU in FP64."""
    of = OracleFrame(frame, T_hyps=T_hyps, ref_feat=ref_feat, qry_feat=qry_feat)
    M = of.M
    T = np.zeros((M, 12))
    cost = np.zeros(M)
    nv = np.zeros(M, np.int32)
    st = np.zeros(M, np.int32)
    best = np.zeros(1, np.int32)
    hi = np.zeros(1, np.int64)
    r = OrResult(_p(T, _f64p), _p(cost, _f64p), _p(nv, _i32p), _p(st, _i32p), _p(best, _i32p),
                 _p(hi, _i64p))
    c = make_config(opts)
    lib().or_solve(ct.byref(of.c), ct.byref(c), ct.byref(r), int(n_threads))
    return SolveResult(T, cost, nv, st, int(best[0]), int(hi[0]))


def evaluate(frame, opts: SolverOptions, level: int, T, **kw) -> np.ndarray:
    """H(21) | g(6) | cost | n_valid at pose T and `level` (Eq. 7 and its normal equation)."""
    of = OracleFrame(frame, T_hyps=np.asarray(T).reshape(1, 12), **kw)
    out = np.zeros(29)
    c = make_config(opts)
    lib().or_evaluate(ct.byref(of.c), ct.byref(c), int(level), _p(_f64(T), _f64p), _p(out, _f64p))
    return out


def evaluate_many(frame, opts: SolverOptions, level: int, Ts, **kw) -> np.ndarray:
    of = OracleFrame(frame, T_hyps=np.asarray(Ts).reshape(-1, 12), **kw)
    c = make_config(opts)
    out = np.zeros((len(Ts), 29))
    for m, T in enumerate(np.asarray(Ts).reshape(-1, 12)):
        row = np.zeros(29)
        lib().or_evaluate(ct.byref(of.c), ct.byref(c), int(level), _p(_f64(T), _f64p), _p(row, _f64p))
        out[m] = row
    return out


def photo_terms(frame, opts, level, T, **kw):
    of = OracleFrame(frame, T_hyps=np.asarray(T).reshape(1, 12), **kw)
    c = make_config(opts)
    H = np.zeros(21)
    g = np.zeros(6)
    cost = np.zeros(1)
    n = np.zeros(1, np.int32)
    lib().or_photo_terms(ct.byref(of.c), ct.byref(c), int(level), _p(_f64(T), _f64p),
                         _p(H, _f64p), _p(g, _f64p), _p(cost, _f64p), _p(n, _i32p))
    return H, g, float(cost[0]), int(n[0])


def point_residual(frame, level, T, j, with_jacobian=True, **kw):
    of = OracleFrame(frame, T_hyps=np.asarray(T).reshape(1, 12), **kw)
    C = of.c.C
    r = np.zeros(C)
    J = np.zeros((C, 6))
    vis = lib().or_point_residual(ct.byref(of.c), int(level), _p(_f64(T), _f64p), int(j),
                                  _p(r, _f64p), _p(J, _f64p) if with_jacobian else None)
    return bool(vis), r, J


def query_confidences(frame, level, T, **kw) -> np.ndarray:
    """w^q_l at every anchor's projection under T (0 where not visible)."""
    of = OracleFrame(frame, **kw)
    Tp = _p(_f64(T), _f64p)
    return np.array([lib().or_query_confidence(ct.byref(of.c), int(level), Tp, j) for j in range(of.c.N)])


def point_margins(frame, level, T, **kw) -> np.ndarray:
    of = OracleFrame(frame, T_hyps=np.asarray(T).reshape(1, 12), **kw)
    Tp = _p(_f64(T), _f64p)
    return np.array([lib().or_point_margin(ct.byref(of.c), int(level), Tp, j) for j in range(of.c.N)])


def prior_terms(frame, opts: SolverOptions, which: str, T):
    """H (21), g (6) and cost of one sensor prior ("gravity" or "range") at pose T."""
    of = OracleFrame(frame, T_hyps=np.asarray(T).reshape(1, 12))
    c = make_config(opts)
    H, g, cost = np.zeros(21), np.zeros(6), np.zeros(1)
    fn = lib().or_gravity_terms if which == "gravity" else lib().or_range_terms
    fn(ct.byref(of.c), ct.byref(c), _p(_f64(T), _f64p), _p(H, _f64p), _p(g, _f64p), _p(cost, _f64p))
    return H, g, float(cost[0])


def gravity_residual(frame, T):
    of = OracleFrame(frame, T_hyps=np.asarray(T).reshape(1, 12))
    r = np.zeros(3)
    J = np.zeros((3, 6))
    lib().or_gravity_residual(ct.byref(of.c), _p(_f64(T), _f64p), _p(r, _f64p), _p(J, _f64p))
    return r, J


def range_residual(frame, T):
    of = OracleFrame(frame, T_hyps=np.asarray(T).reshape(1, 12))
    r = np.zeros(1)
    J = np.zeros(6)
    ok = lib().or_range_residual(ct.byref(of.c), _p(_f64(T), _f64p), _p(r, _f64p), _p(J, _f64p))
    return bool(ok), float(r[0]), J


def so3_exp(w):
    R = np.zeros(9)
    lib().or_so3_exp(_p(_f64(w), _f64p), _p(R, _f64p))
    return R.reshape(3, 3)


def se3_exp(xi):
    T = np.zeros(12)
    lib().or_se3_exp(_p(_f64(xi), _f64p), _p(T, _f64p))
    return T


def se3_log(T):
    xi = np.zeros(6)
    lib().or_se3_log(_p(_f64(T), _f64p), _p(xi, _f64p))
    return xi


def pose_update(xi, T):
    out = np.zeros(12)
    lib().or_pose_update(_p(_f64(xi), _f64p), _p(_f64(T), _f64p), _p(out, _f64p))
    return out


def huber(s, delta):
    rho = np.zeros(1)
    d = np.zeros(1)
    lib().or_huber(float(s), float(delta), _p(rho, _f64p), _p(d, _f64p))
    return float(rho[0]), float(d[0])


def bilinear(fmap, x, y):
    fmap = np.ascontiguousarray(fmap, np.float32)
    H, W, C = fmap.shape
    f = np.zeros(C)
    fx = np.zeros(C)
    fy = np.zeros(C)
    ok = lib().or_bilinear(_p(fmap, _f32p), H, W, C, float(x), float(y), _p(f, _f64p),
                           _p(fx, _f64p), _p(fy, _f64p))
    return bool(ok), f, fx, fy


def cholesky_solve(A, b):
    x = np.zeros(6)
    ok = lib().or_cholesky_solve(_p(_f64(A), _f64p), _p(_f64(b), _f64p), _p(x, _f64p))
    return bool(ok), x


def lm_level(frame, opts, level, T):
    of = OracleFrame(frame, T_hyps=np.asarray(T).reshape(1, 12))
    c = make_config(opts)
    Tw = _f64(T).copy()
    E = np.zeros(29)
    fail = np.zeros(1, np.int32)
    lib().or_lm_level(ct.byref(of.c), ct.byref(c), int(level), _p(Tw, _f64p), _p(E, _f64p), _p(fail, _i32p))
    return Tw, E, bool(fail[0])


def num_threads() -> int:
    return int(lib().or_num_threads())


def unpack_H(H21) -> np.ndarray:
    """Symmetric 6x6 from the 21-entry upper triangle (row-major)."""
    H = np.zeros((6, 6))
    k = 0
    for a in range(6):
        for b in range(a, 6):
            H[a, b] = H[b, a] = H21[k]
            k += 1
    return H
