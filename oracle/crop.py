"""ctypes wrapper of the FP64 CPU oracle of the TDOM/DSM reference crop (crop_oracle.c).

Test infrastructure: the plain reference the CUDA crop kernels are checked against
(Supp. "TDOM/DSM Reference Crop": map footprint from the corner rays, one homography
warping the TDOM / DSM / map-coordinate grids, geo-anchor lift).  Only tests/ and the
benchmark's CPU-baseline leg use it.
"""
from __future__ import annotations

import ctypes as ct

import numpy as np

from . import build_oracle

_f64p = ct.POINTER(ct.c_double)
_f32p = ct.POINTER(ct.c_float)
_u8p = ct.POINTER(ct.c_uint8)
_i32p = ct.POINTER(ct.c_int)


class OrcMap(ct.Structure):
    _fields_ = [("dsm", _f32p), ("tdom", _u8p), ("H", ct.c_int), ("W", ct.c_int),
                ("x0", ct.c_double), ("y0", ct.c_double), ("gsd", ct.c_double)]


class OrcParams(ct.Structure):
    _fields_ = [("T_cw", ct.c_double * 12), ("fx", ct.c_double), ("fy", ct.c_double),
                ("cx", ct.c_double), ("cy", ct.c_double), ("img_w", ct.c_int), ("img_h", ct.c_int),
                ("s_min", ct.c_double), ("s_step", ct.c_double), ("n_samples", ct.c_int), ("S", ct.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ct.CDLL(build_oracle.build())
        L.orc_dsm_height.argtypes = [ct.POINTER(OrcMap), ct.c_double, ct.c_double, _f64p]
        L.orc_dsm_height.restype = ct.c_int
        L.orc_footprint.argtypes = [ct.POINTER(OrcMap), ct.POINTER(OrcParams), _f64p, _i32p]
        L.orc_homography.argtypes = [_f64p, _f64p, _f64p]
        L.orc_homography.restype = ct.c_int
        L.orc_warp.argtypes = [ct.POINTER(OrcMap), _f64p, ct.c_int, ct.c_double, ct.c_double, _f32p, _u8p, _f32p]
        L.orc_crop.argtypes = [ct.POINTER(OrcMap), ct.POINTER(OrcParams), _f64p, _f32p, _u8p, _f32p]
        L.orc_crop.restype = ct.c_int
        _lib = L
    return _lib


class MapArgs:
    """An orc_map over numpy arrays kept alive with it."""

    def __init__(self, dsm: np.ndarray, tdom: np.ndarray | None, x0: float, y0: float, gsd: float):
        self.dsm = np.ascontiguousarray(dsm, np.float32)
        self.tdom = None if tdom is None else np.ascontiguousarray(tdom, np.uint8)
        self.c = OrcMap(self.dsm.ctypes.data_as(_f32p),
                        None if self.tdom is None else self.tdom.ctypes.data_as(_u8p),
                        self.dsm.shape[0], self.dsm.shape[1], x0, y0, gsd)


def params(T_cw, fx, fy, cx, cy, img_w, img_h, s_min, s_step, n_samples, S) -> OrcParams:
    p = OrcParams()
    p.T_cw[:] = [float(v) for v in np.asarray(T_cw, np.float64).ravel()]
    p.fx, p.fy, p.cx, p.cy = fx, fy, cx, cy
    p.img_w, p.img_h = img_w, img_h
    p.s_min, p.s_step, p.n_samples, p.S = s_min, s_step, n_samples, S
    return p


def dsm_height(m: MapArgs, x: float, y: float):
    h = ct.c_double()
    ok = lib().orc_dsm_height(ct.byref(m.c), x, y, ct.byref(h))
    return bool(ok), h.value


def footprint(m: MapArgs, p: OrcParams):
    quad = np.zeros(12)
    idx = np.zeros(4, np.int32)
    lib().orc_footprint(ct.byref(m.c), ct.byref(p), quad.ctypes.data_as(_f64p), idx.ctypes.data_as(_i32p))
    return quad.reshape(4, 3), idx


def homography(src, dst):
    src = np.ascontiguousarray(src, np.float64).ravel()
    dst = np.ascontiguousarray(dst, np.float64).ravel()
    H = np.zeros(9)
    ok = lib().orc_homography(src.ctypes.data_as(_f64p), dst.ctypes.data_as(_f64p), H.ctypes.data_as(_f64p))
    return bool(ok), H


def warp(m: MapArgs, H, S: int, ox: float, oy: float, with_rgb: bool = True):
    H = np.ascontiguousarray(H, np.float64)
    pts = np.zeros((3, S * S), np.float32)
    valid = np.zeros(S * S, np.uint8)
    rgb = np.zeros((S * S, 3), np.float32) if with_rgb else None
    lib().orc_warp(ct.byref(m.c), H.ctypes.data_as(_f64p), S, ox, oy, pts.ctypes.data_as(_f32p),
                   valid.ctypes.data_as(_u8p), None if rgb is None else rgb.ctypes.data_as(_f32p))
    return pts, valid, rgb


def crop(m: MapArgs, p: OrcParams, with_rgb: bool = True) -> dict:
    """Footprint, homography and warp; geometry = H[9], origin[2], quad[12], sample indices[4]."""
    S = p.S
    geom = np.zeros(27)
    pts = np.zeros((3, S * S), np.float32)
    valid = np.zeros(S * S, np.uint8)
    rgb = np.zeros((S * S, 3), np.float32) if with_rgb else None
    ok = lib().orc_crop(ct.byref(m.c), ct.byref(p), geom.ctypes.data_as(_f64p), pts.ctypes.data_as(_f32p),
                        valid.ctypes.data_as(_u8p), None if rgb is None else rgb.ctypes.data_as(_f32p))
    return dict(ok=bool(ok), H=geom[:9].copy(), origin=geom[9:11].copy(), quad=geom[11:23].reshape(4, 3).copy(),
                idx=geom[23:27].astype(np.int64), points=pts, valid=valid, rgb=rgb)
