"""C-ABI checks that need no GPU: the CUDA library builds and loads, it exports every
function include/*.h declares, and the host-side validation rejects malformed frames
with PILOT_EINVAL (no compute call is made here)."""
import ctypes as ct
import glob
import os
import re

import numpy as np
import pytest

from paper_2606_31098_gb300 import binding as B
from paper_2606_31098_gb300 import build_ext
from paper_2606_31098_gb300 import scenes as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build_ext.build()
    return B.load()


def declared_functions():
    names = []
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(pilot_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_function(lib):
    names = declared_functions()
    assert "pilot_align_solve" in names and "pilot_align_create" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"
    assert set(names) <= set(B.SIGNATURES) | set(getattr(B, "EXTRA_SIGNATURES", {}))


def small_host_frame(**over):
    f = S.make_frame(S.config_reduced_frame(crop_side=16, n_hyps=3), 5)
    return f, B.host_arrays(f)


def test_validate_accepts_a_good_frame(lib):
    f, arrs = small_host_frame()
    st, msg = B.validate(B.Options(), B.FrameArgs(f, arrs, is_device=False))
    assert st == B.PILOT_OK, msg


@pytest.mark.parametrize("mutation,needle", [
    (lambda c: setattr(c, "C", 12), "C = 12"),
    (lambda c: setattr(c, "L", 0), "L = 0"),
    (lambda c: setattr(c, "L", 5), "L = 5"),
    (lambda c: setattr(c, "N", -1), "N = -1"),
    (lambda c: setattr(c, "M", 100000), "M = 100000"),
    (lambda c: setattr(c, "fx", 0.0), "intrinsics"),
    (lambda c: setattr(c, "fy", float("nan")), "intrinsics"),
    (lambda c: c.H.__setitem__(0, 1), "both sides"),
    (lambda c: setattr(c, "feat_dtype", 9), "feat_dtype"),
    (lambda c: setattr(c, "points", None), "points"),
    (lambda c: setattr(c, "T_cw", None), "T_cw"),
    (lambda c: c.qry_feat.__setitem__(1, None), "qry_feat[1]"),
    (lambda c: c.qry_feat.__setitem__(0, c.qry_feat[0] + 4), "aligned"),
    (lambda c: setattr(c, "dsm", None), "DSM"),
    (lambda c: setattr(c, "dsm_gsd", 0.0), "gsd"),
    (lambda c: setattr(c, "w_grav", -1.0), "w_grav"),
])
def test_validate_rejects_malformed_frames(lib, mutation, needle):
    f, arrs = small_host_frame()
    fa = B.FrameArgs(f, arrs, is_device=False)
    mutation(fa.c)
    st, msg = B.validate(B.Options(), fa)
    assert st == B.PILOT_EINVAL
    assert needle in msg


def test_device_feature_pointers_need_32_byte_alignment(lib):
    """Device maps are read with loads of up to 32 bytes; host frames are staged into the
    solver's own buffers and need only 16.  Validation reads no memory, so the pointer
    values alone are checked here."""
    f, arrs = small_host_frame()
    for is_device, ok in ((1, False), (0, True)):
        fa = B.FrameArgs(f, arrs, is_device=False)
        fa.c.is_device = is_device
        fa.c.qry_feat[0] = (fa.c.qry_feat[0] // 32) * 32 + 16     # 16- but not 32-byte aligned
        st, msg = B.validate(B.Options(), fa)
        if ok:
            assert st == B.PILOT_OK, msg
        else:
            assert st == B.PILOT_EINVAL and "32-byte aligned" in msg


@pytest.mark.parametrize("field,value", [("lambda0", -1.0), ("damping_mode", 3), ("huber_photo", -0.1),
                                         ("min_valid_frac", 1.5), ("max_channels", 12), ("gate_range", -1.0),
                                         ("gate_grav", float("nan"))])
def test_validate_rejects_bad_options(lib, field, value):
    f, arrs = small_host_frame()
    opts = B.Options()
    setattr(opts, field, value)
    st, _ = B.validate(opts, B.FrameArgs(f, arrs, is_device=False))
    assert st == B.PILOT_EINVAL


def test_frame_beyond_the_handle_size_is_rejected(lib):
    f, arrs = small_host_frame()
    st, msg = B.validate(B.Options(max_points=100), B.FrameArgs(f, arrs, is_device=False))
    assert st == B.PILOT_EINVAL and "max_points" in msg


def test_null_arguments_are_errors_not_crashes(lib):
    assert lib.pilot_align_validate(None, None) == B.PILOT_EINVAL
    assert lib.pilot_align_create(None, None) == B.PILOT_EINVAL
    assert lib.pilot_align_solve(None, None, None, None) == B.PILOT_EINVAL
    lib.pilot_align_destroy(None)
    assert isinstance(B.pilot_align_last_error(), str)


def test_confidence_map_alignment_is_checked(lib):
    f, arrs = small_host_frame()
    buf = np.zeros(f.qry_feat[0].shape[0] * f.qry_feat[0].shape[1] + 1, np.float32)
    fa = B.FrameArgs(f, arrs, is_device=False)
    fa.c.qry_conf[0] = buf.ctypes.data + 2            # not 4-byte aligned
    st, msg = B.validate(B.Options(), fa)
    assert st == B.PILOT_EINVAL and "confidence" in msg


def test_tracking_entry_points_reject_bad_arguments_before_any_launch(lib):
    """pilot_seed_hypotheses and pilot_crop_reference validate on the host: these calls fail
    without touching a device."""
    T = np.eye(3, 4).ravel()
    p = B.seed_params(T, [0.0], [0.0])
    p.n_xy = 0
    assert lib.pilot_seed_hypotheses(ct.byref(p), None, None) == B.PILOT_EINVAL
    p.n_xy = 1
    assert lib.pilot_seed_hypotheses(ct.byref(p), 3, None) == B.PILOT_EINVAL       # misaligned output
    p.T_prior[0] = float("inf")
    assert lib.pilot_seed_hypotheses(ct.byref(p), 8, None) == B.PILOT_EINVAL
    assert lib.pilot_pose_predict(None, None, 1, None) == B.PILOT_EINVAL
    assert lib.pilot_pose_reorigin(None, 0.0, 0.0, None) == B.PILOT_EINVAL
    assert lib.pilot_crop_reference(None, None, None, None, None, None, None) == B.PILOT_EINVAL
