"""pilot_align_normal_eq_noalloc: the build-pass normal equations for callers that cannot
allocate device memory (an external pool owns it, or a latency-bound loop cannot risk an
allocation's implicit device synchronisation).  The entry point keeps its scratch in a
fixed file-scope device array and writes into a caller-provided device buffer.

Checked through the C-ABI against the handle-based pilot_align_debug_normal_eq on the
same inputs, on two calls in a row with different pose counts (the second call must not
see the first call's scratch).  Both run the same build kernel with the same 1024-anchor
tile and the same FP64 tile sum, so the values must be bitwise equal -- on FP32 maps, on
BF16 maps with per-channel scales, and on FP8 maps with scales and query confidence maps.
One case is also compared with the FP64 oracle directly, and the size limits are checked.
This file is named to be collected last so that a run stopping at the first failure has
run every other test first; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_2606_31098_gb300 import binding as B
from paper_2606_31098_gb300 import scenes as S

from gpu_support import (assert_normal_eq_close, boundary_mask, device_frame, fp32_pose, oracle_normal_eq,
                         require_cuda, to_oracle_opts)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


def noalloc(torch, opts, fa, level, T):
    T_dev = torch.as_tensor(np.ascontiguousarray(T, np.float64), device="cuda")
    out = torch.full((T.shape[0], 29), float("nan"), dtype=torch.float64, device="cuda")
    st = B.normal_eq_noalloc(opts, fa, level, T_dev, out)
    assert st == B.PILOT_OK, B.pilot_align_last_error()
    torch.cuda.synchronize()
    return out.cpu().numpy()


def two_calls(f):
    rng = np.random.default_rng(0)
    return [np.vstack([f.T_gt[None, :], f.T_hyps]), f.T_hyps[rng.permutation(f.M)[:3]]]


def frame_args(f, dt, T, per_channel=False):
    if dt == B.F32:
        return device_frame(f, T)
    return B.FrameArgs(f, B.quantized_device_arrays(f, dt, per_channel=per_channel, T_hyps=T), is_device=True,
                       dtype=dt)


@pytest.mark.parametrize("case", ["f32", "bf16_scaled", "fp8_scaled_confidence"])
def test_noalloc_equals_the_handle_entry_point_bitwise_on_two_calls(torch, case):
    f = S.make_frame(S.config_reduced_frame(n_hyps=6), S.frame_seed(2, 700))
    dt = {"f32": B.F32, "bf16_scaled": B.BF16, "fp8_scaled_confidence": B.FP8E4M3}[case]
    if case == "fp8_scaled_confidence":
        f = S.with_query_confidence(f, 71)
    opts = B.Options()
    solver = B.Solver(opts)
    for call, T in enumerate(two_calls(f)):
        fa = frame_args(f, dt, T, per_channel=(case == "bf16_scaled"))
        for level in (0, 2):
            ref = solver.normal_eq(fa, level, T)
            got = noalloc(torch, opts, fa, level, T)
            assert np.all(np.isfinite(got))
            np.testing.assert_array_equal(got, ref, err_msg=f"{case} call {call} level {level}")
    solver.close()


def test_noalloc_reads_a_missing_scale_as_ones_like_the_handle_entry_point(torch):
    f = S.make_frame(S.config_reduced_frame(crop_side=40, n_hyps=3), S.frame_seed(2, 701))
    arrs = B.quantized_device_arrays(f, B.BF16, per_channel=True)
    arrs["ref_scale"] = None                      # only the query scales are given
    fa = B.FrameArgs(f, arrs, is_device=True, dtype=B.BF16)
    opts = B.Options()
    solver = B.Solver(opts)
    for level in (0, 1):
        np.testing.assert_array_equal(noalloc(torch, opts, fa, level, f.T_hyps),
                                      solver.normal_eq(fa, level, f.T_hyps))
    solver.close()


def test_noalloc_matches_the_oracle(torch):
    f = S.make_frame(S.config_reduced_frame(n_hyps=4), S.frame_seed(2, 702))
    poses = np.vstack([f.T_gt[None, :], f.T_hyps])
    poses32 = [fp32_pose(T) for T in poses]
    f = f.replace(point_valid=boundary_mask(f, [0, 2], poses32))
    opts = B.Options()
    oo = to_oracle_opts(opts)
    fa = device_frame(f, poses)
    for level in (0, 2):
        got = noalloc(torch, opts, fa, level, poses)
        for m, T in enumerate(poses):
            assert_normal_eq_close(got[m], oracle_normal_eq(f, oo, level, T), what=f"level {level} pose {m}")


def test_noalloc_rejects_sizes_beyond_its_scratch(torch):
    f = S.make_frame(S.config_reduced_frame(crop_side=20, n_hyps=2), 5)
    T = np.repeat(f.T_hyps[:1], 257, axis=0)
    fa = device_frame(f, T)
    T_dev = torch.as_tensor(T, device="cuda")
    out = torch.zeros((257, 29), dtype=torch.float64, device="cuda")
    assert B.normal_eq_noalloc(B.Options(max_hyps=512), fa, 0, T_dev, out) == B.PILOT_EINVAL
    assert "256" in B.pilot_align_last_error()
    # the caller's workspace sizes do not limit this call: 100 poses pass with max_hyps = 64
    fa100 = device_frame(f, T[:100])
    assert B.normal_eq_noalloc(B.Options(max_hyps=64), fa100, 0, T_dev[:100], out[:100]) == B.PILOT_OK
    torch.cuda.synchronize()
    host = B.FrameArgs(f, B.host_arrays(f), is_device=False)
    assert B.normal_eq_noalloc(B.Options(), host, 0, T_dev[:2], out[:2]) == B.PILOT_EINVAL
    assert "device frame" in B.pilot_align_last_error()
