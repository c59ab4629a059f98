"""Reduced-precision storage (BF16, FP16, FP8-E4M3 with per-channel scales, FP32 math).

* The GPU quantiser (pilot_quantize_features) produces exactly the codes the format
  definitions give (round to nearest even, E4M3 saturating at 448): bit-exact.
* Build pass and whole solve on quantised storage match the FP64 oracle fed the values
  the solver uses (stored value x scale), under the same tolerances as FP32.
* Against the FP64 oracle on the unquantised FP32 features, the selected pose's error
  per storage type is reported (and bounded loosely).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_31098_gb300 import binding as B
from paper_2606_31098_gb300 import scenes as S

from gpu_support import (assert_normal_eq_close, assert_selection_agrees, assert_solutions_agree,
                         boundary_mask, fp32_pose, oracle_normal_eq, pose_errors, require_cuda,
                         to_oracle_opts)
from precision_support import (BF16, F16, FP8, dequantize, encode_bf16_rne, encode_e4m3_satfinite,
                               to_numpy_bits)

pytestmark = pytest.mark.gpu

DTYPES = [(B.BF16, BF16), (B.F16, F16), (B.FP8E4M3, FP8)]


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


@pytest.mark.parametrize("dt,ref_dt", DTYPES)
@pytest.mark.parametrize("per_channel", [False, True])
def test_quantiser_matches_the_format_definitions(torch, dt, ref_dt, per_channel):
    rng = np.random.default_rng(3)
    C = 32
    x = (rng.standard_normal((5000, C)) * rng.uniform(0.01, 3.0, C)).astype(np.float32)
    x[0, :4] = [0.0, -0.0, 1e-12, -1e-12]
    x[1, 0] = 1e4                                         # saturates in E4M3 without scaling
    q, s = B.quantize_features(torch.as_tensor(x, device="cuda"), dt, per_channel)
    torch.cuda.synchronize()
    s = s.cpu().numpy()
    if per_channel or dt == B.FP8E4M3:
        qmax = {B.FP8E4M3: 448.0, B.F16: 65504.0, B.BF16: 1.0}[dt]
        expect_s = (np.abs(x).max(axis=0) / np.float32(qmax)).astype(np.float32)
    else:
        expect_s = np.ones(C, np.float32)
    np.testing.assert_array_equal(s, expect_s)
    y = x * (np.float32(1.0) / s)                           # FP32, as the kernel computes it
    got = to_numpy_bits(q)
    if ref_dt == BF16:
        want = encode_bf16_rne(y)
    elif ref_dt == F16:
        want = y.astype(np.float16).view(np.uint16)
    else:
        want = encode_e4m3_satfinite(y)
    np.testing.assert_array_equal(got, want)


def quantised_frame(torch, frame, dt, T=None):
    arrs = B.quantized_device_arrays(frame, dt, T_hyps=T)
    L = len(arrs["qry_feat"])
    deq = dict(qry_feat=[dequantize(q, s, {B.BF16: BF16, B.F16: F16, B.FP8E4M3: FP8}[dt]).reshape(q.shape)
                         for q, s in zip(arrs["qry_feat"], arrs.get("qry_scale") or [None] * L)],
               ref_feat=[dequantize(r, s, {B.BF16: BF16, B.F16: F16, B.FP8E4M3: FP8}[dt]).reshape(r.shape)
                         for r, s in zip(arrs["ref_feat"], arrs.get("ref_scale") or [None] * L)])
    return B.FrameArgs(frame, arrs, is_device=True, dtype=dt), frame.replace(**deq)


@pytest.mark.parametrize("dt,_", DTYPES)
def test_normal_equations_on_quantised_storage(torch, dt, _):
    f = S.make_frame(S.config_reduced_frame(n_hyps=3), S.frame_seed(2, 500))
    poses = [f.T_gt, *f.T_hyps]
    poses32 = [fp32_pose(T) for T in poses]
    valid = boundary_mask(f, [0, 1, 2], poses32)
    f = f.replace(point_valid=valid)
    fa, fdeq = quantised_frame(torch, f, dt, np.array(poses))
    solver = B.Solver(B.Options())
    oo = to_oracle_opts(B.Options())
    for level in (0, 1, 2):
        gpu = solver.normal_eq(fa, level, np.array(poses))
        for m, T in enumerate(poses):
            assert_normal_eq_close(gpu[m], oracle_normal_eq(fdeq, oo, level, T), what=f"level {level} pose {m}")


@pytest.mark.parametrize("dt,_", DTYPES)
def test_solve_on_quantised_storage_matches_dequantised_oracle(torch, dt, _):
    f = S.make_frame(S.config_reduced_frame(n_hyps=7), S.frame_seed(2, 200))
    fa, fdeq = quantised_frame(torch, f, dt)
    opts = B.Options()
    g = B.Solver(opts).solve(fa)
    o = O.solve(fdeq, to_oracle_opts(opts))
    assert_solutions_agree(fdeq, opts, g, o, min_converged=2)
    assert_selection_agrees(fdeq, opts, g, o)


def test_selected_pose_error_per_storage_type(torch):
    """The precision form's accuracy against the FP64 oracle on the FP32 features
    (the reduced-precision path is judged on equal pose accuracy)."""
    f = S.make_frame(S.config_reduced_frame(n_hyps=7), S.frame_seed(2, 201))
    opts = B.Options()
    o = O.solve(f, to_oracle_opts(opts))
    report = {}
    for dt in (B.F32, B.BF16, B.F16, B.FP8E4M3):
        arrs = B.quantized_device_arrays(f, dt)
        g = B.Solver(opts).solve(B.FrameArgs(f, arrs, is_device=True, dtype=dt))
        report[B.DTYPE_NAMES[dt]] = pose_errors(g.T_cw[g.best], o.T_cw[o.best])
    print("selected-pose error vs FP64 oracle (deg, m):", report)
    assert report["f32"][0] < 1e-3 and report["f32"][1] < 1e-3
    assert report["bf16"][0] < 0.05 and report["bf16"][1] < 0.25
    assert report["f16"][0] < 0.01 and report["f16"][1] < 0.05
    assert report["fp8e4m3"][0] < 0.2 and report["fp8e4m3"][1] < 1.0
