"""Sensor-prior residual gates on the GPU (Supp. "Sensor-Prior Fusion in LM"; a residual
above its gate adds a constant and no pull): with a range reading several metres off and a
tilted IMU reading, the gated solve agrees with the FP64 oracle hypothesis by hypothesis and
in its selection, and the gates change the result (they are not ignored)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_31098_gb300 import binding as B
from paper_2606_31098_gb300 import scenes as S

from gpu_support import assert_selection_agrees, assert_solutions_agree, device_frame, require_cuda, to_oracle_opts

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


def bad_sensor_frame(seed):
    f = S.make_frame(S.config_reduced_frame(n_hyps=6), S.frame_seed(2, seed))
    g = f.gravity_cam + np.array([0.0, 0.08, 0.0])
    return f.replace(gravity_cam=g / np.linalg.norm(g), range_m=f.range_m + 6.0)


@pytest.mark.parametrize("gates", [(0.05, 2.0), (0.2, 2.5), (0.0, 1.0)])
def test_gated_solve_matches_the_oracle(torch, gates):
    """Both gates closed at the solution; the gravity gate open (residual 0.05 < 0.2) with
    the range gate closed; the range gate alone."""
    f = bad_sensor_frame(950)
    opts = B.Options(gate_grav=gates[0], gate_range=gates[1])
    g = B.Solver(opts).solve(device_frame(f))
    o = O.solve(f, to_oracle_opts(opts))
    assert_solutions_agree(f, opts, g, o, min_converged=2)
    assert_selection_agrees(f, opts, g, o)


def test_gates_change_the_objective(torch):
    f = bad_sensor_frame(951)
    fa = device_frame(f)
    open_ = B.Solver(B.Options()).solve(fa)
    gated = B.Solver(B.Options(gate_grav=0.05, gate_range=2.0)).solve(fa)
    assert not np.allclose(open_.cost, gated.cost)
    # the gated solve ignores the bad readings: its pose is closer to the ground truth
    e_open = S.translation_error_m(open_.T_cw[open_.best], f.T_gt)
    e_gated = S.translation_error_m(gated.T_cw[gated.best], f.T_gt)
    assert e_gated < e_open


def test_negative_gate_is_rejected(torch):
    with pytest.raises(B.PilotError, match="gates"):
        B.Solver(B.Options(gate_range=-1.0))


def test_gated_forms_agree_bitwise(torch):
    """The gates sit in the FP64 step every form shares: plain, batched and served solves of
    frames with bad readings give bitwise the same outputs."""
    from test_gpu_batch import args_for, assert_same
    frames = [bad_sensor_frame(960 + i) for i in range(2)]
    opts = B.Options(iters=(3, 3, 3, 0), gate_grav=0.05, gate_range=2.0)
    solver = B.Solver(opts)
    fas = args_for(frames)
    plain = [solver.solve(fa) for fa in fas]
    batch = solver.solve_batch(fas)
    for i in range(2):
        assert_same(batch[i], plain[i], what=f"batched frame {i}")
    server = B.Server(opts, 1 << 30, max_slots=4)
    res, _ = server.wait(server.submit(fas[0]))
    assert_same(res, plain[0], what="served frame")
    server.close()
