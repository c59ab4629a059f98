"""Query-confidence weighting on the GPU (Eq. 2's w_l(j) = anchor weight x w^q_l read
bilinearly at the projection; w^q_l is the query uncertainty map of Sec. IV-C): parity with the FP64 oracle
for the normal equations at every level and for the whole solve, and bitwise agreement of the
plain, host-staged, batched and served forms.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_31098_gb300 import binding as B
from paper_2606_31098_gb300 import scenes as S

from gpu_support import assert_selection_agrees, assert_solutions_agree, device_frame, require_cuda, to_oracle_opts
from test_gpu_batch import args_for, assert_same
from test_gpu_parity import check_normal_eq, random_poses

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


def conf_frame(seed, n_hyps=5, **kw):
    f = S.make_frame(S.config_reduced_frame(n_hyps=n_hyps, **kw), S.frame_seed(2, seed))
    return S.with_query_confidence(f, seed + 17)


def test_normal_equations_with_query_confidence(torch):
    f = conf_frame(610, n_hyps=2)
    poses = [f.T_gt, *f.T_hyps, *random_poses(f.T_gt, 2, 611)]
    check_normal_eq(f, B.Options(), [0, 1, 2], poses)


def test_solve_with_query_confidence_matches_the_oracle(torch):
    f = conf_frame(620, n_hyps=6)
    opts = B.Options()
    g = B.Solver(opts).solve(device_frame(f))
    o = O.solve(f, to_oracle_opts(opts))
    assert_solutions_agree(f, opts, g, o, min_converged=2)
    assert_selection_agrees(f, opts, g, o)
    # the confidence changes the objective (it is not ignored)
    base = O.evaluate(f.replace(qry_conf=None), to_oracle_opts(opts), 0, g.T_cw[g.best])
    assert g.cost[g.best] != pytest.approx(base[27], rel=1e-3)


def test_confidence_forms_agree_bitwise(torch):
    frames = [conf_frame(630 + i, n_hyps=3, crop_side=s) for i, s in enumerate((40, 55))]
    opts = B.Options(iters=(3, 3, 3, 0))
    solver = B.Solver(opts)
    fas = args_for(frames)
    plain = [solver.solve(fa) for fa in fas]
    host = B.FrameArgs(frames[0], B.host_arrays(frames[0]), is_device=False)
    assert_same(solver.solve(host), plain[0], what="host-staged frame")
    batch = solver.solve_batch(fas)
    for i in range(2):
        assert_same(batch[i], plain[i], what=f"batched frame {i}")
    server = B.Server(opts, 1 << 30, max_slots=4)
    res, _ = server.wait(server.submit(fas[1]))
    assert_same(res, plain[1], what="served frame")
    server.close()


def test_batch_and_server_reject_mixed_confidence_presence(torch):
    """The batched and served forms run one kernel variant per launch, so every frame gives
    a confidence map on every level or none; the plain form takes any mix."""
    with_conf = conf_frame(640, n_hyps=2, crop_side=40)
    without = S.make_frame(S.config_reduced_frame(n_hyps=2, crop_side=40), S.frame_seed(2, 641))
    solver = B.Solver(B.Options(iters=(2, 2, 2, 0)))
    fas = args_for([with_conf, without])
    with pytest.raises(B.PilotError, match="confidence presence"):
        solver.solve_batch(fas)
    one_level = with_conf.replace(qry_conf=[with_conf.qry_conf[0]] + [None] * (len(with_conf.qry_conf) - 1))
    fa = args_for([one_level])[0]
    with pytest.raises(B.PilotError, match="confidence map on every level"):
        solver.solve_batch([fa])
    assert solver.solve(fa).best >= 0            # the plain form dispatches per level
    server = B.Server(B.Options(iters=(2, 2, 2, 0)), 1 << 28, max_slots=2)
    server.submit(fas[0])
    with pytest.raises(B.PilotError, match="confidence presence"):
        server.submit(fas[1])
    server.close()
