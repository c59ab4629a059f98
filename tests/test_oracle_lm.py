"""Pins of the oracle's whole LM solve (Eq. 7-9, Sec. IV-E) against closed forms,
brute force and invariants.

* Noiseless scene: the ground truth is a fixed point (cost and gradient vanish up to
  FP32 storage of the descriptors) and LM recovers it from a small perturbation.
* Tiny scene: a brute-force grid around the LM result finds nothing lower, in 6-DoF
  locally and over the (x, y, psi) hypothesis space globally.
* Gravity only (Eq. 3): LM converges to the minimal rotation that maps R gamma^W onto
  the measurement, leaving the camera centre untouched.
* Range only (Eq. 4-6): a nadir camera over a flat DSM settles at height h0 + d.
* Top-K (Supp. "Multi-Hypothesis Refinement") keeps exactly the K lowest costs.
* Hypotheses are independent: any subset or permutation solves to the same poses.
"""
import dataclasses

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import oracle as O
from paper_2606_31098_gb300 import scenes as S


def noiseless_cfg(**kw):
    base = dict(ref_noise=0.0, gravity_noise_deg=0.0, range_noise=0.0, hyp_xy=0.5, hyp_yaw_deg=0.5)
    base.update(kw)
    return dataclasses.replace(S.config_reduced_frame(crop_side=40, n_hyps=4), **base)


def test_ground_truth_is_a_fixed_point_of_the_noiseless_scene():
    f = S.make_frame(noiseless_cfg(), 7)
    opts = O.SolverOptions()
    for level in range(f.L):
        E = O.evaluate(f, opts, level, f.T_gt)
        H = O.unpack_H(E[:21])
        assert E[27] < 1e-10                      # FP32 storage of descriptors only
        # gradient is zero relative to the curvature: |g_a| << sqrt(H_aa)
        assert np.all(np.abs(E[21:27]) < 1e-7 * np.sqrt(np.diag(H)) * np.sqrt(E[28]))


def test_lm_recovers_ground_truth_from_small_perturbations():
    f = S.make_frame(noiseless_cfg(), 7)
    r = O.solve(f, O.SolverOptions())
    assert np.all(r.status == O.HYP_OK)
    for m in range(f.M):
        assert S.translation_error_m(r.T_cw[m], f.T_gt) < 1e-6
        assert S.rotation_error_deg(r.T_cw[m], f.T_gt) < 1e-5
        np.testing.assert_allclose(r.T_cw[m], f.T_gt, atol=1e-7)


def tiny_frame(seed=5):
    """8x8 anchors, C = 4, one 32x32 level (the brute-force workload)."""
    cfg = S.SceneConfig(crop_side=8, gsd=4.0, hill_sigma=8.0, n_boxes=1, box_side=(6.0, 10.0),
                        channels=4, levels=((32, 32),), f0=40.0, blob_sigma=(3.0, 6.0),
                        altitude=(120.0, 120.0), pitch_deg=(50.0, 50.0), n_hyps=1,
                        hyp_mode="rot_trans", hyp_rot_deg=1.0, hyp_trans=1.0,
                        use_gravity=False, use_range=False)
    return S.make_frame(cfg, seed)


def xy_yaw_pose(T_ref, dx, dy, dyaw):
    R = np.asarray(T_ref).reshape(3, 4)[:, :3]
    C = S.camera_centre(T_ref)
    Rz = Rotation.from_rotvec([0, 0, dyaw]).as_matrix()
    return S.compose_pose((Rz @ R.T).T, C + np.array([dx, dy, 0.0]))


def test_lm_optimum_is_a_brute_force_minimum_on_a_tiny_grid():
    f = tiny_frame()
    opts = O.SolverOptions(iters=(40, 0, 0, 0), huber_photo=10.0)
    r = O.solve(f, opts)
    assert r.status[0] == O.HYP_OK
    T_star = r.T_cw[0]
    c_star = r.cost[0]
    # (1) local 6-DoF brute force: every neighbour on a +-1 step grid is not lower
    steps = np.array([1e-3] * 3 + [np.deg2rad(1e-3)] * 3)
    grid = np.stack(np.meshgrid(*[[-1, 0, 1]] * 6, indexing="ij"), -1).reshape(-1, 6)
    Ts = [O.pose_update(g * steps, T_star) for g in grid]
    costs = O.evaluate_many(f, opts, 0, Ts)[:, 27]
    assert costs.min() >= c_star - 1e-9 * max(1.0, c_star)
    # (2) (x, y, psi) brute force through the LM optimum (the other three degrees of
    # freedom held at their optimal values), +-1 m / +-1 deg in 0.1 steps: the grid
    # minimum is the centre cell and nothing on the grid is lower than the LM cost
    vals = np.arange(-10, 11) * 0.1
    Tg = [xy_yaw_pose(T_star, dx, dy, np.deg2rad(dp)) for dx in vals for dy in vals for dp in vals]
    cg = O.evaluate_many(f, opts, 0, Tg)[:, 27]
    best = int(np.argmin(cg))
    assert cg[best] >= c_star - 1e-9 * max(1.0, c_star)
    ix, iy, ip = np.unravel_index(best, (21, 21, 21))
    assert (ix, iy, ip) == (10, 10, 10)
    # and the optimum is at least as good as the ground truth of this noisy scene
    assert c_star <= O.evaluate(f, opts, 0, f.T_gt)[27]


def only_priors(f, gravity, rng_prior):
    return f.replace(point_valid=np.zeros(f.N, np.uint8), use_gravity=gravity, use_range=rng_prior)


def test_gravity_only_solve_is_the_minimal_rotation():
    f0 = S.make_frame(S.config_reduced_frame(crop_side=20, n_hyps=5), 21)
    f = only_priors(f0, True, False)
    opts = O.SolverOptions(iters=(30, 0, 0, 0), huber_grav=10.0, min_valid_frac=0.0)
    r = O.solve(f, opts)
    for m in range(f.M):
        T0 = f.T_hyps[m]
        R0 = T0.reshape(3, 4)[:, :3]
        a0 = R0 @ f.gravity_world
        gm = f.gravity_cam / np.linalg.norm(f.gravity_cam)
        axis = np.cross(a0, gm)
        ang = np.arctan2(np.linalg.norm(axis), a0 @ gm)
        R_expected = Rotation.from_rotvec(axis / np.linalg.norm(axis) * ang).as_matrix() @ R0
        R_got = r.T_cw[m].reshape(3, 4)[:, :3]
        np.testing.assert_allclose(R_got, R_expected, atol=1e-9)
        np.testing.assert_allclose(S.camera_centre(r.T_cw[m]), S.camera_centre(T0), atol=1e-9)


def test_range_only_nadir_over_flat_ground_settles_at_h0_plus_d():
    f0 = S.make_frame(S.config_reduced_frame(crop_side=40, n_hyps=1), 22)
    h0, d = 12.5, 140.0
    Tn = S.look_pose(np.array([3.0, -2.0, 150.0]), 0.3, np.pi / 2)
    f = only_priors(f0, False, True).replace(dsm=np.full_like(f0.dsm, h0), range_m=d,
                                             T_hyps=Tn[None, :].copy())
    opts = O.SolverOptions(iters=(20, 0, 0, 0), min_valid_frac=0.0)
    r = O.solve(f, opts)
    C = S.camera_centre(r.T_cw[0])
    assert C[2] == pytest.approx(h0 + d, abs=1e-9)
    assert C[0] == pytest.approx(3.0, abs=1e-9) and C[1] == pytest.approx(-2.0, abs=1e-9)
    np.testing.assert_allclose(r.T_cw[0].reshape(3, 4)[:, :3], Tn.reshape(3, 4)[:, :3], atol=1e-12)


def test_top_k_keeps_the_k_lowest_coarse_costs():
    f = S.make_frame(S.config_reduced_frame(crop_side=24, n_hyps=9), 31)
    base = O.SolverOptions(iters=(2, 2, 3, 0))
    K = 4
    coarse = [O.lm_level(f, base, 2, f.T_hyps[m]) for m in range(f.M)]
    costs = np.array([c[1][27] for c in coarse])
    keep = set(np.argsort(costs, kind="stable")[:K].tolist())
    r = O.solve(f, dataclasses.replace(base, keep_top_k=(0, 0, K, 0)))
    pruned = set(np.flatnonzero(r.status == O.HYP_PRUNED).tolist())
    assert pruned == set(range(f.M)) - keep
    assert r.hyp_iters == f.M * 3 + K * (2 + 2)
    for m in pruned:
        np.testing.assert_array_equal(r.T_cw[m], coarse[m][0])
        assert r.cost[m] == costs[m]
    assert r.best in keep


def test_hypotheses_are_independent_and_permutation_invariant():
    f = S.make_frame(S.config_reduced_frame(crop_side=24, n_hyps=6), 41)
    opts = O.SolverOptions(iters=(3, 3, 3, 0))
    full = O.solve(f, opts)
    perm = np.array([4, 1, 5, 0, 3, 2])
    sub = O.solve(f, opts, T_hyps=f.T_hyps[perm])
    np.testing.assert_array_equal(sub.T_cw, full.T_cw[perm])
    np.testing.assert_array_equal(sub.cost, full.cost[perm])
    one = O.solve(f, opts, T_hyps=f.T_hyps[3:4], n_threads=1)
    np.testing.assert_array_equal(one.T_cw[0], full.T_cw[3])
    assert full.hyp_iters == 6 * 9


def test_status_codes():
    f = S.make_frame(S.config_reduced_frame(crop_side=20, n_hyps=2), 51)
    opts = O.SolverOptions(iters=(2, 2, 2, 0))
    # every anchor invisible at the hypotheses (moved 10 km away): too few valid anchors
    T = f.T_hyps.copy()
    T[:, 3] += 1e4
    r = O.solve(f, opts, T_hyps=T)
    assert np.all(r.status == O.HYP_FEW_VALID) and r.best == -1
    # NaN in the query map reaches the cost: non-finite
    q = [m.copy() for m in f.qry_feat]
    for m in q:
        m[:] = np.nan
    r = O.solve(f, opts, qry_feat=q)
    assert np.all(r.status == O.HYP_NONFINITE) and r.best == -1
    # diag(H) damping with no information at all: the damped system is singular
    empty = only_priors(f, False, False)
    r = O.solve(empty, dataclasses.replace(opts, damping_mode=1, min_valid_frac=0.0))
    assert np.all(r.status == O.HYP_NOT_PD)
    np.testing.assert_array_equal(r.T_cw, f.T_hyps)
    # zero hypotheses
    r = O.solve(f, opts, T_hyps=np.zeros((0, 12)))
    assert r.best == -1 and r.hyp_iters == 0


def test_accepted_cost_never_increases():
    """A step is kept only if it lowers the objective: the cost after k iterations is a
    non-increasing sequence in k, at every level."""
    f = S.make_frame(S.config_reduced_frame(crop_side=30, n_hyps=3), 61)
    for m in range(f.M):
        for level in (2, 0):
            costs = [O.lm_level(f, O.SolverOptions(iters=(k, k, k, 0)), level, f.T_hyps[m])[1][27]
                     for k in range(0, 12)]
            assert all(b <= a for a, b in zip(costs, costs[1:])), costs
            assert costs[-1] < costs[0]


def test_range_residual_vanishes_where_the_centre_pixel_meets_flat_ground():
    """Eq. 4-6 with c away from the image centre, pinned by forward projection: find the
    point X on the plane z = h0 whose projection K [R | t] X is the level-0 image centre
    (two linear equations), set the measured range to |X - C|; the oracle's range
    residual must then vanish.  A laser ray through the wrong pixel does not."""
    f0 = S.make_frame(S.config_reduced_frame(crop_side=40, n_hyps=1), 23)
    h0 = 4.0
    H0, W0 = f0.qry_feat[0].shape[:2]
    rng = np.random.default_rng(5)
    for _ in range(10):
        T = S.look_pose(np.array([*rng.uniform(-20, 20, 2), rng.uniform(100, 200)]),
                        rng.uniform(0, 2 * np.pi), np.deg2rad(rng.uniform(40, 80)))
        cx, cy = f0.cx + rng.uniform(-40, 40), f0.cy + rng.uniform(-30, 30)
        P = np.array([[f0.fx, 0, cx], [0, f0.fy, cy], [0, 0, 1.0]]) @ T.reshape(3, 4)
        u, v = W0 / 2, H0 / 2
        # rows (P0 - u P2) X = 0 and (P1 - v P2) X = 0 with X = (x, y, h0, 1)
        A = np.array([P[0] - u * P[2], P[1] - v * P[2]])
        xy = np.linalg.solve(A[:, :2], -(A[:, 2] * h0 + A[:, 3]))
        X = np.array([xy[0], xy[1], h0])
        d = np.linalg.norm(X - S.camera_centre(T))
        f = f0.replace(dsm=np.full((200, 200), h0, np.float32), dsm_x0=-1000.0, dsm_y0=-1000.0,
                       dsm_gsd=10.0, range_m=d, cx=cx, cy=cy)
        ok, r, _ = O.range_residual(f, T)
        assert ok and abs(r) < 1e-9
        ok, r, _ = O.range_residual(f.replace(range_m=d + 1.0), T)
        assert ok and abs(r) > 0.1
