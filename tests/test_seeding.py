"""Host side of the seeding ablation (Supp. "Effect of Multi-hypothesis Sampling"): the four
hypothesis sets around a prior and the ring-shaped prior error used for it."""
import numpy as np
import pytest

from paper_2606_31098_gb300 import scenes as S


def xy_yaw_offset(T_prior, T):
    """(dx, dy, dyaw deg) taking the prior to T: camera centres differ by a horizontal shift,
    rotations by a rotation about world z."""
    Cp, C = S.camera_centre(T_prior), S.camera_centre(T)
    Rp, _ = S.pose_parts(T_prior)
    R, _ = S.pose_parts(T)
    Rz = R.T @ Rp                        # R_wc = Rz R_wc,prior
    assert abs(Rz[2, 2] - 1.0) < 1e-12 and abs(C[2] - Cp[2]) < 1e-9
    return C[0] - Cp[0], C[1] - Cp[1], np.rad2deg(np.arctan2(Rz[1, 0], Rz[0, 0]))


@pytest.mark.parametrize("strategy,size", [("none", 1), ("yaw", 10), ("xy", 121), ("joint", 1210)])
def test_hypothesis_sets_are_the_grid_offsets_of_the_prior(strategy, size):
    cfg = S.SceneConfig()
    T0 = S.look_pose(np.array([10.0, -20.0, 150.0]), 0.7, np.deg2rad(50.0))
    H = S.seeding_hypotheses(T0, strategy, cfg)
    assert H.shape == (size, 12)
    offs = np.array([xy_yaw_offset(T0, h.reshape(3, 4)) for h in H])
    xs = cfg.grid_xy if strategy in ("xy", "joint") else (0.0,)
    ys = cfg.grid_yaw_deg if strategy in ("yaw", "joint") else (0.0,)
    want = np.array([(x, y, p) for x in xs for y in xs for p in ys])
    np.testing.assert_allclose(offs, want, atol=1e-9)


def test_unknown_strategy_is_rejected():
    with pytest.raises(ValueError):
        S.seeding_hypotheses(np.eye(3, 4), "random")


def test_ring_prior_lies_in_the_stated_band():
    """config_seeding_ablation draws the prior 5-15 m and 5-15 deg away from the truth."""
    cfg = S.config_seeding_ablation()
    cfg.levels = ((48, 64),)             # only the prior matters here
    cfg.crop_side, cfg.n_anchors, cfg.channels = 32, 0, 4
    for i in range(6):
        f = S.make_frame(cfg, S.frame_seed(7, 100 + i))
        dx, dy, dyaw = xy_yaw_offset(f.T_gt, f.meta["T_prior"])
        assert 5.0 - 1e-9 <= np.hypot(dx, dy) <= 15.0 + 1e-9
        assert 5.0 - 1e-9 <= abs(dyaw) <= 15.0 + 1e-9
