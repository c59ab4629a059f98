"""Pins of the sequential-tracking oracle (oracle/tracking.py) against closed forms:

* on a screw motion T_k = A^k T_0 (A built from an axis-angle rotation and a translation,
  independently of the oracle), the constant-velocity prediction from T_k and T_{k-1} is
  exactly T_{k+s} for every s, and without a second pose the last one is held;
* every seed of the (x, y, psi) grid has the same roll and pitch as the prior, its camera
  centre moved by (x, y, 0) and its heading by psi (read back with an independent formula);
* a world point projects identically through T with world coordinates and through
  to_local(T, o) with crop offsets, and to_world inverts to_local;
* the loop: a localiser returning ground truth on a screw trajectory gives priors equal to
  ground truth from frame 2 on (serial) and crop poses equal to ground truth from frame 3
  on (lookahead); planted failures count one recovery each and restart the next frame
  from its ground truth, in both modes.
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import tracking as TR


def rigid(rotvec, t):
    M = np.eye(4)
    M[:3, :3] = Rotation.from_rotvec(rotvec).as_matrix()
    M[:3, 3] = t
    return M


def screw_sequence(n, seed=0):
    rng = np.random.default_rng(seed)
    A = rigid(rng.normal(0, 0.03, 3), rng.normal(0, 2.0, 3))
    T0 = rigid(rng.normal(0, 1.0, 3), rng.normal(0, 50.0, 3))
    out, M = [], T0
    for _ in range(n):
        out.append(M[:3, :].ravel().copy())
        M = A @ M
    return np.array(out)


@pytest.mark.parametrize("steps", [0, 1, 2, 5])
def test_prediction_is_exact_on_a_screw_motion(steps):
    seq = screw_sequence(12, seed=steps)
    for k in range(1, 12 - steps):
        np.testing.assert_allclose(TR.predict(seq[k], seq[k - 1], steps), seq[k + steps], atol=1e-9)


def test_prediction_without_history_holds_the_pose():
    seq = screw_sequence(2, seed=9)
    np.testing.assert_array_equal(TR.predict(seq[1], None, 3), seq[1])
    with pytest.raises(ValueError):
        TR.predict(seq[1], seq[0], -1)


def heading_offset(T_prior, T):
    """(dx, dy, dpsi deg, change of the optical axis' elevation): rotations compared through
    the optical axis in the world (third row of R_cw), centres through -R^T t."""
    Rp, Rn = T_prior.reshape(3, 4)[:, :3], T.reshape(3, 4)[:, :3]
    Cp = -Rp.T @ T_prior.reshape(3, 4)[:, 3]
    Cn = -Rn.T @ T.reshape(3, 4)[:, 3]
    ap, an = Rp[2], Rn[2]                         # optical axes in world coordinates
    dpsi = np.rad2deg(np.arctan2(an[1], an[0]) - np.arctan2(ap[1], ap[0]))
    dpsi = (dpsi + 180.0) % 360.0 - 180.0
    return Cn[0] - Cp[0], Cn[1] - Cp[1], Cn[2] - Cp[2], dpsi, an[2] - ap[2]


def test_seed_grid_moves_the_centre_and_turns_the_heading():
    seq = screw_sequence(1, seed=4)
    T = seq[0]
    xy, yaw = (-4.0, 0.0, 6.0), (-9.0, 1.0, 7.0)
    H = TR.seed_grid(T, xy, yaw)
    assert H.shape == (27, 12)
    m = 0
    for gx in xy:
        for gy in xy:
            for gp in yaw:
                dx, dy, dz, dpsi, dtilt = heading_offset(T, H[m])
                np.testing.assert_allclose([dx, dy, dz, dpsi, dtilt], [gx, gy, 0.0, gp, 0.0], atol=1e-9)
                R = H[m].reshape(3, 4)[:, :3]
                np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-12)
                # the world-frame turn from the prior's camera to the seed's is about +z by psi
                turn = Rotation.from_matrix(R.T @ T.reshape(3, 4)[:, :3]).as_rotvec()
                np.testing.assert_allclose(turn, [0.0, 0.0, np.deg2rad(gp)], atol=1e-9)
                m += 1


def test_local_frame_projects_like_the_world_frame():
    T = screw_sequence(1, seed=5)[0]
    o = (123.5, -77.25)
    P = np.array([130.0, -70.0, 12.0])
    Tl = TR.to_local(T, o)
    pw = T.reshape(3, 4) @ np.append(P, 1.0)
    pl = Tl.reshape(3, 4) @ np.append(P - np.array([o[0], o[1], 0.0]), 1.0)
    np.testing.assert_allclose(pl, pw, atol=1e-9)
    np.testing.assert_allclose(TR.to_world(Tl, o), T, atol=1e-12)


def test_pose_error_reads_a_known_offset():
    T = screw_sequence(1, seed=6)[0]
    U = TR.seed_grid(T, (3.0,), (4.0,))[0]
    e_t, e_R = TR.pose_error(U, T)
    assert e_t == pytest.approx(np.hypot(3.0, 3.0), abs=1e-9)
    assert e_R == pytest.approx(4.0, abs=1e-9)


@pytest.mark.parametrize("mode", ["serial", "lookahead"])
def test_perfect_localiser_on_a_screw_trajectory(mode):
    gt = screw_sequence(10, seed=7)
    seen = []

    def localise(t, prior, crop):
        seen.append((t, prior, crop))
        return gt[t], None

    log = TR.track(gt, localise, mode=mode)
    assert log.frc == 0 and not log.failed.any()
    np.testing.assert_allclose(log.priors[0], gt[0])
    np.testing.assert_allclose(log.priors[1], gt[0])            # one estimate: held
    for t in range(2, 10):
        np.testing.assert_allclose(log.priors[t], gt[t], atol=1e-9)
    first_exact = 2 if mode == "serial" else 3
    for t in range(first_exact, 10):
        np.testing.assert_allclose(log.crop_priors[t], gt[t], atol=1e-9)
    if mode == "lookahead":
        np.testing.assert_allclose(log.crop_priors[1], gt[0])
        np.testing.assert_allclose(log.crop_priors[2], gt[0])   # est[0] held two frames


@pytest.mark.parametrize("mode", ["serial", "lookahead"])
def test_failures_are_counted_and_the_next_frame_restarts_from_ground_truth(mode):
    gt = screw_sequence(12, seed=8)
    bad = {3: (25.0, 0.0), 7: (0.0, 30.0), 8: (21.0, 0.0)}

    def localise(t, prior, crop):
        if t in bad:
            dxy, dpsi = bad[t]
            return TR.seed_grid(gt[t], (dxy,), (dpsi,))[0], None
        return gt[t], None

    log = TR.track(gt, localise, mode=mode)
    assert log.frc == 3
    assert list(np.flatnonzero(log.failed)) == [3, 7, 8]
    for t in (4, 8, 9):
        np.testing.assert_array_equal(log.priors[t], gt[t])
        np.testing.assert_array_equal(log.crop_priors[t], gt[t])
    # after a failure the history holds ground truth, so the following priors are exact
    for t in (5, 6, 10, 11):
        np.testing.assert_allclose(log.priors[t], gt[t], atol=1e-9)
    # 19.9 m is not a failure
    log2 = TR.track(gt, lambda t, p, c: (TR.seed_grid(gt[t], (19.9 / np.sqrt(2),), (0.0,))[0] if t == 5 else gt[t], None),
                    mode=mode)
    assert log2.frc == 0
