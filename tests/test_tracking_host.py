"""Host-side pieces of sequential tracking in the library (pilot_pose_predict,
pilot_pose_reorigin; FP64 on the CPU, no GPU needed) against the tracking oracle."""
import numpy as np
import pytest

from oracle import tracking as TR
from paper_2606_31098_gb300 import binding as B
from paper_2606_31098_gb300 import tracking as TK

from test_oracle_tracking import screw_sequence


@pytest.fixture(scope="module")
def lib():
    return B.load()


@pytest.mark.parametrize("steps", [0, 1, 2, 3])
def test_prediction_matches_the_oracle(lib, steps):
    seq = screw_sequence(8, seed=20 + steps)
    rng = np.random.default_rng(steps)
    for k in range(1, 8):
        a = seq[k] + 1e-3 * rng.standard_normal(12) * (k % 2)    # not exactly rigid either
        np.testing.assert_allclose(B.pose_predict(a, seq[k - 1], steps), TR.predict(a, seq[k - 1], steps),
                                   rtol=1e-13, atol=1e-10)
        np.testing.assert_array_equal(B.pose_predict(a, None, steps), TR.predict(a, None, steps))


def test_reorigin_matches_the_oracle(lib):
    T = screw_sequence(1, seed=30)[0]
    o = (-812.25, 301.5)
    np.testing.assert_allclose(B.pose_reorigin(T, *o), TR.to_local(T, o), rtol=0, atol=1e-10)
    np.testing.assert_allclose(B.pose_reorigin(TR.to_local(T, o), -o[0], -o[1]), T, rtol=0, atol=1e-9)


def test_bad_arguments_are_rejected(lib):
    T = screw_sequence(1, seed=31)[0]
    with pytest.raises(B.PilotError, match="steps"):
        B.pose_predict(T, T, -1)
    bad = T.copy()
    bad[3] = np.nan
    with pytest.raises(B.PilotError, match="non-finite"):
        B.pose_predict(bad, T, 1)
    with pytest.raises(ValueError):
        B.seed_params(T, [], [0.0])
    with pytest.raises(ValueError):
        B.seed_params(T, [0.0] * 33, [0.0])


def test_tracker_pose_rules_match_the_oracle(lib):
    """The tracker's prior and look-ahead crop pose (host code over pilot_pose_predict) follow
    the oracle loop's rules for every frame of a history."""
    hist = list(screw_sequence(9, seed=40) + 1e-4 * np.random.default_rng(1).standard_normal((9, 12)))
    T0 = hist[0]
    for t in range(1, 9):
        np.testing.assert_allclose(TK.frame_prior(t, hist), TR.predict(hist[t - 1], hist[t - 2] if t >= 2 else None, 1),
                                   rtol=1e-13, atol=1e-10)
        np.testing.assert_allclose(TK.lookahead_crop_pose(t, hist, T0), TR.crop_prior_lookahead(t, hist, T0),
                                   rtol=1e-13, atol=1e-10)
    np.testing.assert_array_equal(TK.frame_prior(5, hist, given=T0), T0)
