"""Pins of the sensor-prior residual gates in the oracle (Supp. "Sensor-Prior Fusion in LM":
an excessively large prior residual is down-weighted so that it cannot corrupt the visual
registration; the gate reading is a truncated Huber):

* a gate of 0, or one above the residual, leaves the prior's terms exactly as without it;
* above the gate the prior adds nothing to H and g, and a central finite difference of the
  whole objective along each pose direction equals the visual and the other prior's
  gradient alone (the gated prior exerts no pull);
* the cost is continuous at the gate: a gate just below the residual gives the ungated
  cost to first order, and the gated cost is the textbook Huber at the gate, times the
  prior's weight.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_31098_gb300 import scenes as S


@pytest.fixture(scope="module")
def frame():
    f = S.make_frame(S.config_reduced_frame(crop_side=40, n_hyps=1), S.frame_seed(2, 900))
    # a tilted IMU reading (0.05 residual) and a range 3 m long: both priors have sizeable residuals
    g = f.gravity_cam + np.array([0.05, 0.0, 0.0])
    return f.replace(gravity_cam=g / np.linalg.norm(g), range_m=f.range_m + 3.0)


def huber(s, d):
    return s if s <= d * d else 2.0 * d * np.sqrt(s) - d * d


def residual_norm(f, which, T):
    if which == "gravity":
        return float(np.linalg.norm(O.gravity_residual(f, T)[0]))
    ok, r, _ = O.range_residual(f, T)
    assert ok
    return abs(r)


@pytest.mark.parametrize("which", ["gravity", "range"])
def test_open_gate_changes_nothing(frame, which):
    T = frame.T_gt
    r = residual_norm(frame, which, T)
    base = O.prior_terms(frame, O.SolverOptions(), which, T)
    for gate in (0.0, 1.5 * r):
        kw = {"gate_grav": gate} if which == "gravity" else {"gate_range": gate}
        got = O.prior_terms(frame, O.SolverOptions(**kw), which, T)
        np.testing.assert_array_equal(got[0], base[0])
        np.testing.assert_array_equal(got[1], base[1])
        assert got[2] == base[2]


@pytest.mark.parametrize("which", ["gravity", "range"])
def test_closed_gate_is_a_constant(frame, which):
    T = frame.T_gt
    r = residual_norm(frame, which, T)
    gate = 0.5 * r
    opts = O.SolverOptions(**({"gate_grav": gate} if which == "gravity" else {"gate_range": gate}))
    H, g, cost = O.prior_terms(frame, opts, which, T)
    assert not H.any() and not g.any()
    w, d = (frame.w_grav, opts.huber_grav) if which == "gravity" else (frame.w_range, opts.huber_range)
    assert cost == pytest.approx(w * huber(gate * gate, d), rel=1e-12)
    # continuity: a gate a hair below the residual costs what the ungated prior does
    near = O.SolverOptions(**({"gate_grav": r * (1 - 1e-9)} if which == "gravity" else {"gate_range": r * (1 - 1e-9)}))
    assert O.prior_terms(frame, near, which, T)[2] == pytest.approx(O.prior_terms(frame, O.SolverOptions(), which, T)[2],
                                                                    rel=1e-7)


def test_gated_prior_exerts_no_pull_on_the_objective(frame):
    """Finite differences of the whole objective (Eq. 7) with the range prior gated equal
    those of the objective without the range prior."""
    T = frame.T_gt
    r = residual_norm(frame, "range", T)
    gated = O.SolverOptions(gate_range=0.5 * r)
    no_range = frame.replace(use_range=False)
    h = 1e-6
    for k in range(6):
        xi = np.zeros(6)
        xi[k] = h
        Tp, Tm = O.pose_update(xi, T), O.pose_update(-xi, T)
        d_gated = (O.evaluate(frame, gated, 0, Tp)[27] - O.evaluate(frame, gated, 0, Tm)[27]) / (2 * h)
        d_none = (O.evaluate(no_range, gated, 0, Tp)[27] - O.evaluate(no_range, gated, 0, Tm)[27]) / (2 * h)
        assert d_gated == pytest.approx(d_none, rel=1e-6, abs=1e-6)
