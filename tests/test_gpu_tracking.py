"""Sequential tracking on the GPU (Supp. "Runtime Analysis"; Sec. V-A's Failure Recovery
Count) against the tracking oracle:

* the seeds written by pilot_seed_hypotheses equal the oracle's grid re-origined to the crop;
* on a short synthetic flight with one visually failed frame, the tracker (serial, and with
  the map preparation one frame ahead) and the oracle's loop (oracle crop, FP64 solve) fail
  on the same frame, count the same recoveries and agree frame by frame; the tracker's
  priors and crop poses are exactly what the oracle's rules give for its own estimates.

The paper's schedule stops after 2 / 3 / 4 iterations, so many hypotheses end millimetres
apart near one optimum and which is selected is a near-tie (as in the paper-schedule
tests); the crops also differ in the last FP32 bits.  Estimates are compared within 2 cm
and 0.02 deg, priors (which extrapolate them) within 5 cm and 0.05 deg.
"""
import numpy as np
import pytest

from oracle import crop as OC
from oracle import oracle as O
from oracle import sampler as OS
from oracle import tracking as TR
from paper_2606_31098_gb300 import binding as B
from paper_2606_31098_gb300 import scenes as S
from paper_2606_31098_gb300 import tracking as TK

from gpu_support import require_cuda

pytestmark = pytest.mark.gpu

GRID_XY = tuple(float(v) for v in range(-10, 11, 2))
GRID_YAW = (-9.0, -7.0, -5.0, -3.0, -1.0, 1.0, 3.0, 5.0, 7.0, 9.0)
# recovery thresholds of the test: the visually failed frame lands 5-15 m off, inside the
# paper's 20 m / 20 deg, so the test uses 5 m / 5 deg to exercise the recovery path
T_FAIL, R_FAIL = 5.0, 5.0
OPTS = dict(iters=(4, 3, 2, 0), keep_top_k=(0, 0, 128, 0), max_hyps=1210, max_points=500, gate_grav=0.1,
            gate_range=3.0)


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


@pytest.fixture(scope="module")
def world():
    g = S.make_global_map(side=2048, n_hills=512, n_boxes=1024, seed=3)
    tc = S.TrackConfig(n_frames=6, degrade_prob=0.0, degraded_frames=(2,), query_bank=2)
    gt = S.make_trajectory(g, tc, seed=41)
    bank = S.query_bank(tc, seed=42)
    return g, tc, gt, bank


def camera(tc):
    H0, W0 = tc.levels[0]
    return TK.Camera(tc.f0, tc.f0, W0 / 2.0, H0 / 2.0, W0, H0)


def test_seeds_match_the_oracle(torch):
    T = S.look_pose(np.array([40.0, -25.0, 130.0]), 0.9, np.deg2rad(52.0))
    origin = (61.25, -17.5)
    p = B.seed_params(T, GRID_XY, GRID_YAW, origin)
    got = B.seed_hypotheses(p).cpu().numpy()
    want = np.array([TR.to_local(h, origin) for h in TR.seed_grid(T, GRID_XY, GRID_YAW)])
    assert got.shape == (1210, 12)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-10)


def oracle_log(world, mode):
    g, tc, gt, bank = world
    om = OC.MapArgs(g.dsm, g.tdom, g.x0, g.y0, g.gsd)
    cam = camera(tc)
    oo = O.SolverOptions(iters=OPTS["iters"], keep_top_k=OPTS["keep_top_k"], gate_grav=OPTS["gate_grav"],
                         gate_range=OPTS["gate_range"])

    def localise(t, prior, crop_pose):
        p = OC.params(crop_pose, cam.fx, cam.fy, cam.cx, cam.cy, cam.img_w, cam.img_h, 0.0, tc.ray_step,
                      tc.ray_samples, tc.crop_side)
        r = OC.crop(om, p, with_rgb=False)
        assert r["ok"]
        idx = OS.sample_anchors(r["valid"], tc.n_anchors, TK.frame_anchor_seed(0, t))
        f = S.track_inputs(g, tc, bank, t, gt[t], r["points"], r["valid"], r["origin"], 77, idx)
        hyps = np.array([TR.to_local(h, r["origin"]) for h in TR.seed_grid(prior, GRID_XY, GRID_YAW)])
        o = O.solve(f.replace(T_hyps=hyps), oo)
        return TR.to_world(o.T_cw[o.best], r["origin"]), None

    return TR.track(gt, localise, mode=mode, t_fail=T_FAIL, r_fail=R_FAIL)


@pytest.mark.parametrize("mode", ["serial", "lookahead"])
def test_tracker_follows_the_oracle(torch, world, mode):
    g, tc, gt, bank = world
    tr = TK.SequentialTracker(g.dsm, None, g.x0, g.y0, g.gsd, camera(tc),
                              TK.CropSettings(tc.crop_side, 0.0, tc.ray_step, tc.ray_samples),
                              B.Options(**OPTS), GRID_XY, GRID_YAW, mode=mode)
    net = S.SyntheticNetwork(g, tc, bank, gt, 77)
    res = TK.run_sequence(tr, gt, net, t_fail=T_FAIL, r_fail=R_FAIL)
    tr.close()
    ref = oracle_log(world, mode)
    assert list(np.flatnonzero(res["failed"])) == list(np.flatnonzero(ref.failed)) == [2]
    assert res["frc"] == ref.frc == 1
    for t in range(len(gt)):
        if ref.failed[t]:
            continue
        et, er = TR.pose_error(res["estimates"][t], ref.estimates[t])
        assert et < 2e-2 and er < 2e-2, f"frame {t}: {et:.3e} m {er:.3e} deg from the oracle"
        et, er = TR.pose_error(res["priors"][t], ref.priors[t])
        assert et < 5e-2 and er < 5e-2, f"frame {t} prior: {et:.3e} m {er:.3e} deg"
        assert res["err"][t][0] < 1.0, f"frame {t}: {res['err'][t][0]:.2f} m from the ground truth"
    # the tracker's own priors and crop poses are the oracle's rules applied to its estimates
    hist = [gt[t] if res["failed"][t] else res["estimates"][t] for t in range(len(gt))]
    for t in range(len(gt)):
        if t == 0 or res["failed"][t - 1]:
            want_p = gt[t]
            want_c = gt[t]
        else:
            want_p = TR.predict(hist[t - 1], hist[t - 2] if t >= 2 else None, 1)
            want_c = want_p if mode == "serial" else TR.crop_prior_lookahead(t, hist, gt[0])
        np.testing.assert_allclose(res["priors"][t], want_p, rtol=0, atol=1e-9)
        np.testing.assert_allclose(res["crop_poses"][t], want_c, rtol=0, atol=1e-9)
    if mode == "lookahead":
        ahead = [tm.prepared_ahead for tm in res["timings"]]
        assert ahead == [False, True, True, False, True, True]   # frame 3 restarts: cropped in place
