"""Finite-difference pins of the oracle's residual Jacobians and normal equations.

The oracle forms each anchor's dense C x 6 Jacobian from the chain rule
(feature gradient x projection Jacobian x se(3) generators, Eq. 1 and Eq. 8) and the
prior Jacobians analytically (Eq. 3, Eq. 6).  Here they are compared with central
differences of the residuals under the left perturbation T <- exp(h e_k) T (Eq. 9),
and the accumulated gradient with the finite-difference gradient of the total cost
(Eq. 7): d cost / d delta = 2 g because the IRLS weight of rho(w s) is w rho'(w s).
A dropped term, a sign error or a transposed operand anywhere in the chain fails here.
"""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_31098_gb300 import scenes as S


@pytest.fixture(scope="module")
def small_frame():
    cfg = dataclasses.replace(S.config_reduced_frame(crop_side=24, n_hyps=2), box_height=(5.0, 20.0))
    return S.make_frame(cfg, 11)


def perturbed(T, k, h):
    xi = np.zeros(6)
    xi[k] = h
    return O.pose_update(xi, T)


def random_poses(frame, n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        xi = np.concatenate([rng.uniform(-2, 2, 3), np.deg2rad(rng.uniform(-1.5, 1.5, 3))])
        out.append(O.pose_update(xi, frame.T_gt))
    return out


def test_photo_jacobian_matches_central_differences(small_frame):
    f = small_frame
    checked = 0
    for level in range(f.L):
        for T in random_poses(f, 3, 100 + level):
            margins = O.point_margins(f, level, T)
            idx = np.flatnonzero(margins > 0.02)[::7]
            for j in idx:
                vis, r, J = O.point_residual(f, level, T, j)
                if not vis:
                    continue
                h = 1e-6
                Jfd = np.empty_like(J)
                for k in range(6):
                    vp, rp, _ = O.point_residual(f, level, perturbed(T, k, h), j, with_jacobian=False)
                    vm, rm, _ = O.point_residual(f, level, perturbed(T, k, -h), j, with_jacobian=False)
                    assert vp and vm
                    Jfd[:, k] = (rp - rm) / (2 * h)
                scale = np.abs(J).max()
                np.testing.assert_allclose(J, Jfd, atol=1e-6 * scale, rtol=0)
                checked += 1
    assert checked > 100


def test_gravity_jacobian_matches_central_differences(small_frame):
    f = small_frame
    for T in random_poses(f, 20, 7):
        r, J = O.gravity_residual(f, T)
        h = 1e-6
        Jfd = np.stack([(O.gravity_residual(f, perturbed(T, k, h))[0] -
                         O.gravity_residual(f, perturbed(T, k, -h))[0]) / (2 * h) for k in range(6)], 1)
        np.testing.assert_allclose(J, Jfd, atol=1e-9)
        assert np.all(J[:, :3] == 0.0)


def test_range_jacobian_matches_central_differences(small_frame):
    f = small_frame
    checked = 0
    for T in random_poses(f, 40, 8):
        ok, r, J = O.range_residual(f, T)
        if not ok:
            continue
        h = 1e-7
        okp = [O.range_residual(f, perturbed(T, k, h)) for k in range(6)]
        okm = [O.range_residual(f, perturbed(T, k, -h)) for k in range(6)]
        Jfd = np.array([(okp[k][1] - okm[k][1]) / (2 * h) for k in range(6)])
        # one-sided differences that disagree mean the range point sits on a DSM cell edge
        fwd = np.array([(okp[k][1] - r) / h for k in range(6)])
        bwd = np.array([(r - okm[k][1]) / h for k in range(6)])
        if np.abs(fwd - bwd).max() > 1e-3 * (1 + np.abs(J).max()):
            continue
        np.testing.assert_allclose(J, Jfd, atol=1e-5 * (1 + np.abs(J).max()))
        checked += 1
    assert checked >= 20


def test_range_jacobian_on_tilted_plane_has_closed_form():
    """On a planar DSM z = a x + b y + c the residual is affine in the range point, so
    d r / d P = (-a, -b, 1) exactly; check J against that row times dP/ddelta built from
    the finite differences of the range point itself (via the residual on a flat DSM)."""
    cfg = dataclasses.replace(S.config_reduced_frame(crop_side=40, n_hyps=1), n_hills=0, n_boxes=0)
    f = S.make_frame(cfg, 3)
    a, b, c0 = 0.05, -0.03, 2.0
    S_ = f.dsm.shape[0]
    xs = f.dsm_x0 + (np.arange(S_) + 0.5) * f.dsm_gsd
    ys = f.dsm_y0 + (np.arange(S_) + 0.5) * f.dsm_gsd
    X, Y = np.meshgrid(xs, ys)
    plane = f.replace(dsm=(a * X + b * Y + c0).astype(np.float64).astype(np.float32))
    flat = f.replace(dsm=np.zeros_like(f.dsm))
    for T in random_poses(f, 10, 9):
        ok, r, J = O.range_residual(plane, T)
        assert ok
        okf, zr, _ = O.range_residual(flat, T)            # residual on z = 0 is the height of P
        assert okf
        h = 1e-6
        # x and y of the range point follow from the plane/flat residual difference:
        # r_plane - r_flat = -(a x + b y + c0)
        dP = []
        for k in range(6):
            vals = []
            for sgn in (1, -1):
                Tk = perturbed(T, k, sgn * h)
                vals.append((O.range_residual(plane, Tk)[1], O.range_residual(flat, Tk)[1]))
            dP.append(((vals[0][0] - vals[1][0]) / (2 * h), (vals[0][1] - vals[1][1]) / (2 * h)))
        J_plane_fd = np.array([d[0] for d in dP])
        np.testing.assert_allclose(J, J_plane_fd, atol=1e-5)


def test_gradient_is_half_the_cost_derivative(small_frame):
    """2 g == d cost / d delta (Eq. 7), with anchors near a cell edge set aside."""
    f = small_frame
    opts = O.SolverOptions()
    for level in range(f.L):
        T = random_poses(f, 1, 50 + level)[0]
        margins = O.point_margins(f, level, T)
        valid = (f.point_valid.astype(bool) & (margins > 1e-3)).astype(np.uint8)
        fm = f.replace(point_valid=valid)
        E = O.evaluate(fm, opts, level, T)
        h = 1e-7
        fd = np.array([(O.evaluate(fm, opts, level, perturbed(T, k, h))[27] -
                        O.evaluate(fm, opts, level, perturbed(T, k, -h))[27]) / (2 * h) for k in range(6)])
        np.testing.assert_allclose(2 * E[21:27], fd, rtol=2e-5, atol=1e-6 * np.abs(fd).max())


def test_hessian_equals_weighted_sum_of_fd_jacobians(small_frame):
    """H = sum_j w_j J_j^T J_j (Eq. 8) with J_j from finite differences and the Huber
    IRLS weight restated from its closed form, on a subset of anchors."""
    f = small_frame
    opts = O.SolverOptions()
    level = 1
    T = random_poses(f, 1, 77)[0]
    margins = O.point_margins(f, level, T)
    keep = np.flatnonzero(f.point_valid.astype(bool) & (margins > 0.02))[::5]
    valid = np.zeros(f.N, np.uint8)
    valid[keep] = 1
    fm = f.replace(point_valid=valid)
    H21, g, cost, n = O.photo_terms(fm, opts, level, T)
    Hfd = np.zeros((6, 6))
    gfd = np.zeros(6)
    cost_ref = 0.0
    h = 1e-6
    for j in keep:
        vis, r, _ = O.point_residual(fm, level, T, j, with_jacobian=False)
        if not vis:
            continue
        J = np.stack([(O.point_residual(fm, level, perturbed(T, k, h), j, False)[1] -
                       O.point_residual(fm, level, perturbed(T, k, -h), j, False)[1]) / (2 * h)
                      for k in range(6)], 1)
        s = float(r @ r)
        d = opts.huber_photo
        w = 1.0 if s <= d * d else d / np.sqrt(s)
        cost_ref += s if s <= d * d else 2 * d * np.sqrt(s) - d * d
        Hfd += w * J.T @ J
        gfd += w * J.T @ r
    np.testing.assert_allclose(O.unpack_H(H21), Hfd, rtol=1e-6, atol=1e-7 * np.abs(Hfd).max())
    np.testing.assert_allclose(g, gfd, atol=1e-6 * np.abs(gfd).max() + 1e-12)
    assert cost == pytest.approx(cost_ref, rel=1e-12)
    assert n == len(keep)


def test_visibility_rules(small_frame):
    """Points behind the camera, outside the map or flagged invalid contribute nothing."""
    f = small_frame
    T = f.T_gt.copy().reshape(3, 4)
    T_behind = T.copy()
    T_behind[:, :3] = -T_behind[:, :3]          # looks the other way: every Z < 0
    T_behind[:, 3] = -T_behind[:, 3]
    H, g, cost, n = O.photo_terms(f, O.SolverOptions(), 0, T_behind.ravel())
    assert n == 0 and cost == 0.0 and not np.any(H) and not np.any(g)
    none_valid = f.replace(point_valid=np.zeros(f.N, np.uint8))
    assert O.photo_terms(none_valid, O.SolverOptions(), 0, f.T_gt)[3] == 0
    far = T.copy()
    far[0, 3] += 1e4                              # shifted far sideways: all off the map
    assert O.photo_terms(f, O.SolverOptions(), 0, far.ravel())[3] == 0


def test_gradient_and_hessian_with_non_uniform_anchor_weights(small_frame):
    """The anchor weight w_l(j) sits inside the robust loss, rho(w ||r||^2) (Eq. 2), so
    the cost derivative is 2 sum_j w_j rho'(w_j s_j) J^T r; check with random weights and a
    small Huber threshold so that both Huber branches are active."""
    f = small_frame
    rng = np.random.default_rng(99)
    level = 1
    T = random_poses(f, 1, 123)[0]
    margins = O.point_margins(f, level, T)
    valid = (f.point_valid.astype(bool) & (margins > 1e-3)).astype(np.uint8)
    fm = f.replace(point_valid=valid, point_weight=rng.uniform(0.2, 3.0, f.N).astype(np.float32))
    # Huber threshold at the median of w ||r||^2, so that both branches are exercised
    ws = []
    for j in np.flatnonzero(valid):
        vis, r, _ = O.point_residual(fm, level, T, j, with_jacobian=False)
        if vis:
            ws.append(fm.point_weight[j] * float(r @ r))
    opts = O.SolverOptions(huber_photo=float(np.sqrt(np.median(ws))))
    E = O.evaluate(fm, opts, level, T)
    h = 1e-7
    fd = np.array([(O.evaluate(fm, opts, level, perturbed(T, k, h))[27] -
                    O.evaluate(fm, opts, level, perturbed(T, k, -h))[27]) / (2 * h) for k in range(6)])
    np.testing.assert_allclose(2 * E[21:27], fd, rtol=2e-5, atol=1e-6 * np.abs(fd).max())
    # Hessian: sum_j w_j rho'(w_j s_j) J_j^T J_j with FD Jacobians on a subset
    keep = np.flatnonzero(valid)[::9]
    sub = np.zeros(f.N, np.uint8)
    sub[keep] = 1
    fs = fm.replace(point_valid=sub)
    H21, _, _, _ = O.photo_terms(fs, opts, level, T)
    Hfd = np.zeros((6, 6))
    d = opts.huber_photo
    n_clipped = 0
    for j in keep:
        vis, r, _ = O.point_residual(fs, level, T, j, with_jacobian=False)
        if not vis:
            continue
        J = np.stack([(O.point_residual(fs, level, perturbed(T, k, 1e-6), j, False)[1] -
                       O.point_residual(fs, level, perturbed(T, k, -1e-6), j, False)[1]) / 2e-6
                      for k in range(6)], 1)
        w = float(fs.point_weight[j])
        s = w * float(r @ r)
        n_clipped += s > d * d
        Hfd += w * (1.0 if s <= d * d else d / np.sqrt(s)) * J.T @ J
    assert 0 < n_clipped < len(keep)
    np.testing.assert_allclose(O.unpack_H(H21), Hfd, rtol=1e-6, atol=1e-7 * np.abs(Hfd).max())
