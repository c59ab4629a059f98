"""Pins of the oracle's building blocks against closed forms and library routines.

SE(3) (Eq. 9), Huber (Eq. 2), bilinear sampling with analytic gradient, and the 6x6
Cholesky solve (Eq. 8) are checked against values fixed outside the oracle: textbook
rotation matrices, scipy's matrix exponential of the twist, scipy's linear
interpolation, numpy's dense solver, exact affine maps and finite differences.
"""
import os

import numpy as np
import pytest
from scipy import linalg, ndimage

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def hat(w):
    return np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])


def twist_matrix(xi):
    """4x4 se(3) matrix of xi = (nu, omega)."""
    X = np.zeros((4, 4))
    X[:3, :3] = hat(xi[3:])
    X[:3, 3] = xi[:3]
    return X


def as4(T):
    M = np.eye(4)
    M[:3, :] = np.asarray(T).reshape(3, 4)
    return M


# ------------------------------------------------------------------------ SE(3)

def test_so3_exp_textbook_matrices():
    rows = [l for l in open(os.path.join(GOLDEN, "so3_textbook.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) >= 4
    for row in rows:
        lhs, rhs = row.split("|")
        ax = np.array([float(v) for v in lhs.split()[:3]])
        ang = np.deg2rad(float(lhs.split()[3]))
        R_expected = np.array([float(v) for v in rhs.split()]).reshape(3, 3)
        np.testing.assert_allclose(O.so3_exp(ax * ang), R_expected, atol=1e-15)


def test_se3_exp_matches_matrix_exponential():
    rng = np.random.default_rng(0)
    for _ in range(200):
        xi = rng.standard_normal(6) * rng.choice([1e-9, 1e-7, 1e-4, 0.1, 1.0])
        got = as4(O.se3_exp(xi))
        ref = linalg.expm(twist_matrix(xi))
        np.testing.assert_allclose(got, ref, atol=1e-13, rtol=0)


def test_se3_small_angle_branch_is_continuous():
    axis = np.array([0.3, -0.5, 0.81])
    axis /= np.linalg.norm(axis)
    for th in (0.999e-6, 1.0e-6, 1.001e-6, 1e-8):
        xi = np.concatenate([[1.0, -2.0, 3.0], axis * th])
        np.testing.assert_allclose(as4(O.se3_exp(xi)), linalg.expm(twist_matrix(xi)), atol=1e-15)


def test_se3_log_exp_round_trip():
    rng = np.random.default_rng(1)
    for _ in range(200):
        w = rng.standard_normal(3)
        w *= rng.uniform(1e-8, 3.0) / np.linalg.norm(w)
        xi = np.concatenate([rng.standard_normal(3) * 50, w])
        np.testing.assert_allclose(O.se3_log(O.se3_exp(xi)), xi, atol=1e-10, rtol=1e-10)


def test_pose_update_is_left_multiplication():
    rng = np.random.default_rng(2)
    for _ in range(50):
        T = O.se3_exp(rng.standard_normal(6))
        xi = rng.standard_normal(6) * 0.1
        np.testing.assert_allclose(as4(O.pose_update(xi, T)), linalg.expm(twist_matrix(xi)) @ as4(T),
                                   atol=1e-13)


# ------------------------------------------------------------------------ Huber

@pytest.mark.parametrize("delta", [0.1, 1.0, 2.5])
def test_huber_closed_form_and_continuity(delta):
    d2 = delta * delta
    for s in (0.0, 0.3 * d2, d2):
        rho, d = O.huber(s, delta)
        assert rho == pytest.approx(s) and d == 1.0
    for s in (1.5 * d2, 10 * d2, 1e4 * d2):
        rho, d = O.huber(s, delta)
        assert rho == pytest.approx(2 * delta * np.sqrt(s) - d2, rel=1e-14)
        assert d == pytest.approx(delta / np.sqrt(s), rel=1e-14)
    eps = 1e-9 * d2
    lo, dlo = O.huber(d2 - eps, delta)
    hi, dhi = O.huber(d2 + eps, delta)
    assert abs(hi - lo) < 3 * eps and abs(dhi - dlo) < 1e-8
    for s in (0.5 * d2, 3 * d2, 50 * d2):
        h = 1e-6 * s
        fd = (O.huber(s + h, delta)[0] - O.huber(s - h, delta)[0]) / (2 * h)
        assert O.huber(s, delta)[1] == pytest.approx(fd, rel=1e-7)


# --------------------------------------------------------------------- bilinear

def test_bilinear_exact_on_affine_maps():
    rng = np.random.default_rng(3)
    H, W, C = 9, 13, 5
    a, b, c = rng.standard_normal((3, C))
    yy, xx = np.mgrid[0:H, 0:W]
    fmap = (a[None, None] * xx[..., None] + b[None, None] * yy[..., None] + c[None, None]).astype(np.float32)
    pts = [(0.0, 0.0), (W - 1.0, H - 1.0), (3.0, 4.0), (W - 1.0, 2.5), (5.5, H - 1.0)]
    pts += [tuple(rng.uniform([0, 0], [W - 1, H - 1])) for _ in range(50)]
    for x, y in pts:
        ok, f, fx, fy = O.bilinear(fmap, x, y)
        assert ok
        np.testing.assert_allclose(f, (a * x + b * y + c).astype(np.float64), atol=2e-5)
        np.testing.assert_allclose(fx, a, atol=2e-5)
        np.testing.assert_allclose(fy, b, atol=2e-5)


def test_bilinear_matches_scipy_linear_interpolation():
    rng = np.random.default_rng(4)
    fmap = rng.standard_normal((20, 30, 3)).astype(np.float32)
    for _ in range(200):
        x, y = rng.uniform(0, 29), rng.uniform(0, 19)
        ok, f, _, _ = O.bilinear(fmap, x, y)
        ref = [ndimage.map_coordinates(fmap[:, :, ch].astype(np.float64), [[y], [x]], order=1)[0]
               for ch in range(3)]
        np.testing.assert_allclose(f, ref, atol=1e-12)


def test_bilinear_gradient_matches_finite_differences_inside_cells():
    rng = np.random.default_rng(5)
    fmap = rng.standard_normal((16, 16, 4)).astype(np.float32)
    for _ in range(100):
        x = rng.integers(0, 14) + rng.uniform(0.05, 0.95)
        y = rng.integers(0, 14) + rng.uniform(0.05, 0.95)
        h = 1e-6
        _, f, fx, fy = O.bilinear(fmap, x, y)
        fdx = (O.bilinear(fmap, x + h, y)[1] - O.bilinear(fmap, x - h, y)[1]) / (2 * h)
        fdy = (O.bilinear(fmap, x, y + h)[1] - O.bilinear(fmap, x, y - h)[1]) / (2 * h)
        np.testing.assert_allclose(fx, fdx, atol=1e-8)
        np.testing.assert_allclose(fy, fdy, atol=1e-8)


def test_bilinear_bounds():
    fmap = np.ones((4, 5, 2), np.float32)
    assert not O.bilinear(fmap, -1e-9, 1.0)[0]
    assert not O.bilinear(fmap, 4.0 + 1e-9, 1.0)[0]
    assert not O.bilinear(fmap, 1.0, 3.0 + 1e-9)[0]
    assert not O.bilinear(fmap, np.nan, 1.0)[0]
    assert O.bilinear(fmap, 4.0, 3.0)[0]


# --------------------------------------------------------------------- Cholesky

def test_cholesky_solve_matches_dense_solver():
    rng = np.random.default_rng(6)
    for _ in range(100):
        A = rng.standard_normal((6, 6))
        A = A @ A.T + rng.uniform(1e-6, 1.0) * np.eye(6)
        b = rng.standard_normal(6)
        ok, x = O.cholesky_solve(A, b)
        assert ok
        np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-9, atol=1e-9)


def test_cholesky_rejects_indefinite_and_nan():
    A = np.eye(6)
    A[3, 3] = -1.0
    assert not O.cholesky_solve(A, np.ones(6))[0]
    assert not O.cholesky_solve(np.zeros((6, 6)), np.ones(6))[0]
    B = np.eye(6)
    B[0, 0] = np.nan
    assert not O.cholesky_solve(B, np.ones(6))[0]
