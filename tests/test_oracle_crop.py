"""Pins of the FP64 crop oracle (Supp. "TDOM/DSM Reference Crop") against closed forms and
an independent library routine:

* a flat DSM: each corner ray's selected sample is the one nearest the ray-plane
  intersection, whose distance has a closed form;
* the homography maps its four source points exactly onto the four targets, and recovers a
  known projective map;
* warping an affine DSM / TDOM reproduces the affine values (bilinear interpolation is exact
  on affine fields);
* every valid geo-anchor's height equals scipy's bilinear read of the DSM at its map
  coordinates (an implementation independent of the oracle).
"""
import numpy as np
import pytest
from scipy import ndimage

from oracle import crop as OC
from paper_2606_31098_gb300 import scenes as S


def flat_map(side=512, gsd=1.0, h0=12.5, tdom=None):
    dsm = np.full((side, side), h0, np.float32)
    return OC.MapArgs(dsm, tdom, -side * gsd / 2, -side * gsd / 2, gsd)


def prior(seed=3, **kw):
    g = S.GlobalMap(dsm=np.zeros((512, 512), np.float32), tdom=np.zeros((512, 512, 3), np.uint8),
                    x0=-256.0, y0=-256.0, gsd=1.0)
    return S.crop_prior(g, seed, margin=150.0, altitude=(80.0, 120.0), pitch_deg=(45.0, 70.0), **kw)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_flat_dsm_footprint_is_the_nearest_sample_to_the_ray_plane_intersection(seed):
    m = flat_map()
    pr = prior(seed)
    step = 0.5
    p = OC.params(pr["T_cw"], pr["fx"], pr["fy"], pr["cx"], pr["cy"], pr["img_w"], pr["img_h"], 0.0, step, 1200, 64)
    quad, idx = OC.footprint(m, p)
    T = np.asarray(pr["T_cw"]).reshape(3, 4)
    R, t = T[:, :3], T[:, 3]
    C = -R.T @ t
    for k, (u, v) in enumerate([(0, 0), (pr["img_w"], 0), (pr["img_w"], pr["img_h"]), (0, pr["img_h"])]):
        d = R.T @ np.array([(u - pr["cx"]) / pr["fx"], (v - pr["cy"]) / pr["fy"], 1.0])
        d /= np.linalg.norm(d)
        t_star = (12.5 - C[2]) / d[2]
        assert idx[k] == int(np.floor(t_star / step + 0.5)), (k, idx[k], t_star / step)
        np.testing.assert_allclose(quad[k], C + idx[k] * step * d, atol=1e-9)
        assert abs(quad[k][2] - 12.5) <= abs(d[2]) * step / 2 + 1e-9


def test_homography_maps_the_four_points_and_recovers_a_projective_map():
    rng = np.random.default_rng(7)
    src = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], float)
    Htrue = np.array([[120.0, 30.0, -40.0], [-25.0, 95.0, 10.0], [0.15, -0.08, 1.0]])
    dst = np.array([(Htrue @ [u, v, 1.0])[:2] / (Htrue @ [u, v, 1.0])[2] for u, v in src])
    ok, H = OC.homography(src, dst)
    assert ok
    np.testing.assert_allclose(H.reshape(3, 3), Htrue, rtol=1e-10, atol=1e-9)
    for _ in range(5):
        quad = rng.uniform(-300, 300, (4, 2))
        ok, H = OC.homography(src, quad)
        assert ok
        for (u, v), q in zip(src, quad):
            w = H[6] * u + H[7] * v + H[8]
            np.testing.assert_allclose([(H[0] * u + H[1] * v + H[2]) / w, (H[3] * u + H[4] * v + H[5]) / w], q,
                                       atol=1e-9)


def test_warp_is_exact_on_affine_layers():
    side, gsd = 256, 0.5
    x0 = y0 = -side * gsd / 2
    cc, rr = np.meshgrid(np.arange(side) + 0.5, np.arange(side) + 0.5)
    X, Y = x0 + cc * gsd, y0 + rr * gsd
    dsm = (0.03 * X - 0.02 * Y + 7.0).astype(np.float32)
    tdom = np.stack([np.round(100 + 0.8 * (cc - 100)), np.round(90 + 0.5 * (rr - 80)),
                     np.full_like(cc, 60.0)], axis=2)
    tdom = np.clip(tdom, 0, 255).astype(np.uint8)
    m = OC.MapArgs(dsm, tdom, x0, y0, gsd)
    quad = np.array([[-40.0, 30.0], [35.0, 42.0], [30.0, -33.0], [-38.0, -28.0]])
    ok, H = OC.homography(np.array([[0, 0], [1, 0], [1, 1], [0, 1]], float), quad)
    S_ = 48
    pts, valid, rgb = OC.warp(m, H, S_, 0.0, 0.0)
    assert valid.all()
    x, y, z = pts.astype(np.float64)
    np.testing.assert_allclose(z, 0.03 * x - 0.02 * y + 7.0, atol=1e-4)
    col, row = (x - x0) / gsd - 0.5, (y - y0) / gsd - 0.5
    inner = (col > 1) & (col < side - 2) & (row > 1) & (row < side - 2)
    np.testing.assert_allclose(rgb[inner, 2], 60.0, atol=1e-4)
    # red and green are affine in the cell index up to the 8-bit rounding of the stored texels
    np.testing.assert_allclose(rgb[inner, 0], 100 + 0.8 * (col[inner] + 0.5 - 100), atol=0.51)
    np.testing.assert_allclose(rgb[inner, 1], 90 + 0.5 * (row[inner] + 0.5 - 80), atol=0.51)


def test_anchors_lie_on_the_dsm_read_by_scipy():
    g = S.make_global_map(side=1024, gsd=0.5, n_hills=128, n_boxes=256, seed=11)
    m = OC.MapArgs(g.dsm, g.tdom, g.x0, g.y0, g.gsd)
    pr = S.crop_prior(g, 4, margin=150.0, altitude=(80.0, 120.0), pitch_deg=(45.0, 70.0))
    p = OC.params(pr["T_cw"], pr["fx"], pr["fy"], pr["cx"], pr["cy"], pr["img_w"], pr["img_h"], 0.0, 0.25, 2400, 96)
    r = OC.crop(m, p)
    assert r["ok"] and r["valid"].mean() > 0.9
    x = r["points"][0].astype(np.float64) + r["origin"][0]
    y = r["points"][1].astype(np.float64) + r["origin"][1]
    v = r["valid"].astype(bool)
    col, row = (x - g.x0) / g.gsd - 0.5, (y - g.y0) / g.gsd - 0.5
    ref = ndimage.map_coordinates(g.dsm.astype(np.float64), [row[v], col[v]], order=1, mode="nearest")
    # float32 storage of the anchors' x, y moves the read point by < 1e-4 m
    np.testing.assert_allclose(r["points"][2][v], ref, atol=2e-3)
    # the crop corners map onto the footprint (homography of the normalised crop square)
    H = r["H"]
    for (a, b), q in zip([(0, 0), (1, 0), (1, 1), (0, 1)], r["quad"]):
        w = H[6] * a + H[7] * b + H[8]
        np.testing.assert_allclose([(H[0] * a + H[1] * b + H[2]) / w + r["origin"][0],
                                    (H[3] * a + H[4] * b + H[5]) / w + r["origin"][1]], q[:2], atol=1e-8)


def test_equal_distances_select_the_first_sample():
    """Arg-min ties go to the nearest sample along the ray: a nadir ray (R = diag(1, -1, -1),
    principal point at the image corner) midway between two samples over a flat DSM."""
    m = flat_map(h0=10.0)
    C = np.array([3.0, -4.0, 10.0 + 100.5 * 0.5])
    R = np.diag([1.0, -1.0, -1.0])
    T = np.hstack([R, (-R @ C)[:, None]])
    p = OC.params(T, 500.0, 500.0, 0.0, 0.0, 640, 480, 0.0, 0.5, 400, 32)
    quad, idx = OC.footprint(m, p)
    assert idx[0] == 100
    np.testing.assert_allclose(quad[0], [3.0, -4.0, 10.25], atol=1e-12)


def test_square_footprint_samples_the_map_at_crop_pixel_centres():
    """Pixel alignment: for an axis-aligned square footprint of side L, crop pixel (u, v)
    reads the map at (X0 + (u + 1/2) L / S, Y0 + (v + 1/2) L / S)."""
    side, gsd = 128, 1.0
    x0 = y0 = -side * gsd / 2
    cc, rr = np.meshgrid(np.arange(side) + 0.5, np.arange(side) + 0.5)
    dsm = (0.25 * (x0 + cc * gsd) + 0.5 * (y0 + rr * gsd) + 3.0).astype(np.float32)
    m = OC.MapArgs(dsm, None, x0, y0, gsd)
    X0, Y0, L, S_ = -20.0, -10.0, 32.0, 16
    ok, H = OC.homography(np.array([[0, 0], [1, 0], [1, 1], [0, 1]], float),
                          np.array([[X0, Y0], [X0 + L, Y0], [X0 + L, Y0 + L], [X0, Y0 + L]]))
    pts, valid, _ = OC.warp(m, H, S_, 0.0, 0.0, with_rgb=False)
    u, v = np.meshgrid(np.arange(S_), np.arange(S_))
    xs, ys = X0 + (u.ravel() + 0.5) * L / S_, Y0 + (v.ravel() + 0.5) * L / S_
    assert valid.all()
    np.testing.assert_allclose(pts[0], xs, atol=1e-5)
    np.testing.assert_allclose(pts[1], ys, atol=1e-5)
    np.testing.assert_allclose(pts[2], 0.25 * xs + 0.5 * ys + 3.0, atol=1e-4)
