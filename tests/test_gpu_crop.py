"""Parity of the CUDA reference crop (pilot_crop_reference) with the FP64 crop oracle
(Supp. "TDOM/DSM Reference Crop"), on the seeded global map of the serving workload
(4096 x 4096 cells at 0.5 m) and on a smaller one.

Both sides compute the geometry in FP64 with the same formulas, so: equal sample indices
per corner ray (an arg-min), footprint points and origin within 1e-9 m, homography within
1e-9 (relative), equal validity masks, anchors within one FP32 rounding of the same doubles
(1e-4 m in x and y, 1e-5 m in height), TDOM colours within 1e-3.
"""
import numpy as np
import pytest

from oracle import crop as OC
from paper_2606_31098_gb300 import binding as B
from paper_2606_31098_gb300 import scenes as S

from gpu_support import require_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


@pytest.fixture(scope="module")
def maps(torch):
    out = {}
    for name, side, hills, boxes in (("small", 1024, 128, 256), ("full", 4096, 2048, 4096)):
        g = S.make_global_map(side=side, gsd=0.5, n_hills=hills, n_boxes=boxes, seed=21)
        out[name] = (g, OC.MapArgs(g.dsm, g.tdom, g.x0, g.y0, g.gsd),
                     B.MapArgs(torch.as_tensor(g.dsm, device="cuda"), torch.as_tensor(g.tdom, device="cuda"),
                               g.x0, g.y0, g.gsd))
    return out


def compare(torch, maps, name, seed, S_, step=0.25, n=8000, prior_kw=None):
    g, om, dm = maps[name]
    pr = S.crop_prior(g, seed, **(prior_kw or {}))
    args = (pr["T_cw"], pr["fx"], pr["fy"], pr["cx"], pr["cy"], pr["img_w"], pr["img_h"], 0.0, step, n, S_)
    o = OC.crop(om, OC.params(*args))
    d = B.crop_reference(dm, B.crop_params(*args))
    torch.cuda.synchronize()
    geo = d["geometry"].cpu().numpy()
    idx = geo[23:27].astype(int)
    np.testing.assert_array_equal(idx, o["idx"])
    assert bool(geo[27]) == o["ok"]
    np.testing.assert_allclose(geo[11:23].reshape(4, 3), o["quad"], atol=1e-9)
    if not o["ok"]:
        assert not d["valid"].any()
        return o, d
    np.testing.assert_allclose(geo[9:11], o["origin"], atol=1e-9)
    np.testing.assert_allclose(geo[:9], o["H"], rtol=1e-9, atol=1e-9)
    valid = d["valid"].cpu().numpy()
    np.testing.assert_array_equal(valid, o["valid"])
    pts = d["points"].cpu().numpy()
    np.testing.assert_allclose(pts[:2], o["points"][:2], atol=1e-4)
    np.testing.assert_allclose(pts[2], o["points"][2], atol=1e-5)
    np.testing.assert_allclose(d["rgb"].cpu().numpy(), o["rgb"], atol=1e-3)
    return o, d


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_crop_matches_the_oracle_small_map(torch, maps, seed):
    o, _ = compare(torch, maps, "small", seed, 96, n=4000,
                   prior_kw=dict(margin=150.0, altitude=(80.0, 120.0), pitch_deg=(45.0, 70.0)))
    assert o["ok"] and o["valid"].mean() > 0.9


@pytest.mark.parametrize("seed,S_", [(0, 256), (1, 384), (2, 256), (3, 383)])
def test_crop_matches_the_oracle_full_map(torch, maps, seed, S_):
    o, _ = compare(torch, maps, "full", seed, S_)
    assert o["ok"] and o["valid"].mean() > 0.9


def test_crop_edge_cases(torch, maps):
    # a shallow prior whose upper corner rays never come down to the DSM: no crop, all invalid
    o, d = compare(torch, maps, "small", 5, 32, n=600,
                   prior_kw=dict(margin=150.0, altitude=(80.0, 120.0), pitch_deg=(5.0, 6.0)))
    assert not o["ok"]
    # a one-pixel crop, and a crop without a TDOM (colours zero)
    compare(torch, maps, "small", 6, 1, n=4000, prior_kw=dict(margin=150.0, altitude=(80.0, 120.0), pitch_deg=(45.0, 70.0)))
    g, om, dm = maps["small"]
    bare = B.MapArgs(dm.dsm, None, g.x0, g.y0, g.gsd)
    pr = S.crop_prior(g, 7, margin=150.0, altitude=(80.0, 120.0), pitch_deg=(45.0, 70.0))
    p = B.crop_params(pr["T_cw"], pr["fx"], pr["fy"], pr["cx"], pr["cy"], pr["img_w"], pr["img_h"], 0.0, 0.25, 4000, 16)
    d = B.crop_reference(bare, p)
    torch.cuda.synchronize()
    assert float(d["rgb"].abs().max()) == 0.0 and bool(d["valid"].any())
    with pytest.raises(B.PilotError, match="S must"):
        B.crop_reference(dm, B.crop_params(pr["T_cw"], pr["fx"], pr["fy"], pr["cx"], pr["cy"], pr["img_w"],
                                           pr["img_h"], 0.0, 0.25, 4000, 0))
