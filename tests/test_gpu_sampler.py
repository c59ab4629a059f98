"""Geo-anchor sampling on the GPU (pilot_sample_anchors; Supp. "TDOM/DSM Reference Crop")
against the oracle's seeded draw: the drawn pixel indices are integer work and must be
bit-exact, the gathered anchors exact copies.  Sizes span the batched crop sizes (up to
384^2 pixels = 144 CTA chunks per thread), ragged masks, fewer valid pixels than asked for,
nothing asked, and a real reference crop's mask.
"""
import numpy as np
import pytest

from oracle import sampler as OS
from paper_2606_31098_gb300 import binding as B

from gpu_support import require_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


def draw(torch, valid, points, n, seed):
    v = torch.as_tensor(np.asarray(valid, np.uint8), device="cuda")
    p = torch.as_tensor(np.ascontiguousarray(points, np.float32), device="cuda")
    out = B.sample_anchors(v, p, n, seed)
    torch.cuda.synchronize()
    c = int(out["count"].item())
    return out["idx"][:c].cpu().numpy(), out["points"][:, :c].cpu().numpy(), c


@pytest.mark.parametrize("n_pix,frac,n,seed", [(90 * 90, 0.8, 500, 1), (256 * 256, 0.95, 500, 2),
                                               (384 * 384, 0.6, 4000, 3), (1000, 0.01, 500, 4),
                                               (4097, 1.0, 4097, 5), (300, 0.5, 0, 6), (1, 1.0, 1, 7),
                                               (128 * 128, 0.5, 1, 2 ** 63 + 11)])
def test_device_draw_equals_the_oracle(torch, n_pix, frac, n, seed):
    rng = np.random.default_rng(seed % 1000)
    valid = rng.random(n_pix) < frac
    points = rng.standard_normal((3, n_pix)).astype(np.float32)
    idx, pts, c = draw(torch, valid, points, n, seed)
    want = OS.sample_anchors(valid, n, seed)
    assert c == len(want)
    np.testing.assert_array_equal(idx, want)
    np.testing.assert_array_equal(pts, points[:, want])


def test_draw_from_a_reference_crop(torch):
    from paper_2606_31098_gb300 import scenes as S
    g = S.make_global_map(side=2048, seed=3, n_hills=256, n_boxes=512)
    dm = B.MapArgs(torch.as_tensor(g.dsm, device="cuda"), None, g.x0, g.y0, g.gsd)
    pr = S.crop_prior(g, 1, margin=150.0)
    p = B.crop_params(pr["T_cw"], pr["fx"], pr["fy"], pr["cx"], pr["cy"], pr["img_w"], pr["img_h"],
                      0.0, 0.25, 8000, 192)
    crop = B.crop_reference(dm, p, with_rgb=False)
    out = B.sample_anchors(crop["valid"], crop["points"], 500, 2024)
    torch.cuda.synchronize()
    valid = crop["valid"].cpu().numpy()
    want = OS.sample_anchors(valid, 500, 2024)
    c = int(out["count"].item())
    assert c == len(want) == min(500, int(valid.astype(bool).sum()))
    np.testing.assert_array_equal(out["idx"][:c].cpu().numpy(), want)
    np.testing.assert_array_equal(out["points"][:, :c].cpu().numpy(), crop["points"].cpu().numpy()[:, want])
