"""Pins of the oracle's query-confidence weighting (Eq. 2's w_l(j) = anchor weight x query
confidence w^q_l at the anchor's projection, held constant when linearising):

* an affine confidence map is read exactly (bilinear interpolation is exact on affine maps)
  at the projection computed independently through the 3 x 4 matrix K [R | t];
* a constant confidence c weights the photo term exactly like an anchor weight c;
* an anchor that does not project into the map has confidence 0 (it is not counted).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_31098_gb300 import scenes as S


@pytest.fixture(scope="module")
def frame():
    return S.make_frame(S.config_reduced_frame(crop_side=40, n_hyps=2), S.frame_seed(2, 700))


def test_affine_confidence_is_read_at_the_projection(frame):
    confs = []
    for q in frame.qry_feat:
        H, W = q.shape[:2]
        rr, cc = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
        confs.append((0.3 + 0.002 * cc + 0.001 * rr).astype(np.float32))
    f = frame.replace(qry_conf=confs)
    T = f.T_hyps[0]
    for level in range(f.L):
        s = 2.0 ** -level
        u, v, z = S.project_gt(f.points, T, f.fx * s, f.cx * s, f.cy * s)
        x, y = u - 0.5, v - 0.5
        H, W = f.qry_feat[level].shape[:2]
        inside = (z > 0.1) & (x >= 0) & (x <= W - 1) & (y >= 0) & (y <= H - 1) & (f.point_valid > 0)
        w = O.query_confidences(f, level, T)
        np.testing.assert_allclose(w[inside], 0.3 + 0.002 * x[inside] + 0.001 * y[inside], atol=1e-6)
        assert np.all(w[~inside] == 0.0)


def test_constant_confidence_acts_as_an_anchor_weight(frame):
    c = 0.37
    confs = [np.full(q.shape[:2], c, np.float32) for q in frame.qry_feat]
    oo = O.SolverOptions()
    T = frame.T_hyps[1]
    for level in range(frame.L):
        a = O.evaluate(frame.replace(qry_conf=confs), oo, level, T)
        b = O.evaluate(frame.replace(point_weight=(frame.point_weight * np.float32(c)).astype(np.float32)),
                       oo, level, T)
        np.testing.assert_allclose(a, b, rtol=1e-6, atol=1e-12)
        base = O.evaluate(frame, oo, level, T)
        assert a[27] != pytest.approx(base[27], rel=1e-3)
