"""Precision sweep on the full-frame scene: the selected pose of each storage type (FP32,
BF16, FP16, FP8-E4M3 with per-channel absmax scales; FP32 arithmetic) against the FP64
oracle, over seeded frames.

For every seed the GPU solves the frame once per storage type; the oracle (on the FP32
features) then solves the hypotheses any storage type selected, and each type's selected
pose is compared with the oracle's end point of the same hypothesis (hypotheses are
independent without pruning, so this equals the oracle's full solve for them).  Also
reported: the oracle's end point against the synthetic ground truth.

The bar: FP32, BF16 and FP16 storage must be within the pose tolerance (1e-3 deg, 1 mm)
on every seed -- these are the forms at equal pose accuracy.  FP8-E4M3 is reported, not
bounded: on some seeds its objective selects another basin.

By default a few seeds run; PILOT_SWEEP_SEEDS=256 runs the full sweep and PILOT_SWEEP_OUT
names a JSON file for the report:

    PILOT_SWEEP_SEEDS=256 PILOT_SWEEP_OUT=sweep.json python -m pytest -m gpu -s \
        tests/test_gpu_precision_sweep.py
"""
import json
import multiprocessing as mp
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_31098_gb300 import binding as B
from paper_2606_31098_gb300 import scenes as S

from gpu_support import ROT_TOL_DEG, TRANS_TOL_M, require_cuda

pytestmark = pytest.mark.gpu

EQUAL_ACCURACY = ("f32", "bf16", "f16")


def sweep(n_seeds: int, chunk: int = 16) -> dict:
    dtypes = (B.F32, B.BF16, B.F16, B.FP8E4M3)
    solver = B.Solver(B.Options())
    errs = {B.DTYPE_NAMES[d]: [] for d in dtypes}
    gt_err = []
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(chunk, os.cpu_count() or 4)) as pool:
        for start in range(0, n_seeds, chunk):
            frames = pool.starmap(S.make_frame, [(S.config_full_frame(), S.frame_seed(4, k))
                                                 for k in range(start, min(start + chunk, n_seeds))])
            for f in frames:
                winners = {}
                for d in dtypes:
                    r = solver.solve(B.FrameArgs(f, B.quantized_device_arrays(f, d), is_device=True, dtype=d))
                    winners[d] = (r.best, r.T_cw[r.best].copy() if r.best >= 0 else None)
                hyps = sorted({b for b, _ in winners.values() if b >= 0})
                o = O.solve(f, O.SolverOptions(), T_hyps=f.T_hyps[hyps])
                by_hyp = {h: o.T_cw[k] for k, h in enumerate(hyps)}
                for d, (b, T) in winners.items():
                    if b < 0:
                        errs[B.DTYPE_NAMES[d]].append((np.inf, np.inf))
                        continue
                    errs[B.DTYPE_NAMES[d]].append((S.rotation_error_deg(T, by_hyp[b]),
                                                   S.translation_error_m(T, by_hyp[b])))
                b32 = winners[B.F32][0]
                if b32 >= 0:
                    gt_err.append((S.rotation_error_deg(by_hyp[b32], f.T_gt),
                                   S.translation_error_m(by_hyp[b32], f.T_gt)))
    solver.close()

    def stats(v):
        a = np.array(v)
        return {"p50": float(np.percentile(a, 50)), "p99": float(np.percentile(a, 99)), "max": float(a.max())}

    return {"seeds": n_seeds, "scene": "full frame (256^2 anchors, C=32, 3 levels, 64 hypotheses, priors)",
            "comparison": "selected pose vs the FP64 oracle's end point of the same hypothesis",
            "per_dtype": {k: {"rot_deg": stats([e[0] for e in v]), "trans_m": stats([e[1] for e in v])}
                          for k, v in errs.items()},
            "oracle_vs_ground_truth": {"rot_deg": stats([e[0] for e in gt_err]),
                                       "trans_m": stats([e[1] for e in gt_err])}}


def test_precision_sweep_selected_pose_error(tmp_path):
    require_cuda()
    n = int(os.environ.get("PILOT_SWEEP_SEEDS", "4"))
    report = sweep(n)
    print(json.dumps(report, indent=1))
    out = os.environ.get("PILOT_SWEEP_OUT")
    if out:
        os.makedirs(os.path.dirname(out) or ".", exist_ok=True)
        json.dump(report, open(out, "w"), indent=1)
    for name in EQUAL_ACCURACY:
        worst = report["per_dtype"][name]
        assert worst["rot_deg"]["max"] <= ROT_TOL_DEG and worst["trans_m"]["max"] <= TRANS_TOL_M, (name, worst)
