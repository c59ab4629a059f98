"""Precision sweep on the full-frame scene: selected-pose error of each storage type
(FP32, BF16, FP16, FP8-E4M3, per-channel absmax scales, FP32 arithmetic) against the FP64
oracle, over many seeds.

For every seed the GPU solves the frame once per storage type; the oracle (on the FP32
features) then solves the hypotheses any storage type selected, and each type's selected
pose is compared with the oracle's end point of the same hypothesis.  (Solving all 64
hypotheses per seed in FP64 would take minutes per seed; hypotheses are independent, so the
subset gives the same end points.)  Also reported: the error of the oracle's end point
against the synthetic ground truth.

    python tests/precision_sweep.py --seeds 64 --out precision_sweep.json

Test infrastructure (it runs the oracle); not collected by pytest.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2606_31098_gb300 import scenes as S  # noqa: E402


def _make(seed):
    return S.make_frame(S.config_full_frame(), S.frame_seed(4, seed))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--seeds", type=int, default=64)
    ap.add_argument("--chunk", type=int, default=16)
    ap.add_argument("--out", default="")
    args = ap.parse_args()
    pool = mp.get_context("spawn").Pool(min(args.chunk, os.cpu_count() or 4))   # before any CUDA call
    import torch

    from oracle import oracle as O
    from paper_2606_31098_gb300 import binding as B
    from paper_2606_31098_gb300 import build_ext

    build_ext.build()
    B.load()
    dtypes = (B.F32, B.BF16, B.F16, B.FP8E4M3)
    solver = B.Solver(B.Options())
    errs = {B.DTYPE_NAMES[d]: [] for d in dtypes}
    gt_err = []
    t0 = time.time()
    for start in range(0, args.seeds, args.chunk):
        frames = pool.map(_make, range(start, min(start + args.chunk, args.seeds)))
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
                gt_err.append((S.rotation_error_deg(by_hyp[b32], f.T_gt), S.translation_error_m(by_hyp[b32], f.T_gt)))
        torch.cuda.synchronize()
        print(f"{min(start + args.chunk, args.seeds)} seeds, {time.time() - t0:.0f} s", flush=True)
    pool.close()

    def stats(v):
        a = np.array(v)
        return {"p50": float(np.percentile(a, 50)), "p99": float(np.percentile(a, 99)), "max": float(a.max())}

    report = {"seeds": args.seeds, "scene": "full frame (256^2 anchors, C=32, 3 levels, 64 hypotheses, priors)",
              "comparison": "selected pose vs the FP64 oracle's end point of the same hypothesis",
              "per_dtype": {k: {"rot_deg": stats([e[0] for e in v]), "trans_m": stats([e[1] for e in v])}
                            for k, v in errs.items()},
              "oracle_vs_ground_truth": {"rot_deg": stats([e[0] for e in gt_err]),
                                         "trans_m": stats([e[1] for e in gt_err])}}
    print(json.dumps(report, indent=1))
    if args.out:
        os.makedirs(os.path.dirname(args.out) or ".", exist_ok=True)
        json.dump(report, open(args.out, "w"), indent=1)


if __name__ == "__main__":
    main()
