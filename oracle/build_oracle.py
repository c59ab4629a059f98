"""Compile the FP64 CPU oracles (plain C: the pose solver and the reference crop) into
oracle/_lib/libpilot_oracle.so.

Test infrastructure only.  Uses gcc with OpenMP when the compiler supports it (the
loop over independent hypotheses is the only parallel loop); portable flags only.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, "pilot_oracle.c"), os.path.join(HERE, "crop_oracle.c")]
HDRS = [os.path.join(HERE, "pilot_oracle.h"), os.path.join(HERE, "crop_oracle.h")]
OUT_DIR = os.path.join(HERE, "_lib")
OUT = os.path.join(OUT_DIR, "libpilot_oracle.so")


def _compile(openmp: bool) -> subprocess.CompletedProcess:
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-Wextra",
           "-Wno-unused-parameter", "-ffp-contract=off", *SRCS, "-o", OUT + ".tmp", "-lm"]
    if openmp:
        cmd.insert(1, "-fopenmp")
    return subprocess.run(cmd, capture_output=True, text=True)


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(OUT)
            and os.path.getmtime(OUT) >= max(os.path.getmtime(f) for f in SRCS + HDRS)):
        return OUT
    res = _compile(openmp=True)
    if res.returncode != 0:
        res = _compile(openmp=False)
    if res.returncode != 0:
        raise RuntimeError("oracle build failed:\n" + res.stderr)
    os.replace(OUT + ".tmp", OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
