"""Vendor baselines (cuSOLVER/cuBLAS) and pipe probes, timed beside libgp but never used by it."""
from __future__ import annotations

import json
import os
import subprocess

from .. import build as _b

SRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "vendor_baselines.cu")
EXE = os.path.join(_b.BUILD, "vendor_baselines")


def build() -> str:
    if not os.path.exists(EXE) or os.path.getmtime(EXE) < os.path.getmtime(SRC):
        os.makedirs(_b.BUILD, exist_ok=True)
        subprocess.check_call([_b._nvcc(), *_b.ARCH, "-O3", "-o", EXE, SRC, "-lcublas", "-lcusolver"])
    return EXE


def run(n: int = 32768, potrf: bool = True, timeout: float = 600.0, probes: bool = True, spotrf: bool = True,
        once: bool = False) -> dict:
    """Runs the probes; returns {probe name: record}. once: time the first Dpotrf call (no warm-up)."""
    args = [build(), str(n)] + ([] if potrf else ["--no-potrf"]) + ([] if probes else ["--no-probes"]) + \
        ([] if spotrf else ["--no-spotrf"]) + (["--once"] if once else [])
    out = subprocess.run(args, capture_output=True, text=True, timeout=timeout, check=True).stdout
    res = {}
    for line in out.splitlines():
        line = line.strip()
        if line.startswith("{"):
            rec = json.loads(line)
            res[rec.get("probe", "error")] = rec
    return res
