"""Pipe-rate probe (measurement support): builds ``pipe_rates.cu`` for sm_103a, runs it while
nvidia-smi samples the SM clock, and prints one JSON line with each instruction kind's rate in
operations per second and per SM per clock at the median sampled clock.

Usage: ``python -m paper_2312_02756_gb300.probe [iters]``.
"""
from __future__ import annotations

import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(os.path.dirname(HERE), "_build")
EXE = os.path.join(BUILD, "pipe_rates_%s" % platform.machine())


def build() -> str:
    from ..build import ARCH, nvcc
    os.makedirs(BUILD, exist_ok=True)
    src = os.path.join(HERE, "pipe_rates.cu")
    if not os.path.exists(EXE) or os.path.getmtime(EXE) < os.path.getmtime(src):
        subprocess.run([nvcc(), *ARCH, "-O3", src, "-o", EXE], check=True)
    return EXE


def run(iters: int = 4096) -> dict:
    exe = build()
    with tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False) as log:
        path = log.name
    smi = None
    try:
        smi = subprocess.Popen(["nvidia-smi", "--query-gpu=clocks.sm,clocks.max.sm",
                                "--format=csv,noheader,nounits", "-lms", "100", "-f", path])
        time.sleep(0.3)
    except OSError:
        smi = None
    try:
        out = subprocess.run([exe, str(iters)], check=True, capture_output=True, text=True).stdout
    finally:
        if smi is not None:
            smi.terminate()
            smi.wait()
    res = json.loads(out.strip().splitlines()[-1])
    clocks = []
    try:
        with open(path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 2 and parts[0].isdigit():
                    clocks.append((int(parts[0]), int(parts[1])))
        os.unlink(path)
    except OSError:
        pass
    loaded = [c for c, mx in clocks if c > 0.5 * mx] or [c for c, _ in clocks]
    if loaded:
        mhz = statistics.median(loaded)
        res["sm_mhz_median"] = mhz
        res["clock_samples"] = len(clocks)
        for k, v in list(res.items()):
            if isinstance(v, dict) and "ops_per_s" in v:
                v["per_sm_per_clock"] = round(v["ops_per_s"] / (res["sms"] * mhz * 1e6), 3)
    return res


if __name__ == "__main__":
    print(json.dumps(run(int(sys.argv[1]) if len(sys.argv) > 1 else 4096)))
