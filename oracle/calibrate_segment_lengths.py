"""Calibrates L(N): the longest uniform segment (as a divisor of the orbital
period) for which the oracle converges to tol 1e-13 within 40 sweeps, with the
resolution test passing and no halving, over one revolution of the config-1
orbit (a = 0.75 AU, e = 0.3, Sun + Venus + Earth).  The uneven-batching
workload draws segment counts from this table.

    python -m oracle.calibrate_segment_lengths

Test infrastructure: runs the oracle only.
"""
import numpy as np

from oracle import oracle as ora
from paper_2301_03989_gb300 import workloads as W


def segments_per_period(N: int) -> int:
    w = W.config1(M=1)
    m = ora.Model.from_workload(w)
    T = w.meta["revolution_s"]
    for k in range(1, 257):
        o = ora.Opts(N=N, segments=k, seg_mode=0, tol=1e-13, max_iters=40, max_depth=0)
        r = ora.propagate(m, o, w.x0[:1], 0.0, T)
        if r["status"][0] == 0 and r["nseg"][0] == k:
            return k
    raise RuntimeError(f"no segment count up to 256 converges at N = {N}")


if __name__ == "__main__":
    for N in (32, 64, 128, 256):
        k = segments_per_period(N)
        print(f"N = {N:3d}: {k} segments per revolution")
