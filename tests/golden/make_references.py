"""Write the FP64 oracle's result for the full 512x512, N=32 workload
(beta = 0.25, 10 restoration intervals of 500 Crank-Nicolson steps, T = 2
per interval, eps = 0.5) to curves_noise_512_N32.npz.

Calls only oracle/ and synth/. The orientation bins are the oracle's own
(FP64 decision on the FP32-rounded image the GPU also receives); the stored
image is the oracle's projected output, rounded to float32 (its 6e-8
relative resolution is far below the 1e-5 comparison tolerance).
Takes about 3 minutes on 8 cores.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(HERE, "curves_noise_512_N32.npz")


def main():
    w = synth.workload_512()
    f = w.f.astype(np.float32).astype(np.float64)
    p = oracle.Params(N=w.N, beta=w.beta, T=w.T, steps=w.steps, rounds=w.rounds, eps=w.eps)
    bins = oracle.orient(f, w.mask, p.N)["bins"]
    t0 = time.time()
    out = oracle.inpaint(f, w.mask, p, bins=bins)["out"]
    secs = time.time() - t0
    np.savez_compressed(OUT, out=out.astype(np.float32), bins=bins,
                        params=np.array([p.N, p.beta, p.T, p.steps, p.rounds, p.eps]),
                        oracle_seconds=np.array([secs]))
    print(f"wrote {OUT} in {secs:.1f} s")


if __name__ == "__main__":
    main()
