"""Write lines_patches_2048_N64.npz: the FP64 oracle's result for the
2048x2048, N=64 workload (85 % of the pixels corrupted, one interval of
1000 Crank-Nicolson steps), for the main run (beta = 0.25, T = 50) and the
stiff run (beta = 10, T = 1000, so beta dt = 10).

Calls only oracle/ and synth/. The orientation bins are the oracle's own
(FP64 decision on the FP32-rounded image the GPU also receives; the GPU
tests recompute them with oracle.orient, a few seconds). The projected
images are stored at every 4th row and column (512 x 512 samples of the
2048 x 2048 result, float32: its 6e-8 relative resolution is far below the
1e-5 comparison tolerance). Takes about 20 minutes per run on 8 cores (the
oracle integrates all 2048^2 frequencies x 64 angles x 1000 steps);
`python make_reference_2048.py main` writes only the main run.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(HERE, "lines_patches_2048_N64.npz")
STRIDE = 4


def run(stress):
    w = synth.workload_2048(stress=stress)
    f = w.f.astype(np.float32).astype(np.float64)
    p = oracle.Params(N=w.N, beta=w.beta, T=w.T, steps=w.steps, rounds=w.rounds, eps=w.eps)
    bins = oracle.orient(f, w.mask, p.N)["bins"]
    t0 = time.time()
    out = oracle.inpaint(f, w.mask, p, bins=bins)["out"]
    secs = time.time() - t0
    print(f"{w.name}: {secs:.1f} s", flush=True)
    return out[::STRIDE, ::STRIDE].astype(np.float32), np.array([p.N, p.beta, p.T, p.steps, p.rounds]), secs


def main():
    which = sys.argv[1:] or ["main", "stress"]
    data = dict(np.load(OUT)) if os.path.exists(OUT) else {}
    for name in which:
        out, params, secs = run(name == "stress")
        data[f"{name}_out"] = out
        data[f"{name}_params"] = params
        data[f"{name}_seconds"] = np.array([secs])
    data["stride"] = np.array([STRIDE])
    np.savez_compressed(OUT, **data)
    print(f"wrote {OUT}")


if __name__ == "__main__":
    main()
