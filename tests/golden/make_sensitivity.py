"""Write sensitivity_512_N32.json: how far FP32 rounding moves the FP64
oracle's result on the full 512x512, N=32 workload (beta = 0.25, 10
restoration intervals of 500 Crank-Nicolson steps, T = 2 per interval,
eps = 0.5, guard 0.1), measured against the oracle's own FP64 run.

Calls only oracle/ and synth/ (oracle.sensitivity injects the rounding; see
its docstring). Each variant takes about 2-4 minutes on 8 cores.
`python make_sensitivity.py 30` does the same for the paper's angle count
N = 30 (sensitivity_512_N30.json).
Entries: max-abs of the change relative to max|f|, its pixel, and the
relative L2 change of the image, for
  storage_full / perturb_full   -- FP32 storage rounding, or a random
                                   2^-24 relative perturbation, full spectrum;
  fp32_full / fp32_half         -- FP32 transforms and storage, on the full
                                   spectrum or on the Hermitian half (the
                                   layout of the library's default path).
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402
from oracle import sensitivity  # noqa: E402

def main():
    N = int(sys.argv[1]) if len(sys.argv) > 1 else 32
    out_path = os.path.join(HERE, f"sensitivity_512_N{N}.json")
    w = synth.workload_512(N=N)
    f = w.f.astype(np.float32).astype(np.float64)
    p = oracle.Params(N=w.N, beta=w.beta, T=w.T, steps=w.steps, rounds=w.rounds, eps=w.eps)
    bins = oracle.orient(f, w.mask, p.N)["bins"]
    t0 = time.time()
    ref = oracle.inpaint(f, w.mask, p, bins=bins)["out"]
    res = {"workload": f"curves_noise_512_N{N}: 512x512, N={N}, beta=0.25, 10 x 500 steps, T=20, eps=0.5, guard=0.1",
           "reference": "oracle.inpaint in FP64", "oracle_seconds": round(time.time() - t0, 1)}
    mf = float(np.abs(f).max())
    for name, mode, half in [("storage_full", "storage", False), ("perturb_full", "perturb", False),
                             ("fp32_full", "fp32", False), ("fp32_half", "fp32", True)]:
        t0 = time.time()
        out = sensitivity.inpaint_rounded(f, w.mask, p, bins=bins, mode=mode, half=half)
        d = np.abs(out - ref)
        y, x = np.unravel_index(int(d.argmax()), d.shape)
        res[name] = {"max_abs_over_max_f": float(d.max() / mf), "pixel": [int(y), int(x)],
                     "rel_l2": float(np.linalg.norm(out - ref) / np.linalg.norm(ref)),
                     "seconds": round(time.time() - t0, 1)}
        print(name, res[name], flush=True)
    with open(out_path, "w") as fh:
        json.dump(res, fh, indent=1)
    print(f"wrote {out_path}")


if __name__ == "__main__":
    main()
