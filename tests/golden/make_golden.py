"""Write the oracle's expected values for the full-size workloads.

Calls only ``oracle`` (and the seeded generators in ``workloads``).  For each
workload it stores the r leading singular values and the left singular
vectors U (L x r) of the FP64 oracle, plus the shape counts; the GPU parity
tests compare against these and recompute sampled reconstruction elements from
U with ``oracle.reconstruct_at``.

Run from the repository root:  python tests/golden/make_golden.py [name ...]
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import ssa_oracle as O  # noqa: E402
import workloads as W  # noqa: E402


def problem(name):
    cfg = W.CONFIGS[name]
    if cfg["kind"] == "1d":
        return O.Problem.series(W.series_1d(cfg["n"], seed=cfg["seed"]), cfg["L"]), cfg
    if cfg["kind"] == "mssa":
        return O.Problem.multi(W.mssa_series(cfg["s"], seed=cfg["seed"]), cfg["L"]), cfg
    if cfg["kind"] == "2d":
        x = W.harmonic_image(cfg["nx"], cfg["ny"], seed=cfg["seed"])
        return O.Problem.image(x, cfg["lx"], cfg["ly"]), cfg
    x, mask, info = W.shaped_image(cfg["nx"], cfg["ny"], seed=cfg["seed"])
    cfg = dict(cfg, **info)
    return O.Problem.image(x, cfg["lx"], cfg["ly"], mask=mask), cfg


def main(names):
    for name in names:
        t0 = time.time()
        P, cfg = problem(name)
        r = cfg["rank"]
        sigma, U, V = O.decompose(P, r, "eigen")
        extra = {k: v for k, v in cfg.items() if isinstance(v, (int, float))}
        np.savez_compressed(os.path.join(HERE, f"{name}.npz"), sigma=sigma, U=U,
                            L=P.L, K=P.K, Ks=np.array(P.Ks),
                            meta=np.array(repr(extra)))
        print(f"{name}: L={P.L} K={P.K} sigma[0]={sigma[0]:.6g} "
              f"sigma[-1]={sigma[-1]:.6g}  {time.time() - t0:.1f}s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(W.CONFIGS))
