"""Run a few coupled steps on an L^3 BPII lattice, for profilers.

    python -m paper_0901_3293_gb300.profile --size 128 --steps 4 [--dtype f32]

Each step launches the three step kernels once (no CUDA graph), so a
profiler can select them by name and launch index.
"""

from __future__ import annotations

import argparse
import math

import torch

from . import build, lcbp


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--size", type=int, default=128)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--dtype", default="f32")
    args = ap.parse_args()
    build.build()
    torch.cuda.set_device(0)
    n = args.size
    lat = lcbp.Lattice(n, n, n, dtype=args.dtype)
    lat.set_ldg(0.01, 3.1, 0.01, 2 * math.pi / 32)
    lat.init_q(lcbp.BPII, 0.3, noise=1e-4, seed=20090119).init_f_equilibrium(1.0)
    ms = lat.profile_steps(args.steps)
    print({"size": n, "steps": args.steps, "kernel_ms": ms, "F": lat.free_energy()})


if __name__ == "__main__":
    main()
