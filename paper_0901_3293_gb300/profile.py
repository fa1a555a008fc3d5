"""Run a few coupled steps on an L^3 BPII lattice, for profilers.

    python -m paper_0901_3293_gb300.profile --size 128 --steps 4 [--dtype f32] [--walls]
    python -m paper_0901_3293_gb300.profile --conv --dims 64 64 256 --steps 3
    python -m paper_0901_3293_gb300.profile --texture --dims 256 256 256 --steps 3
    python -m paper_0901_3293_gb300.profile --batch --steps 4
    python -m paper_0901_3293_gb300.profile --diag --size 160 --steps 3
    python -m paper_0901_3293_gb300.profile --train --dims 64 64 64 --steps 10

Each step launches the step kernels once (no CUDA graph), so a profiler can
select them by name and launch index.  --conv instead runs surrogate calls
(ten tensor-core convolutions each) on a lattice of the given dims.  --walls
puts walls in z with a planar anchored Q (S (x x - I/3), S = 0.3).  --texture
renders the polarised-light texture of a BPII lattice of the given dims
(pitch 32) `steps` times.  --batch steps the 48-replica chirality/temperature
sweep (24 x 32^3 + 24 x 48^3) in one batch: ten steps (kernel selection and
tuning), then `steps` single steps inside the NVTX range "timed", so that a
profiler can take exactly those launches (--nvtx --nvtx-include "timed/").
--diag runs the FP64 diagnostics (free energy, mass and momentum, defect
fraction: one pass) `steps` times on the L^3 lattice after one step.
--train runs `steps` surrogate training steps (forward, backward, weight
gradients on the tensor cores, masked loss and Adam) on a random crop of the
given dims, after three untimed ones, inside the NVTX range "timed".
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
    ap.add_argument("--conv", action="store_true")
    ap.add_argument("--dims", type=int, nargs=3, default=[64, 64, 256])
    ap.add_argument("--walls", action="store_true")
    ap.add_argument("--texture", action="store_true")
    ap.add_argument("--batch", action="store_true")
    ap.add_argument("--diag", action="store_true")
    ap.add_argument("--train", action="store_true")
    args = ap.parse_args()
    build.build()
    torch.cuda.set_device(0)
    if args.conv:
        import time

        import numpy as np
        nx, ny, nz = args.dims
        lat = lcbp.Lattice(nx, ny, nz)
        lat.init_q(lcbp.BPII, 0.3, noise=1e-4, seed=1).init_f_equilibrium(1.0)
        sur = lcbp.Surrogate(nx, ny, nz)
        rng = np.random.default_rng(0)
        sur.set_params((rng.normal(size=sur.count) * 0.02).astype(np.float32))
        t0 = time.perf_counter()
        sur.step(lat, 1.0, -0.5, args.steps)
        print({"dims": args.dims, "calls": args.steps, "ms_per_call": 1e3 * (time.perf_counter() - t0) / args.steps})
        return
    if args.train:
        import time

        import numpy as np
        nx, ny, nz = args.dims
        sur = lcbp.Surrogate(nx, ny, nz, training=True)
        rng = np.random.default_rng(0)
        sur.set_params((rng.normal(size=sur.count) * 0.02).astype(np.float32))
        dev = dict(device="cuda", dtype=torch.float32)
        q = torch.from_numpy(rng.uniform(-0.3, 0.3, (5, nz, ny, nx)).astype(np.float32)).to(**dev)
        u = torch.from_numpy(rng.uniform(-1e-3, 1e-3, (3, nz, ny, nx)).astype(np.float32)).to(**dev)
        r = torch.from_numpy(rng.uniform(-1e-4, 1e-4, (5, nz, ny, nx)).astype(np.float32)).to(**dev)
        dq = torch.from_numpy(rng.uniform(-1e-3, 1e-3, (5, nz, ny, nx)).astype(np.float32)).to(**dev)
        mask = torch.ones((nz, ny, nx), **dev)
        for _ in range(3):
            sur.train_step(q, u, r, 1.0, -0.5, dq, mask)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed")
        t0 = time.perf_counter()
        for _ in range(args.steps):
            loss = sur.train_step(q, u, r, 1.0, -0.5, dq, mask)
        dt = time.perf_counter() - t0
        torch.cuda.nvtx.range_pop()
        print({"dims": args.dims, "train_steps": args.steps, "ms_per_step": 1e3 * dt / args.steps, "loss": loss})
        sur.close()
        return
    if args.batch:
        import time

        from . import workloads
        batch = workloads.replica_sweep_batch(48, dtype=args.dtype)
        batch.step(10)
        batch.synchronize()
        torch.cuda.nvtx.range_push("timed")
        t0 = time.perf_counter()
        for _ in range(args.steps):
            batch.step(1)
        batch.synchronize()
        dt = time.perf_counter() - t0
        torch.cuda.nvtx.range_pop()
        print({"replicas": 48, "steps": args.steps, "path": batch.path(), "ms_per_step": 1e3 * dt / args.steps})
        return
    if args.texture:
        import time
        nx, ny, nz = args.dims
        lat = lcbp.Lattice(nx, ny, nz, dtype=args.dtype)
        lat.set_ldg(0.01, 3.1, 0.01, 2 * math.pi / 32)
        lat.init_q(lcbp.BPII, 0.3, noise=1e-4, seed=20090119)
        lat.texture()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            img = lat.texture()
        print({"dims": args.dims, "images": args.steps, "ms_per_image": 1e3 * (time.perf_counter() - t0) / args.steps,
               "mean": float(img.mean())})
        return
    n = args.size
    lat = lcbp.Lattice(n, n, n, dtype=args.dtype)
    lat.set_ldg(0.01, 3.1, 0.01, 2 * math.pi / 32)
    lat.init_q(lcbp.BPII, 0.3, noise=1e-4, seed=20090119).init_f_equilibrium(1.0)
    if args.walls:
        lat.set_walls(True, (0.2, 0.0, 0.0, -0.1, 0.0))
    if args.diag:
        import time
        lat.step(1)
        lat.free_energy()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            F = lat.free_energy()
        dt = time.perf_counter() - t0
        print({"size": n, "calls": args.steps, "ms_per_call": 1e3 * dt / args.steps, "F": F,
               "defects": lat.defect_fraction(0.19)})
        return
    ms = lat.profile_steps(args.steps)
    print({"size": n, "steps": args.steps, "walls": args.walls, "kernel_ms": ms, "F": lat.free_energy()})


if __name__ == "__main__":
    main()
