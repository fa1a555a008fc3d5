"""Training data, training loop and judged inference for the learned surrogate.

Everything numerical runs in liblcbp (solver kernels, tensor-core network
kernels, loss and Adam); this module only orchestrates:

* ``generate``: plain FP32 runs of the thin-slab domain-growth problem
  (64 x 64 x 256, BPII seed for z < 32 inside an x-helix, tau = -0.5) at
  several chiralities; every ``every`` steps the state (Q, u) at t and
  Q(t + 10) are kept as a training pair.
* ``train``: Adam on random 64^3 crops (full x, y; a z-window) of those pairs;
  the loss is masked within the network's receptive field (10 sites) of the
  crop's z-faces, where the periodic padding of the crop is not physical.
* ``JudgedRun``: advances a lattice with the surrogate in segments of M calls
  (10 steps each).  After each segment the judge re-equilibrates f, runs 10
  plain steps from the surrogate state and compares the free energy with one
  surrogate call from the same state; a relative gap above ``tol`` switches
  the next segment to plain stepping.
"""

from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import lcbp

Q0 = 2 * np.pi / 16
A0 = 0.01
TAU_R = -0.5  # reduced temperature of the slab runs
K_STEPS = 10  # solver steps per surrogate call
RECEPTIVE = 10  # 10 convolutions of radius 1


def slab_lattice(kappa: float, seed: int = 20090119, shape=(64, 64, 256)) -> lcbp.Lattice:
    nx, ny, nz = shape
    lat = lcbp.Lattice(nx, ny, nz, dtype="f32")
    lat.set_ldg_kappa_tau(A0, Q0, kappa, TAU_R)
    lat.set_flow(2.0, 0.7, 0.3, True, lcbp.JACOBI)
    lat.init_q(lcbp.SLAB_BPII_IN_CHOL, 0.3, noise=1e-4, seed=seed, z0=nz // 8)
    lat.init_f_equilibrium(1.0)
    return lat


@dataclass
class Sample:
    q: np.ndarray  # [5, z, y, x] float32 at t
    u: np.ndarray  # [3, z, y, x]
    dq: np.ndarray  # Q(t + 10) - Q(t)
    kappa: float
    t: int


def generate(kappas, steps: int, every: int, seed: int = 20090119, shape=(64, 64, 256)):
    """Plain runs; returns the list of (state, 10-step change) samples."""
    out = []
    for i, kappa in enumerate(kappas):
        lat = slab_lattice(kappa, seed + i, shape)
        t = 0
        while t + K_STEPS <= steps:
            lat.step(every - K_STEPS if t else 0)
            t += every - K_STEPS if t else 0
            q0 = lat.read_q(dtype=np.float32)
            u0 = lat.read_u(dtype=np.float32)
            lat.step(K_STEPS)
            q1 = lat.read_q(dtype=np.float32)
            out.append(Sample(q0, u0, q1 - q0, float(kappa), t))
            t += K_STEPS
        lat.close()
    return out


def crop(s: Sample, z0: int, depth: int):
    nz = s.q.shape[1]
    idx = np.arange(z0, z0 + depth) % nz
    mask = np.ones((depth,) + s.q.shape[2:], dtype=np.float32)
    mask[:RECEPTIVE] = 0.0
    mask[depth - RECEPTIVE:] = 0.0
    return (np.ascontiguousarray(s.q[:, idx]), np.ascontiguousarray(s.u[:, idx]),
            np.ascontiguousarray(s.dq[:, idx]), mask)


@dataclass
class TrainLog:
    losses: list = field(default_factory=list)
    seconds: float = 0.0
    iters: int = 0


def train(samples, iters: int, lr: float = 1e-3, depth: int = 64, seed: int = 0, params=None,
          s_u: float = 1e-3, s_dq: float = 1e-2):
    """Adam on random crops; returns (parameter vector, TrainLog)."""
    rng = np.random.default_rng(seed)
    nx, ny = samples[0].q.shape[3], samples[0].q.shape[2]
    sur = lcbp.Surrogate(nx, ny, depth, training=True)
    sur.set_scales(s_u, s_dq)
    if params is None:
        params = init_params(rng)
    sur.set_params(params)
    log = TrainLog()
    t0 = time.perf_counter()
    for it in range(iters):
        s = samples[rng.integers(len(samples))]
        z0 = int(rng.integers(s.q.shape[1]))
        q, u, dq, mask = crop(s, z0, depth)
        lr_it = lr if it < iters // 2 else lr * 0.3
        log.losses.append(sur.train_step(q, u, s.kappa, TAU_R, dq, mask, lr=lr_it))
    log.seconds = time.perf_counter() - t0
    log.iters = iters
    p = sur.get_params()
    sur.close()
    return p, log


def init_params(rng, blocks: int = 4, width: int = 32):
    """He-normal weights; the last layer and the second conv of each block start
    small so the untrained network is close to persistence (dQ = 0)."""
    parts = []
    dims = [(10, width)] + [(width, width)] * (2 * blocks) + [(width, 5)]
    for i, (ci, co) in enumerate(dims):
        std = np.sqrt(2.0 / (27 * ci))
        if i == len(dims) - 1 or (i > 0 and i % 2 == 0):
            std *= 0.1
        parts += [rng.normal(0.0, std, size=27 * ci * co), np.zeros(co)]
    return np.concatenate(parts).astype(np.float32)


def evaluate(params, samples, depth: int = 64, s_u: float = 1e-3, s_dq: float = 1e-2):
    """Mean masked MSE of the 10-step change on the given samples, for the
    network and for persistence (dQ = 0, the method without the network)."""
    nx, ny = samples[0].q.shape[3], samples[0].q.shape[2]
    sur = lcbp.Surrogate(nx, ny, depth)
    sur.set_scales(s_u, s_dq)
    sur.set_params(params)
    err_net, err_zero = [], []
    for s in samples:
        q, u, dq, mask = crop(s, 0, depth)
        y = sur.forward(q, u, s.kappa, TAU_R) * s_dq
        w = mask[None]
        err_net.append(float((w * (y - dq) ** 2).sum() / (5 * w.sum())))
        err_zero.append(float((w * dq ** 2).sum() / (5 * w.sum())))
    sur.close()
    return float(np.mean(err_net)), float(np.mean(err_zero))


class JudgedRun:
    """Surrogate-accelerated time stepping with the plain solver as judge and fallback.

    Each segment of M calls starts from a device snapshot of (f, Q).  After the
    segment f is re-equilibrated and the judge compares one surrogate call
    with 10 plain steps from the same state; if the relative free-energy gap
    exceeds tol (or the state is no longer finite) the segment is rolled back
    and redone with plain steps.
    """

    def __init__(self, lat: lcbp.Lattice, params, kappa: float, M: int = 50, tol: float = 1e-3,
                 s_u: float = 1e-3, s_dq: float = 1e-2):
        import torch
        nx, ny, nz = lat.dims
        self.lat, self.kappa, self.M, self.tol, self.s_dq = lat, kappa, M, tol, s_dq
        self.sur = lcbp.Surrogate(nx, ny, nz)
        self.sur.set_scales(s_u, s_dq)
        self.sur.set_params(params)
        self.t = 0
        self.surrogate_calls = 0
        self.plain_steps = 0
        self.fallbacks = 0
        self.judge_gaps = []
        self._f = torch.empty((15, nz, ny, nx), dtype=torch.float32, device="cuda")
        self._q = torch.empty((5, nz, ny, nx), dtype=torch.float32, device="cuda")

    def _log(self, log, log_every, next_log):
        while next_log is not None and self.t >= next_log:
            log.append((next_log, self.lat.free_energy()))
            next_log += log_every
        return next_log

    def advance(self, t_end: int, log_every: int | None = None, log=None):
        """Advance to t_end; optionally record (t, F) at multiples of log_every
        (taken at the first segment boundary at or after each multiple)."""
        next_log = (self.t // log_every + 1) * log_every if log_every else None
        while self.t < t_end:
            seg = min(self.M * K_STEPS, t_end - self.t)
            calls = seg // K_STEPS
            if calls == 0:
                self.lat.step(seg)
                self.t += seg
                self.plain_steps += seg
                next_log = self._log(log, log_every, next_log)
                continue
            t0 = self.t
            self.lat.read_f(out=self._f)
            self.lat.read_q(out=self._q)
            ok = True
            try:
                self.sur.step(self.lat, self.kappa, TAU_R, calls)
                self.lat.reequilibrate_f()
                ok = self._judge()
            except lcbp.LcbpError:
                ok = False
            if ok:
                self.surrogate_calls += calls
                self.t = t0 + calls * K_STEPS + K_STEPS  # the judge's plain steps advance time too
                self.plain_steps += K_STEPS
            else:
                self.fallbacks += 1
                self.lat.set_f(self._f)
                self.lat.set_q(self._q)
                self.lat.step(calls * K_STEPS)
                self.t = t0 + calls * K_STEPS
                self.plain_steps += calls * K_STEPS
            next_log = self._log(log, log_every, next_log)

    def _judge(self) -> bool:
        """One surrogate call vs 10 plain steps from the same state."""
        q = self.lat.read_q(dtype=np.float32)
        u = self.lat.read_u(dtype=np.float32)
        if not (np.isfinite(q).all() and np.isfinite(u).all()):
            return False
        y = self.sur.forward(q, u, self.kappa, TAU_R)
        self.lat.step(K_STEPS)
        F_plain = self.lat.free_energy()
        F_pred = free_energy_of(self.lat.dims, self.kappa, q + self.s_dq * y)
        gap = abs(F_pred - F_plain) / abs(F_plain)
        self.judge_gaps.append(gap)
        return bool(np.isfinite(gap) and gap <= self.tol)

    def close(self):
        self.sur.close()


def free_energy_of(dims, kappa: float, q5) -> float:
    """F_h of an arbitrary Q on a scratch lattice of the same size (slab parameters)."""
    scratch = _SCRATCH.get(dims)
    if scratch is None:
        _SCRATCH.clear()
        scratch = _SCRATCH[dims] = lcbp.Lattice(*dims, dtype="f32")
    scratch.set_ldg_kappa_tau(A0, Q0, kappa, TAU_R)
    scratch.set_q(q5)
    return scratch.free_energy()


_SCRATCH: dict = {}


def time_call(shape=(64, 64, 256), reps: int = 20):
    """Device time of one surrogate call and of 10 plain steps on the slab (ms)."""
    import torch
    lat = slab_lattice(1.0, shape=shape)
    lat.step(20)
    lat.synchronize()
    sur = lcbp.Surrogate(*shape)
    sur.set_params(init_params(np.random.default_rng(0)))
    sur.step(lat, 1.0, TAU_R, 2)  # warm-up
    t0 = time.perf_counter()
    sur.step(lat, 1.0, TAU_R, reps)
    t_sur = (time.perf_counter() - t0) / reps * 1e3
    lat.reequilibrate_f().step(20)
    lat.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(lat._stream)
    lat.step(10 * reps)
    e1.record(lat._stream)
    e1.synchronize()
    t_plain = e0.elapsed_time(e1) / reps
    sur.close()
    lat.close()
    return t_sur, t_plain


def main():
    import argparse
    import json
    import torch
    ap = argparse.ArgumentParser(description="train the surrogate on slab runs and judge it against the solver")
    ap.add_argument("--data-steps", type=int, default=6000)
    ap.add_argument("--every", type=int, default=100)
    ap.add_argument("--iters", type=int, default=1500)
    ap.add_argument("--run-steps", type=int, default=20000)
    ap.add_argument("--kappa", type=float, default=1.0)
    args = ap.parse_args()
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    data = generate([0.5, 1.0, 2.0], args.data_steps, args.every)
    held = generate([1.5], args.data_steps, args.every * 5, seed=7)
    t_gen = time.perf_counter() - t0
    import sys
    params, log = train(data, args.iters)
    print(json.dumps({"train_s": log.seconds, "loss_first": float(np.mean(log.losses[:20])),
                      "loss_last": float(np.mean(log.losses[-20:]))}), file=sys.stderr, flush=True)
    mse_net, mse_zero = evaluate(params, held)
    print(json.dumps({"held_out_mse": [mse_net, mse_zero]}), file=sys.stderr, flush=True)
    t_sur, t_plain = time_call()
    print(json.dumps({"call_ms": [t_sur, t_plain]}), file=sys.stderr, flush=True)
    # time to solution: plain vs judged surrogate run from the same initial state
    plain = slab_lattice(args.kappa)
    F_plain = []
    tp0 = time.perf_counter()
    for t in range(100, args.run_steps + 1, 100):
        plain.step(100)
        F_plain.append((t, plain.free_energy()))
    plain.synchronize()
    t_plain_run = time.perf_counter() - tp0
    hyb = slab_lattice(args.kappa)
    run = JudgedRun(hyb, params, args.kappa)
    F_hyb = []
    th0 = time.perf_counter()
    run.advance(args.run_steps, log_every=100, log=F_hyb)
    hyb.synchronize()
    t_hyb_run = time.perf_counter() - th0
    fp = dict(F_plain)
    errs = [abs(F - fp[t]) / abs(fp[t]) for t, F in F_hyb if t in fp]
    print(json.dumps({
        "data": {"samples": len(data), "held_out": len(held), "seconds": t_gen},
        "train": {"iters": log.iters, "seconds": log.seconds, "ms_per_iter": 1e3 * log.seconds / log.iters,
                  "loss_first": float(np.mean(log.losses[:20])), "loss_last": float(np.mean(log.losses[-20:]))},
        "held_out_mse": {"network": mse_net, "persistence": mse_zero},
        "call_ms": {"surrogate_10_steps": t_sur, "plain_10_steps": t_plain},
        "run": {"steps": args.run_steps, "kappa": args.kappa, "plain_s": t_plain_run, "surrogate_s": t_hyb_run,
                "surrogate_calls": run.surrogate_calls, "plain_steps": run.plain_steps,
                "fallbacks": run.fallbacks, "max_rel_F_error": max(errs) if errs else None,
                "judge_gap_median": float(np.median(run.judge_gaps)) if run.judge_gaps else None,
                "final_F": {"plain": F_plain[-1][1], "surrogate": F_hyb[-1][1] if F_hyb else None}},
    }))


if __name__ == "__main__":
    main()
