"""Training data, training loop and judged inference for the learned surrogate.

Everything numerical runs in liblcbp (solver kernels, tensor-core network
kernels, loss and Adam, the judged run); this module only orchestrates:

* ``generate``: plain FP32 runs of the thin-slab domain-growth problem
  (64 x 64 x 256, BPII seed for z < 32 inside an x-helix, tau = -0.5) at
  several chiralities; every ``every`` steps the state (Q, u) at t and
  Q(t + k) are kept as a training pair (k solver steps per surrogate call).
* ``train``: Adam on random 64^3 crops (full x, y; a z-window) of those pairs;
  the loss is masked within the network's receptive field (10 sites) of the
  crop's z-faces, where the periodic padding of the crop is not physical.
* ``JudgedRun``: the library's judged run (lcbp_judge_*): segments of M
  calls, each judged against k plain steps from the same re-equilibrated
  state by the relative free-energy gap, rolled back and redone plainly when
  the gap exceeds ``tol``.
* ``main``: train at a given k, write the weights file, and compare the
  judged runs of the trained network and of the zero network (k plain Euler
  steps of the rate per call) with the plain solver on the slab workload at
  several chiralities, logging F and the defect fraction every 100 steps.

The surrogate predicts a correction to k explicit Euler steps of the exact
FP32 Beris-Edwards rate R(Q, u): Q(t + k) = Q + k R + s_dq * net(Q, u, kappa, tau, R).
"""

from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import lcbp, synth

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
    r: np.ndarray  # Beris-Edwards rate at t
    dq: np.ndarray  # Q(t + 10) - Q(t)
    kappa: float
    t: int


def generate(kappas, steps: int, every: int, t_min: int = 0, seed: int = 20090119, shape=(64, 64, 256),
             k: int = K_STEPS):
    """Plain runs; a sample (state, rate, k-step change) every `every` steps from t_min."""
    out = []
    for i, kappa in enumerate(kappas):
        lat = slab_lattice(kappa, seed + i, shape)
        lat.step(t_min)
        t = t_min
        while t + k <= steps:
            q0 = lat.read_q(dtype=np.float32)
            u0 = lat.read_u(dtype=np.float32)
            r0 = lat.read_rate(dtype=np.float32)
            lat.step(k)
            q1 = lat.read_q(dtype=np.float32)
            out.append(Sample(q0, u0, r0, q1 - q0, float(kappa), t))
            lat.step(every - k)
            t += every
        lat.close()
    return out


def crop(s: Sample, z0: int, depth: int):
    nz = s.q.shape[1]
    idx = np.arange(z0, z0 + depth) % nz
    mask = np.ones((depth,) + s.q.shape[2:], dtype=np.float32)
    if depth < nz:
        mask[:RECEPTIVE] = 0.0
        mask[depth - RECEPTIVE:] = 0.0
    return (np.ascontiguousarray(s.q[:, idx]), np.ascontiguousarray(s.u[:, idx]),
            np.ascontiguousarray(s.r[:, idx]), np.ascontiguousarray(s.dq[:, idx]), mask)


def rotate_z(q5, u3, k: int):
    """Fields rotated by k quarter turns about z (square x-y planes): F'(r) =
    R F(R^-1 r) R^T for the tensors, R u(R^-1 r) for the velocity, with R
    taking x to y.  The equations of motion are invariant under proper
    rotations of the cubic lattice, so a rotated trajectory is a trajectory."""
    for _ in range(k % 4):
        n = q5.shape[-1]
        yp, xp = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        src_y, src_x = (-xp) % n, yp

        def move(a):
            return a[..., src_y, src_x]

        q5 = np.stack([move(q5[3]), -move(q5[1]), -move(q5[4]), move(q5[0]), move(q5[2])])
        if u3 is not None:
            u3 = np.stack([-move(u3[1]), move(u3[0]), move(u3[2])])
    return q5, u3


@dataclass
class TrainLog:
    losses: list = field(default_factory=list)
    seconds: float = 0.0
    iters: int = 0


# input scales of u and of the rate R, output scale of the correction: chosen so
# that the inputs R / s_r and the target (dq - 10 R) / s_dq are O(1) on the slab
# (the BF16 activations then resolve them)
S_U, S_R, S_DQ = 1e-3, 1e-4, 3e-6


def rotate_z_device(q5, u3, turns: int):
    """rotate_z on CUDA tensors ([C, z, y, x], square x-y planes): the same
    gather and sign changes, done where the training crops live."""
    import torch
    for _ in range(turns % 4):
        n = q5.shape[-1]
        yp, xp = torch.meshgrid(torch.arange(n, device=q5.device), torch.arange(n, device=q5.device), indexing="ij")
        src_y, src_x = (-xp) % n, yp

        def move(a):
            return a[..., src_y, src_x]

        q5 = torch.stack([move(q5[3]), -move(q5[1]), -move(q5[4]), move(q5[0]), move(q5[2])])
        if u3 is not None:
            u3 = torch.stack([-move(u3[1]), move(u3[0]), move(u3[2])])
    return q5, u3


def train(samples, iters: int, lr: float = 1e-3, depth: int = 64, seed: int = 0, params=None,
          augment: bool = True, k: int = K_STEPS):
    """Adam on random crops (rotated by a random quarter turn about z when
    `augment`); returns (parameter vector, TrainLog).  The samples are moved
    to the device once; crops and rotations are gathers there."""
    import torch
    rng = np.random.default_rng(seed)
    nx, ny = samples[0].q.shape[3], samples[0].q.shape[2]
    sur = lcbp.Surrogate(nx, ny, depth, training=True)
    sur.set_scales(S_U, S_R, S_DQ).set_steps(k)
    if params is None:
        params = init_params(rng)
    sur.set_params(params)
    dev = [tuple(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (sm.q, sm.u, sm.r, sm.dq))
           for sm in samples]
    nz = samples[0].q.shape[1]
    mask = torch.ones((depth, ny, nx), dtype=torch.float32, device="cuda")
    if depth < nz:
        mask[:RECEPTIVE] = 0.0
        mask[depth - RECEPTIVE:] = 0.0
    log = TrainLog()
    t0 = time.perf_counter()
    for it in range(iters):
        j = int(rng.integers(len(samples)))
        z0 = int(rng.integers(nz))
        idx = torch.arange(z0, z0 + depth, device="cuda") % nz
        q, u, r, dq = (a.index_select(1, idx) for a in dev[j])
        if augment and nx == ny:
            turns = int(rng.integers(4))
            q, u = rotate_z_device(q, u, turns)
            r, _ = rotate_z_device(r, None, turns)
            dq, _ = rotate_z_device(dq, None, turns)
        q, u, r, dq = (a.contiguous() for a in (q, u, r, dq))
        lr_it = lr if it < iters // 2 else (lr * 0.3 if it < 3 * iters // 4 else lr * 0.1)
        log.losses.append(sur.train_step(q, u, r, samples[j].kappa, TAU_R, dq, mask, lr=lr_it))
    log.seconds = time.perf_counter() - t0
    log.iters = iters
    p = sur.get_params()
    sur.close()
    del dev
    return p, log


def init_params(rng, blocks: int = 4, width: int = 32):
    """He-normal weights; the last layer and the second conv of each block start
    small so the untrained network is close to persistence (dQ = 0)."""
    parts = []
    dims = [(15, width)] + [(width, width)] * (2 * blocks) + [(width, 5)]
    for i, (ci, co) in enumerate(dims):
        std = np.sqrt(2.0 / (27 * ci))
        if i == len(dims) - 1 or (i > 0 and i % 2 == 0):
            std *= 0.1
        parts += [rng.normal(0.0, std, size=27 * ci * co), np.zeros(co)]
    return np.concatenate(parts).astype(np.float32)


def evaluate(params, samples, depth: int = 64, k: int = K_STEPS):
    """Mean masked MSE of the predicted k-step change on the given samples for
    the network, for k Euler steps of the rate (the integrator the network
    corrects) and for persistence (dQ = 0)."""
    nx, ny = samples[0].q.shape[3], samples[0].q.shape[2]
    sur = lcbp.Surrogate(nx, ny, depth)
    sur.set_scales(S_U, S_R, S_DQ).set_steps(k)
    sur.set_params(params)
    err = {"network": [], "euler": [], "persistence": []}
    for s in samples:
        q, u, r, dq, mask = crop(s, 0, depth)
        pred = k * r + S_DQ * sur.forward(q, u, r, s.kappa, TAU_R)
        w = mask[None]
        den = 5 * w.sum()
        err["network"].append(float((w * (pred - dq) ** 2).sum() / den))
        err["euler"].append(float((w * (k * r - dq) ** 2).sum() / den))
        err["persistence"].append(float((w * dq ** 2).sum() / den))
    sur.close()
    return {k: float(np.mean(v)) for k, v in err.items()}


class JudgedRun:
    """Surrogate-accelerated time stepping with the plain solver as judge and
    fallback: the library's judged run (lcbp_judge_*) on a lattice, with this
    module's network scales.  Segments of M calls are each judged against ten
    plain steps; a relative free-energy gap above tol (or a max |dQ| above
    tol_q, if given) rolls the segment back and redoes it with plain steps."""

    def __init__(self, lat: lcbp.Lattice, params, kappa: float, M: int = 49, tol: float = 1e-3,
                 tol_q: float = 0.0, weights: str | None = None, k: int = K_STEPS, warmup: int = 0):
        nx, ny, nz = lat.dims
        self.sur = lcbp.Surrogate(nx, ny, nz)
        if weights is not None:
            self.sur.load(weights)
        else:
            self.sur.set_scales(S_U, S_R, S_DQ).set_steps(k)
            self.sur.set_params(params)
        self.judge = lcbp.Judge(lat, self.sur, kappa, TAU_R, calls_per_segment=M, tol_F=tol, tol_Q=tol_q,
                                warmup_steps=warmup)

    def advance(self, t_end: int, log_every: int = 0):
        """Advance to t_end; with log_every > 0 returns (t, F, defect fraction) at its multiples."""
        return self.judge.advance(t_end, log_every)

    def stats(self) -> dict:
        return self.judge.stats()

    def close(self):
        self.judge.close()
        self.sur.close()


def time_call(shape=(64, 64, 256), reps: int = 20, k: int = K_STEPS):
    """Device time of one surrogate call and of k plain steps on the slab (ms)."""
    import torch
    lat = slab_lattice(1.0, shape=shape)
    lat.step(20)
    lat.synchronize()
    sur = lcbp.Surrogate(*shape)
    sur.set_scales(S_U, S_R, S_DQ).set_steps(k)
    sur.set_params(init_params(np.random.default_rng(0)))
    sur.step(lat, 1.0, TAU_R, 2)  # warm-up
    t0 = time.perf_counter()
    sur.step(lat, 1.0, TAU_R, reps)
    t_sur = (time.perf_counter() - t0) / reps * 1e3
    lat.reequilibrate_f().step(20)
    lat.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(lat._stream)
    lat.step(k * reps)
    e1.record(lat._stream)
    e1.synchronize()
    t_plain = e0.elapsed_time(e1) / reps
    sur.close()
    lat.close()
    return t_sur, t_plain


def final_fields(lat: lcbp.Lattice, fields: dict | None) -> None:
    """Q and u of the lattice's current state into ``fields`` (if given)."""
    if fields is not None:
        fields["q"] = lat.read_q(np.float64)
        fields["u"] = lat.read_u(np.float64)


def field_errors(a: dict, b: dict) -> dict:
    """max |Delta Q| over sites and components, and the r.m.s. |Delta u| over sites."""
    du = a["u"] - b["u"]
    return {"max_abs_dQ": float(np.abs(a["q"] - b["q"]).max()),
            "rms_du": float(np.sqrt(np.mean(np.sum(du * du, axis=0)))),
            "rms_u": float(np.sqrt(np.mean(np.sum(b["u"] * b["u"], axis=0))))}


def plain_log(kappa: float, steps: int, log_every: int = 100, threshold: float = 0.19, fields: dict | None = None,
              perturb: tuple | None = None):
    """The slab workload run plainly: (t, F, defect fraction) every log_every steps, and seconds.
    perturb = (t_p, eps, seed): at step t_p (a multiple of log_every) add
    uniform noise of amplitude eps to every Q component (the solver's own
    sensitivity, as a yardstick for the judged run's field errors)."""
    lat = slab_lattice(kappa)
    rows = []
    t0 = time.perf_counter()
    for t in range(log_every, steps + 1, log_every):
        lat.step(log_every)
        if perturb is not None and t == perturb[0]:
            q = lat.read_q(np.float64)
            lat.set_q(q + synth.random_q5(q.shape[1:], perturb[1], perturb[2]))
        rows.append((t, lat.free_energy(), lat.defect_fraction(threshold)))
    lat.synchronize()
    secs = time.perf_counter() - t0
    final_fields(lat, fields)
    lat.close()
    return rows, secs


def judged_log(params, kappa: float, steps: int, k: int, M: int, tol: float, log_every: int = 100,
               weights: str | None = None, warmup: int = 0, fields: dict | None = None, tol_q: float = 0.0):
    """The judged run on the slab: its log, statistics and seconds."""
    hyb = slab_lattice(kappa)
    run = JudgedRun(hyb, params, kappa, M=M, tol=tol, k=k, weights=weights, warmup=warmup, tol_q=tol_q)
    t0 = time.perf_counter()
    ts, Fs, Ds = run.advance(steps, log_every)
    hyb.synchronize()
    secs = time.perf_counter() - t0
    st = run.stats()
    final_fields(hyb, fields)
    run.close()
    hyb.close()
    return list(zip(ts.tolist(), Fs.tolist(), Ds.tolist())), st, secs


def field_track(params, kappa: float, steps: int, k: int, M: int, tol: float, warmup: int, tol_q: float = 0.0):
    """max |Delta Q| and r.m.s. |Delta u| of the judged run against the plain run
    at every segment boundary (t = warmup + i (M + 1) k, where the judged run's
    state is its own), with the plain run's r.m.s. |u|: (t, dQ, du, u) rows.
    Advancing the judge to segment boundaries leaves its segmentation as in
    one call."""
    plain = slab_lattice(kappa)
    hyb = slab_lattice(kappa)
    run = JudgedRun(hyb, params, kappa, M=M, tol=tol, k=k, warmup=warmup, tol_q=tol_q)
    rows, t = [], 0
    seg = (M + 1) * k
    stops = [warmup] + list(range(warmup + seg, steps, seg)) + [steps]
    for t_next in stops:
        if t_next <= t:
            continue
        run.advance(t_next)
        plain.step(t_next - t)
        t = t_next
        a, b = {}, {}
        final_fields(hyb, a)
        final_fields(plain, b)
        e = field_errors(a, b)
        rows.append((t, e["max_abs_dQ"], e["rms_du"], e["rms_u"]))
    run.close()
    hyb.close()
    plain.close()
    return rows


def main():
    import argparse
    import json
    import sys
    import torch
    ap = argparse.ArgumentParser(description="train the surrogate on slab runs and judge it against the solver")
    ap.add_argument("--k", type=int, default=K_STEPS, help="solver steps per surrogate call")
    ap.add_argument("--data-steps", type=int, default=12000)
    ap.add_argument("--every", type=int, default=400)
    ap.add_argument("--t-min", type=int, default=500)
    ap.add_argument("--iters", type=int, default=2000)
    ap.add_argument("--train-kappas", type=int, default=6, help="training chiralities, evenly in [0.5, 2]")
    ap.add_argument("--run-steps", type=int, default=20000)
    ap.add_argument("--kappas", type=float, nargs="+", default=[0.5, 1.0, 2.0], help="chiralities of the judged runs")
    ap.add_argument("--M", type=int, default=49, help="surrogate calls per judged segment")
    ap.add_argument("--tol", type=float, default=1e-3)
    ap.add_argument("--tol-q", type=float, default=0.0, help="judge bound on max |dQ| of one call (0: off)")
    ap.add_argument("--warmup", type=int, default=1000, help="plain steps before the first surrogate segment")
    ap.add_argument("--out", default=None, help="write the trained weights file here")
    ap.add_argument("--weights", default=None, help="skip training: judge this weights file")
    ap.add_argument("--init-weights", default=None, help="start the training from this weights file")
    ap.add_argument("--lr", type=float, default=1e-3, help="Adam learning rate (0.3x after half, 0.1x after 3/4)")
    ap.add_argument("--log-out", default=None, help="write the per-100-step logs here (JSON lines)")
    ap.add_argument("--s-r", type=float, default=None, help="input scale of the rate R")
    ap.add_argument("--s-dq", type=float, default=None, help="output scale of the correction")
    args = ap.parse_args()
    global S_R, S_DQ
    S_R = args.s_r if args.s_r is not None else S_R
    S_DQ = args.s_dq if args.s_dq is not None else S_DQ
    torch.cuda.set_device(0)
    k = args.k

    def note(d):
        print(json.dumps(d), file=sys.stderr, flush=True)

    t0 = time.perf_counter()
    held = generate([1.5], args.data_steps, args.every * 4, t_min=args.t_min, seed=7, k=k)
    if args.weights:
        sur = lcbp.Surrogate(held[0].q.shape[3], held[0].q.shape[2], 8).load(args.weights)
        params = sur.get_params()
        if sur.steps() != k:
            raise SystemExit(f"{args.weights} was trained for k = {sur.steps()}, not {k}")
        sur.close()
        log, n_data = TrainLog(), 0
        note({"k": k, "weights": args.weights})
    else:
        data = generate(list(np.linspace(0.5, 2.0, args.train_kappas)), args.data_steps, args.every,
                        t_min=args.t_min, k=k)
        n_data = len(data)
        note({"k": k, "samples": n_data, "held_out": len(held), "gen_s": time.perf_counter() - t0})
        init = None
        if args.init_weights:
            sur0 = lcbp.Surrogate(data[0].q.shape[3], data[0].q.shape[2], 8).load(args.init_weights)
            if sur0.steps() != k:
                raise SystemExit(f"{args.init_weights} was trained for k = {sur0.steps()}, not {k}")
            init = sur0.get_params()
            sur0.close()
        params, log = train(data, args.iters, lr=args.lr, k=k, params=init)
        del data
        note({"train_s": log.seconds, "loss_first": float(np.mean(log.losses[:20])),
              "loss_last": float(np.mean(log.losses[-20:]))})
    t_gen = time.perf_counter() - t0 - log.seconds
    mse = evaluate(params, held, depth=held[0].q.shape[1], k=k)
    note({"held_out_mse": mse})
    if args.out:
        nx, ny = held[0].q.shape[3], held[0].q.shape[2]
        sur = lcbp.Surrogate(nx, ny, 8)
        sur.set_scales(S_U, S_R, S_DQ).set_steps(k).set_params(params)
        sur.save(args.out)
        sur.close()
    t_sur, t_plain = time_call(k=k)
    note({"call_ms": [t_sur, t_plain]})
    runs = {}
    logf = open(args.log_out, "w") if args.log_out else None
    for kappa in args.kappas:
        plain_fields = {}
        rows, t_pl = plain_log(kappa, args.run_steps, fields=plain_fields)
        F_plain = {t: F for t, F, _ in rows}
        F_scale = max(abs(F) for _, F, _ in rows)
        out = {"plain_s": t_pl, "final_F": rows[-1][1], "final_defect_fraction": rows[-1][2], "F_scale": F_scale}
        # field errors of the trained network's judged run along the trajectory
        out["judged_network_fields_along_run"] = [
            {"t": t, "max_abs_dQ": dq, "rms_du": du, "rms_u_plain": uu}
            for t, dq, du, uu in field_track(params, kappa, args.run_steps, k, args.M, args.tol, args.warmup,
                                             args.tol_q)]
        # the plain solver's own sensitivity: Q perturbed by 1e-7 after the warm-up
        pert_fields = {}
        prow, _ = plain_log(kappa, args.run_steps, fields=pert_fields, perturb=(args.warmup, 1e-7, 99))
        out["plain_perturbed_1e-7"] = {
            "max_rel_F_error": max(abs(F - F_plain[t]) / abs(F_plain[t]) for t, F, _ in prow),
            "final_fields_vs_plain": field_errors(pert_fields, plain_fields)}
        # judged (tol) and accept-all (equal cost: every segment kept), trained and zero network
        logged = {}
        for mode, tol in (("judged", args.tol), ("accept_all", 1e30)):
            for name, p in (("network", params), ("zero_network", np.zeros_like(params))):
                jf = {}
                jrows, st, secs = judged_log(p, kappa, args.run_steps, k, args.M, tol, warmup=args.warmup, fields=jf,
                                             tol_q=args.tol_q if mode == "judged" else 0.0)
                errs = [abs(F - F_plain[t]) / abs(F_plain[t]) for t, F, _ in jrows]
                errs_s = [abs(F - F_plain[t]) / F_scale for t, F, _ in jrows]
                out[mode + "_" + name] = {"seconds": secs, "speedup_vs_plain": t_pl / secs, "logged": len(jrows),
                                          "max_rel_F_error": max(errs), "mean_rel_F_error": float(np.mean(errs)),
                                          "max_F_error_of_scale": max(errs_s),
                                          "final_fields_vs_plain": field_errors(jf, plain_fields), **st}
                if mode == "judged":
                    logged[name] = {t: (F, D, e) for (t, F, D), e in zip(jrows, errs)}
        if logf:
            # one line per logged step: the plain run, and the judged runs of the
            # trained and the zero network with their relative F error
            g7 = lambda v: float("%.7g" % v)  # noqa: E731  (seven significant digits in the log)
            for t, F, D in rows:
                line = {"kappa": kappa, "k": k, "t": t, "F_plain": g7(F), "defect_plain": g7(D)}
                for name, key in (("network", "judged"), ("zero_network", "judged_zero")):
                    Fj, Dj, e = logged[name][t]
                    line.update({"F_" + key: g7(Fj), "defect_" + key: g7(Dj), "rel_F_err_" + key: float("%.3g" % e)})
                logf.write(json.dumps(line) + "\n")
        runs[str(kappa)] = out
        note({"kappa": kappa, **out})
    if logf:
        logf.close()
    print(json.dumps({
        "k": k,
        "data": {"samples": n_data, "seconds": t_gen},
        "train": {"iters": log.iters, "seconds": log.seconds,
                  "ms_per_iter": 1e3 * log.seconds / log.iters if log.iters else None,
                  "loss_first": float(np.mean(log.losses[:20])) if log.losses else None,
                  "loss_last": float(np.mean(log.losses[-20:])) if log.losses else None,
                  "weights": args.weights},
        "held_out_mse": mse,
        "call_ms": {"surrogate_call": t_sur, "plain_k_steps": t_plain},
        "judged_runs": {"steps": args.run_steps, "M": args.M, "tol": args.tol, "tol_q": args.tol_q,
                        "warmup": args.warmup,
                        "by_kappa": runs},
    }))


if __name__ == "__main__":
    main()
