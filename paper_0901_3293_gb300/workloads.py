"""Ready-made workloads of the benchmark and the profiler.

The chirality/temperature sweep of 48 replicas (24 x 32^3 and 24 x 48^3) as
one batch: per-replica kappa ~ U[0.3, 2] and tau ~ U[-1, 0.5], which the
library turns into the Landau-de Gennes gamma and K of the one-constant energy
(lcbp_params_kappa_tau; A0 = 0.01, pitch 16), and initial states BPII, a
cholesteric along z, or isotropic noise.
"""

from __future__ import annotations

import math

from . import lcbp, synth


def replica_sweep_batch(replicas: int = 48, seed: int = synth.BASE_SEED, dtype: str = "f32") -> "lcbp.Batch":
    """The sweep as an lcbp.Batch with Q set and f at equilibrium (not yet stepped)."""
    sweep = synth.replica_sweep(replicas, seed)
    q0 = 2 * math.pi / 16
    params = [lcbp.params_kappa_tau(0.01, q0, sw["kappa"], sw["tau"], tau_f=2.0, xi=0.7, Gamma=0.3) for sw in sweep]
    batch = lcbp.Batch([sw["dims"] for sw in sweep], params, dtype=dtype)
    for r, sw in enumerate(sweep):
        kind = (lcbp.BPII, lcbp.CHOL_Z, lcbp.ISO_NOISE)[sw["kind"]]
        batch.init_q(r, kind, 0.3 if sw["kind"] == 0 else 0.4, noise=1e-2, seed=sw["seed"])
    return batch.init_f_equilibrium(1.0)
