"""Training protocol of the h-predictor: the network is trained by the
library's own training kernels on the h trajectories that the plain solver
itself generates, then frozen.

Training runs: the 16^3 jittered lattice with variable h (M4, eta 1.2, at
rest, relaxing under its own pressure) and the 64^3 Sedov blast (Wendland C2,
eta 1.2), ``steps`` plain kick-drift-kick steps each (sph_step without the
seed), every step followed by an online Adam round of ``iters`` iterations on
the step's (features, log(h_new/h_old)) samples, on the context's side
stream.  Each run starts from the weights the previous one left.
"""
from __future__ import annotations

import math

import numpy as np

from . import binding as B
from . import inputs


def initial_theta(seed: int = 1234) -> np.ndarray:
    """Seeded initial weights in the flat layout of include/sph.h (W1, b1,
    W2, b2, W3, b3): Gaussian W1 with variance 1/5, W2 and W3 with 1/64,
    zero biases."""
    rng = np.random.default_rng(seed)
    return np.concatenate([rng.normal(scale=s, size=k) for s, k in
                           ((1 / math.sqrt(5), 320), (0, 64), (1 / 8, 4096), (0, 64), (1 / 8, 64), (0, 1))]
                          ).astype(np.float32)


def training_workloads():
    return (("lattice16_variable_h", inputs.lattice(16, kernel=inputs.M4, fixed_h=False)),
            ("sedov64", inputs.sedov(64)))


def train(steps: int = 200, iters: int = 40, lr: float = 1e-3, batch: int = 8192,
          theta: np.ndarray | None = None) -> tuple[np.ndarray, dict]:
    """Run the protocol; returns the trained weights and the last online
    training loss of each run."""
    theta = initial_theta() if theta is None else np.asarray(theta, dtype=np.float32)
    losses = {}
    for name, w in training_workloads():
        params = dict(w.params)
        params.update(hnet_batch=batch, hnet_iters=iters, hnet_lr=lr)
        ctx = B.Context(params, w.n)
        p = B.Particles.from_workload(w, fp64=params.get("precision", "fp64") == "fp64")
        B.sph_build_tree(ctx, p)
        B.sph_density(ctx, p)
        B.sph_forces(ctx, p)
        B.sph_hnet_set_weights(ctx, theta)
        # the workload's fixed step, else the initial CFL step kept fixed
        dt = w.dt if w.dt else float(params["cfl"] * (p.h / p.vsig).min().item())
        last = None
        for _ in range(steps):
            last = B.sph_step(ctx, p, dt, use_hnet=B.SPH_HNET_TRAIN)["hnet_loss"]
        B.sph_step(ctx, p, dt, use_hnet=0)           # joins the last training round
        theta = B.sph_hnet_get_weights(ctx)
        losses[name] = last
        ctx.close()
        del p
    return theta, losses
