"""Training and use of the learned sparse-approximate-inverse preconditioner.

Orchestration only: every computation runs in the library's kernels (network
forward/backward/Adam, s-step GMRES).  Training data are residual vectors that
Jacobi-preconditioned s-step GMRES itself produces on the training matrices (the
true residual at the start of each restart cycle, returned by the solver), plus a
few random probe vectors.  At solve time the network's M is used only if its loss
on probe vectors beats the Jacobi preconditioner's (an untrained network, output
layer zero, *is* Jacobi); otherwise the solve falls back to Jacobi.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

import paper_2503_16717_gb300 as rbo


@dataclass
class Instance:
    A: "rbo.DeviceCSR"
    R: object                      # device n x k residual / probe columns
    n: int
    meta: dict = field(default_factory=dict)


def residual_batch(A: "rbo.DeviceCSR", seed: int, n_resid: int = 6, n_probe: int = 4,
                   s: int = 5, m: int = 30):
    """Residual vectors from Jacobi s-step GMRES on A x = b (b seeded Gaussian) plus
    Gaussian probes, as one column-major device matrix."""
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    b = torch.randn(A.n, generator=g, device="cuda", dtype=torch.float64)
    R = rbo.colmajor(A.n, n_resid + n_probe)
    _, info = rbo.sstep_gmres(A, b, s=s, m=m, tol=1e-12, max_restarts=n_resid - 1,
                              resid=R[:, :n_resid])
    k = info["resid_len"]
    if k < n_resid:  # converged early: fill with more probes
        R[:, k:n_resid].copy_(torch.randn((A.n, n_resid - k), generator=g, device="cuda",
                                          dtype=torch.float64))
    R[:, n_resid:].copy_(torch.randn((A.n, n_probe), generator=g, device="cuda", dtype=torch.float64))
    return R


def make_instances(gen, seeds, N: int, **kw) -> list[Instance]:
    out = []
    for sd in seeds:
        Ah, meta = gen(N, sd)
        Ad = rbo.DeviceCSR.from_host(Ah)
        out.append(Instance(Ad, residual_batch(Ad, sd, **kw), Ad.n, meta))
    return out


def train(net: "rbo.GNN", instances: list[Instance], epochs: int = 4, lr: float = 3e-3,
          lr_decay: float = 0.7, seed: int = 0) -> dict:
    """Adam over the instances (shuffled each epoch); returns loss history."""
    rng = np.random.default_rng(seed)
    hist = []
    t0 = time.perf_counter()
    for ep in range(epochs):
        order = rng.permutation(len(instances))
        losses = [net.train_step(instances[i].A, instances[i].R, lr=lr) for i in order]
        hist.append(float(np.mean(losses)))
        lr *= lr_decay
    return {"epoch_loss": hist, "seconds": time.perf_counter() - t0}


def choose(net: "rbo.GNN", A: "rbo.DeviceCSR", probes, jacobi: "rbo.GNN"):
    """M from the network if it beats Jacobi on the probe vectors, else None
    (fall back to Jacobi).  Returns (M or None, learned loss, Jacobi loss)."""
    Ll, _ = net.loss_grad(A, probes)
    Lj, _ = jacobi.loss_grad(A, probes)
    if Ll < Lj:
        return net.infer(A), Ll, Lj
    return None, Ll, Lj


def solve(net, A, b, *, jacobi=None, probes=None, s=5, s_hat=0, m=60, tol=1e-10, **kw):
    """s-step GMRES with the learned preconditioner (Jacobi fallback).  Returns
    (x, info, used_learned)."""
    import torch
    if jacobi is None:
        jacobi = rbo.GNN(seed=0)
    if probes is None:
        g = torch.Generator(device="cuda")
        g.manual_seed(12345)
        probes = rbo.colmajor(A.n, 4)
        probes.copy_(torch.randn((A.n, 4), generator=g, device="cuda", dtype=torch.float64))
    M, Ll, Lj = choose(net, A, probes, jacobi)
    x, info = rbo.sstep_gmres(A, b, s=s, s_hat=s_hat, m=m, tol=tol, M=M, **kw)
    info["learned_loss"], info["jacobi_loss"] = Ll, Lj
    return x, info, M is not None
