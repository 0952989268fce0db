"""Training recipe of the learned block-Jacobi correction.

Orchestration only: every number is computed by the library's kernels
(data collection, slow-mode probes, the tensor-core network and Adam); this
module draws the Rademacher probes, concatenates and shuffles the samples.

    samples = [collect(prob) for prob in problems]        # Problem objects
    params, hist = train(samples)
    prob.set_preconditioner(params)
"""
from __future__ import annotations

import torch

from . import Problem, mlp_init, mlp_train, mlp_loss_grad

__all__ = ["collect", "concat", "train", "held_out_loss"]


def collect(prob: Problem, states=(0, 1, 3), rademacher: int = 4, slow_iters=(20, 50), seed: int = 0,
            maxiter_ref: int = 600, tol_ref: float = 1e-10):
    """Samples (X [n, 96], A [n, 45], Y [n, K, 9], Z [n, K, 9]) of one problem
    at the LM states after `states` trials (cumulative; the problem is
    advanced by its own solver), K = rademacher + len(slow_iters) probes per
    camera: Rademacher probes and, at the same damping, slow-mode probes
    (scaled errors of truncated block-Jacobi PCG runs)."""
    g = torch.Generator(device=prob.device).manual_seed(int(seed))
    out = []
    done = 0
    for s in states:
        if s > done:
            prob.solve(s - done)
            done = s
        _, lam = prob.scalars()
        z = torch.randint(0, 2, (prob.C, rademacher, 9), generator=g, device=prob.device).float() * 2 - 1
        if slow_iters:
            z = torch.cat([z, prob.learn_slow_probes(lam, slow_iters, maxiter_ref, tol_ref)], 1)
        X, A, Y = prob.learn_collect(lam, z)
        out.append((X, A, Y, z))
    return tuple(torch.cat([o[i] for o in out]) for i in range(4))


def concat(samples, seed: int = 0):
    """Concatenate per-problem samples and shuffle them (minibatches are runs
    of consecutive samples)."""
    parts = [torch.cat([s[i] for s in samples]) for i in range(4)]
    g = torch.Generator().manual_seed(int(seed))
    perm = torch.randperm(parts[0].shape[0], generator=g).to(parts[0].device)
    return tuple(p[perm].contiguous() for p in parts)


def train(samples, epochs: int = 100, batch: int = 512, lr: float = 2e-3, seed: int = 0, params=None):
    """Adam on the network from `params` (default: block-Jacobi start, a zero
    output layer); returns (params, per-epoch losses)."""
    X, A, Y, Z = concat(samples, seed) if isinstance(samples, (list, tuple)) and isinstance(samples[0], tuple) \
        else samples
    p = (mlp_init(seed, device=X.device) if params is None else params.detach().clone()).contiguous()
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    hist = mlp_train(p, m, v, X, A, Y, Z, epochs, batch, lr)
    return p, hist


def held_out_loss(params, samples):
    X, A, Y, Z = samples
    return mlp_loss_grad(params, X, A, Y, Z)[0]
