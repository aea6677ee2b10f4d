"""Gradients of time-averaged observables with respect to (beta, h, J) by the
score function of the simulated paths, as a torch.autograd.Function.

The chain of §3 has path log-likelihood log L = sum over events of
log p_k(event) - integral of sum_k N_k p_k dt.  For a time average A of the
path, d E[A] / d theta = E[A S] + E[dA / d theta] with S = d log L / d theta.
The forward pass simulates the replicas in score mode (the library keeps the
path statistics of S while it runs); the backward pass is the library's
gradient kernel (sr_score_grad).  Replicas are independent estimates: the
gradient of a replica is noisy, its mean over replicas is unbiased.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Sequence, Tuple

import numpy as np
import torch

from . import Batch, _check, library


@dataclass
class AverageSpec:
    """What to simulate: replica i is an L[i] x L[i] lattice with seed seeds[i]
    and parameters theta[i] = (beta, h, J); the averages run over [t1, t2]."""
    L: Sequence[int]
    seeds: Sequence[int]
    t1: float
    t2: float
    region: Tuple[int, int] = (16, 16)
    kappa: float = 8.0
    init: str = "fair"
    rates: str = "metropolis"
    settings: dict = field(default_factory=dict)


def _simulate(theta: np.ndarray, spec: AverageSpec, samples: int = 0):
    """Time averages A [R, 2] (m and energy per site over [t1, t2]), scores
    S [R, 3] and the averages' explicit derivatives E [R, 2, 3]; with
    samples > 0 also m at `samples` equally spaced times in (t1, t2]."""
    R = theta.shape[0]
    reps = [dict(L=int(spec.L[i]), J=float(theta[i, 2]), h=float(theta[i, 1]),
                 T=1.0 / float(theta[i, 0]), seed=int(spec.seeds[i]), init=spec.init,
                 rates=spec.rates) for i in range(R)]
    with Batch(reps, region=spec.region, score=True, **spec.settings) as bt:
        if spec.t1 > 0:
            bt.run_adaptive(spec.t1, kappa=spec.kappa)
        o1 = [bt.observables(b) for b in range(R)]
        msamp = np.zeros((R, max(samples, 0)))
        for j in range(samples):
            t = spec.t1 + (spec.t2 - spec.t1) * (j + 1) / samples
            bt.run_adaptive(t, kappa=spec.kappa)
            for b in range(R):
                msamp[b, j] = bt.observables(b).m
        bt.run_adaptive(spec.t2, kappa=spec.kappa)
        o2 = [bt.observables(b) for b in range(R)]
        S = bt.score()
    A = np.zeros((R, 2))
    E = np.zeros((R, 2, 3))
    for i in range(R):
        n = float(spec.L[i]) ** 2 * (spec.t2 - spec.t1)
        dM = o2[i].int_mag - o1[i].int_mag
        dB = o2[i].int_bonds - o1[i].int_bonds
        h, J = theta[i, 1], theta[i, 2]
        A[i, 0] = dM / n
        A[i, 1] = (-J * dB - h * dM) / n          # energy per site, Eq. 2.1
        E[i, 1, 1] = -dM / n
        E[i, 1, 2] = -dB / n
    if samples:
        return A, S, E, msamp
    return A, S, E


class TimeAverages(torch.autograd.Function):
    """theta [R, 3] (beta, h, J) -> A [R, 2]: time-averaged magnetisation and
    energy per site of R independent replicas over [t1, t2]."""

    @staticmethod
    def forward(ctx, theta: torch.Tensor, spec: AverageSpec):
        if not theta.is_cuda:
            raise RuntimeError("TimeAverages runs on the GPU: pass theta on a CUDA device")
        A, S, E = _simulate(theta.detach().double().cpu().numpy(), spec)
        dev = theta.device
        At = torch.from_numpy(A).to(dev)
        ctx.save_for_backward(At, torch.from_numpy(S).to(dev), torch.from_numpy(E).to(dev))
        return At.to(theta.dtype)

    @staticmethod
    def backward(ctx, gA: torch.Tensor):
        A, S, E = ctx.saved_tensors
        gA = gA.detach().double().contiguous()
        G = torch.empty_like(S)
        stream = torch.cuda.current_stream(A.device).cuda_stream
        n, m = A.shape
        _check(library().sr_score_grad(n, m, S.shape[1], A.data_ptr(), gA.data_ptr(),
                                       S.data_ptr(), E.data_ptr(), G.data_ptr(), stream),
               "sr_score_grad")
        return G, None


def time_averages(theta: torch.Tensor, spec: AverageSpec) -> torch.Tensor:
    return TimeAverages.apply(theta, spec)
