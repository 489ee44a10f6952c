"""One cluster integrated by several ranks, each owning a range of bodies:
the paper's multi-GPU scheme (Sect. 4.2), where every GPU computes the
accelerations of its share of the bodies against all of them and the GPUs
exchange positions between force evaluations.

Each rank holds every body's position and mass, and the velocities of its own
range [i0, i1).  One step of order 2 or 6 is the substep sequence of
``schedule``: a drift of the own range, then, per stage, a force evaluation
of the own range against all bodies, its kick and the following drift
(``nb_substep_range``), with an exchange of the ranges' new positions between
substeps (an all-gather into every rank's buffer, then
``nb_set_state_device``).  The first substep of a step is a drift alone,
so the exchange after a step's last substep waits until then; ``gather``
makes every rank's state whole for reading.

Ranges are equal chunks of whole i-blocks (the last one short), so every
rank's slice of the all-gather has the same size.  A rank's force
evaluation sums each i-block's row in order in one block, so the bits of a
body's result do not depend on how the bodies are split (one rank or many).

This module is host logic over the C ABI and torch.distributed: NCCL between
GPUs, gloo between CPU processes; the exchange is pluggable, and
``LocalExchange`` runs several ranks in one process one after another (no
rank waits on another's kernels).
"""
from __future__ import annotations

import math

import numpy as np

ALIGN = 1024   # bodies per chunk unit: the widest i-block of the pair kernels


def ranges(n: int, world: int, align: int = ALIGN):
    """Bodies [i0, i1) of each rank and the common chunk length: chunks of
    ceil(n / world) bodies rounded up to whole multiples of align."""
    if n < 1 or world < 1:
        raise ValueError("need n >= 1 and world >= 1")
    chunk = math.ceil(math.ceil(n / world) / align) * align
    return [(min(r * chunk, n), min((r + 1) * chunk, n)) for r in range(world)], chunk


def schedule(weights, dt: float):
    """(kick, drift) substeps of one step with the given kick weights: a
    drift of w_0 / 2, then kick w_k and drift (w_k + w_k+1) / 2 per stage, the
    last drift w_last / 2 (adjacent half drifts merged, as nb_step does)."""
    K = len(weights)
    subs = [(0.0, 0.5 * weights[0] * dt)]
    for k in range(K):
        nxt = weights[k + 1] if k + 1 < K else 0.0
        subs.append((weights[k] * dt, 0.5 * (weights[k] + nxt) * dt))
    return subs


class Rank:
    """One rank's share: a backend holding the whole system, its range and
    the chunk length of the exchange.  The backend provides n,
    substep_range(i0, i1, kick, drift), positions() and velocities() (n x 3
    torch tensors), set_positions(t) and set_velocities(t) (n x 3)."""

    def __init__(self, backend, i0: int, i1: int, chunk: int):
        self.b, self.i0, self.i1, self.chunk = backend, i0, i1, chunk

    def substep(self, kick: float, drift: float):
        if self.i1 > self.i0:
            self.b.substep_range(self.i0, self.i1, kick, drift)

    def _rows(self, full):
        """Own rows of a whole (n, 3) tensor, padded to the chunk length."""
        import torch
        out = torch.zeros((self.chunk, 3), dtype=full.dtype, device=full.device)
        out[: self.i1 - self.i0] = full[self.i0:self.i1]
        return out

    def local_positions(self):
        return self._rows(self.b.positions())

    def local_velocities(self):
        return self._rows(self.b.velocities())


class LocalExchange:
    """All ranks in one process: the all-gather is a concatenation in rank
    order, applied to every rank."""

    def positions(self, ranks):
        import torch
        full = torch.cat([r.local_positions() for r in ranks])
        for r in ranks:
            r.b.set_positions(full[: r.b.n])

    def velocities(self, ranks):
        import torch
        full = torch.cat([r.local_velocities() for r in ranks])
        for r in ranks:
            r.b.set_velocities(full[: r.b.n])


class DistExchange:
    """One rank per process over torch.distributed (all_gather_into_tensor
    with NCCL, all_gather with other backends)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist, self.group = dist, group
        self.world = dist.get_world_size(group)

    def _gather(self, local):
        import torch
        if self.dist.get_backend(self.group) == "nccl":
            out = torch.empty((self.world * local.shape[0], 3), dtype=local.dtype,
                              device=local.device)
            self.dist.all_gather_into_tensor(out, local.contiguous(), group=self.group)
            return out
        parts = [torch.empty_like(local) for _ in range(self.world)]
        self.dist.all_gather(parts, local.contiguous(), group=self.group)
        return torch.cat(parts)

    def positions(self, ranks):
        (r,) = ranks
        r.b.set_positions(self._gather(r.local_positions())[: r.b.n])

    def velocities(self, ranks):
        (r,) = ranks
        r.b.set_velocities(self._gather(r.local_velocities())[: r.b.n])


def run(ranks, exchange, weights, dt: float, nsteps: int):
    """nsteps steps of every rank in ``ranks`` (this process's ranks: one
    with DistExchange, all with LocalExchange)."""
    subs = schedule(weights, dt)
    for _ in range(nsteps):
        for q, (kick, drift) in enumerate(subs):
            if q > 0:
                exchange.positions(ranks)   # the kicks need every position
            for r in ranks:
                r.substep(kick, drift)


def gather(ranks, exchange):
    """Make every rank's positions and velocities whole (after run)."""
    exchange.positions(ranks)
    exchange.velocities(ranks)


class ContextBackend:
    """A one-cluster nbsym.Context as a rank's backend (device tensors).

    The context runs on its own stream, torch (the exchange's slicing,
    concatenation and collectives) on torch's current stream: a tensor torch
    produced is waited for before the context reads it, and the context's
    calls return with their work done (they synchronise its stream)."""

    def __init__(self, ctx, device):
        import torch
        self.torch = torch
        self.ctx, self.n = ctx, ctx.n
        self.device = torch.device(device)
        self._pos = torch.empty((self.n, 3), dtype=torch.float64, device=self.device)
        self._vel = torch.empty((self.n, 3), dtype=torch.float64, device=self.device)

    def substep_range(self, i0, i1, kick, drift):
        self.ctx.substep_range(i0, i1, kick, drift)

    def positions(self):
        self.ctx.get_state_device(self._pos, None)
        return self._pos

    def velocities(self):
        self.ctx.get_state_device(None, self._vel)
        return self._vel

    def _ready(self, t):
        t = t.contiguous()
        self.torch.cuda.current_stream(self.device).synchronize()
        return t

    def set_positions(self, t):
        self.ctx.set_state_device(self._ready(t), None)

    def set_velocities(self, t):
        self.ctx.set_state_device(None, self._ready(t))
