"""One instance's plate sharded over processes, one GPU each.

Sec. 6 sums each plate out given its parent's samples.  The elements of the
root's child plate are therefore independent given the root's K samples, and
the root step (Eq. Prmp) sees them only through their plate sum
G[i][k_p] = sum_c log mean_k exp S_c[k_p][k].  A shard holds every root and a
contiguous range of the root's children with all their descendants.  One
E-step on N shards is then

  1. per shard: sample and contract its range into its own G_r
     (``Plan.shard_forward``, no root step);
  2. G = sum_r G_r: one all-reduce of n_inst x K doubles (NCCL between GPUs,
     gloo between CPU processes);
  3. per shard: the root step on G (the roots' samples, hence its result, are
     the same on every shard), then the adjoint and the moments of its own
     range (``Plan.shard_finish``): the adjoint needs no exchange, since the
     root's weights are replicated.

The M-step stays local: each shard updates its own elements, and every shard
updates the roots alike from identical moments.  With ``Plan.set_elem_base``
each shard draws the in-kernel noise of the whole model, so a sharded run
draws the same samples as one process holding everything.
"""
from __future__ import annotations

from dataclasses import replace

import numpy as np

from . import synth as S


def child_ranges(model: S.Model, world: int) -> list:
    """Contiguous ranges [lo, hi) of the root's children (level 1), one per
    rank, balanced by the number of elements in each child's subtree (every
    element below the root costs one K x K contraction).  A chain plate at
    level 1 is cut only between whole chains.  Needs at least one unit (child
    or chain) per rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    lv = model.levels
    if len(lv) < 2:
        raise ValueError("a one-level model has no plate to shard")
    n1 = lv[1].n
    unit = int(getattr(lv[1], "chain", 1) or 1)
    if n1 % unit:
        raise ValueError("level 1 is not a whole number of chains")
    n_units = n1 // unit
    if n_units < world:
        raise ValueError(f"{n_units} shardable units for {world} ranks")
    size = np.ones(n1, np.int64)
    anc = np.arange(n1, dtype=np.int64)
    for l in range(2, len(lv)):
        anc = anc[np.asarray(lv[l].parent, np.int64)]
        size += np.bincount(anc, minlength=n1)
    usize = size.reshape(n_units, unit).sum(1)
    cum = np.cumsum(usize)
    bounds = [0]
    for r in range(1, world):
        b = int(np.searchsorted(cum, cum[-1] * r / world, side="left")) + 1
        b = min(max(b, bounds[-1] + 1), n_units - (world - r))  # at least one unit per rank
        bounds.append(b)
    bounds.append(n_units)
    return [(bounds[r] * unit, bounds[r + 1] * unit) for r in range(world)]


def level_ranges(model: S.Model, lo: int, hi: int) -> list:
    """Per level, the contiguous range of elements that a shard holding the
    root's children [lo, hi) holds: every root, the range itself, then the
    children of each range in turn (parents are non-decreasing)."""
    lv = model.levels
    out = [(0, lv[0].n), (lo, hi)]
    for l in range(2, len(lv)):
        par = np.asarray(lv[l].parent, np.int64)
        plo, phi = out[-1]
        out.append((int(np.searchsorted(par, plo, side="left")), int(np.searchsorted(par, phi, side="left"))))
    return out


def shard_model(model: S.Model, lo: int, hi: int) -> tuple:
    """The sub-model of a shard holding the root's children [lo, hi): returns
    (sub_model, ranges) with ranges[l] = (first, end) of level l's elements
    in the whole model."""
    ranges = level_ranges(model, lo, hi)
    levels = []
    for l, lv in enumerate(model.levels):
        a, b = ranges[l]
        kw = {"n": b - a}
        if lv.parent is not None:
            base = ranges[l - 1][0]
            kw["parent"] = np.ascontiguousarray(np.asarray(lv.parent, np.int64)[a:b] - base)
        if lv.x is not None:
            kw["x"] = lv.x[a:b]
        if lv.y is not None:
            kw["y"] = lv.y[a:b]
        levels.append(replace(lv, **kw))
    return S.Model(levels, name=f"{model.name}_shard{lo}_{hi}"), ranges


def take(per_level: list, ranges: list) -> list:
    """Slice per-level arrays (leading axis = element) to a shard's ranges."""
    return [np.asarray(a)[lo:hi] for a, (lo, hi) in zip(per_level, ranges)]


def assemble(parts: list, ranges_of: list) -> list:
    """Whole-model per-level arrays from every shard's per-level parts
    (parts[r][l], ranges_of[r][l]); the roots come from shard 0 (every
    shard holds the same)."""
    n_levels = len(parts[0])
    out = [np.asarray(parts[0][0])]
    for l in range(1, n_levels):
        order = sorted(range(len(parts)), key=lambda r: ranges_of[r][l][0])
        out.append(np.concatenate([np.asarray(parts[r][l]) for r in order], axis=0))
    return out


class ShardedEStep:
    """The E-step of one shard: ``engine.shard_forward`` -> sum of G over the
    process group -> ``engine.shard_finish``.

    engine: an object with ``shard_forward(q, eps, seed, it) -> G`` (a tensor
    [n_inst, K]) and ``shard_finish(G) -> result``, normally a ``qem.Plan``
    of ``self.sub`` (made here when engine is None).  group: the
    torch.distributed process group (None: the default group; world 1 needs
    none)."""

    def __init__(self, model: S.Model, K: int, rank: int, world: int, engine=None, group=None, **plan_kw):
        self.model, self.K, self.rank, self.world, self.group = model, K, rank, world, group
        self.lo, self.hi = child_ranges(model, world)[rank]
        self.sub, self.ranges = shard_model(model, self.lo, self.hi)
        if engine is None:
            from . import qem
            engine = qem.Plan(self.sub, K, **plan_kw)
            engine.set_elem_base([a for a, _ in self.ranges])
        self.engine = engine

    def reduce(self, G):
        """Sum G over the group in place (on the engine's stream for CUDA tensors)."""
        if self.world == 1:
            return G
        import torch
        import torch.distributed as dist
        stream = getattr(self.engine, "stream", None)
        if G.is_cuda and stream is not None:
            with torch.cuda.stream(stream):
                dist.all_reduce(G, op=dist.ReduceOp.SUM, group=self.group)
        else:
            dist.all_reduce(G, op=dist.ReduceOp.SUM, group=self.group)
        return G

    def estep(self, q, eps=None, seed: int = 0, it: int = 0):
        G = self.engine.shard_forward(q, eps, seed, it)
        self.reduce(G)
        return self.engine.shard_finish(G)
