"""Sharded execution of a rotation sequence over 2^m ranks (see ps_shard_plan).

Each rank holds one slab of the state.  For every window of the plan it
either applies the window to its slab, or exchanges slabs with its partner
once, applies the window to the two slabs as one state (own half first) and
keeps its own half.  The two callbacks carry the device-specific parts:

  exchange(own, partner) -> the partner's slab (the partner sends ours)
  apply(state, x, z, phi) -> the state after the rotations (libps on a GPU)

`torch_exchange` does the exchange with torch.distributed point-to-point
messages (NCCL between GPUs, gloo between CPU processes).
"""
from __future__ import annotations

from . import ps_shard_plan


def run_sharded(n: int, m: int, rank: int, slab, x, z, phi, exchange, apply, concat, split):
    """Evolve this rank's slab through the sequence; returns the new slab.
    concat(own, other) builds the two-slab state; split(state) returns its own half."""
    for partner, xl, zl, pl in ps_shard_plan(n, m, rank, x, z, phi):
        if len(pl) == 0:
            continue
        if partner < 0:
            slab = apply(slab, xl, zl, pl)
        else:
            other = exchange(slab, partner)
            slab = split(apply(concat(slab, other), xl, zl, pl))
    return slab


def torch_exchange(dist):
    """Point-to-point slab exchange over a torch.distributed process group;
    the lower rank sends first, so the pair never waits on itself."""
    def exchange(own, partner):
        import torch
        other = torch.empty_like(own)
        me = dist.get_rank()
        if me < partner:
            dist.send(own, partner)
            dist.recv(other, partner)
        else:
            dist.recv(other, partner)
            dist.send(own, partner)
        return other
    return exchange
