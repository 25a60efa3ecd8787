"""Sharded execution of a rotation sequence over 2^m ranks (see ps_shard_swap_plan).

Each rank holds one slab of 2^(n-m) amplitudes.  The plan alternates
windows, which every rank applies to its own slab with the single-GPU
kernels, and exchanges, which swap k rank bits with k slab bits.  An
exchange runs as 2^k - 1 pairwise rounds: in round t the rank whose swapped
bits spell j trades part j ^ t of its slab (the amplitudes whose swapped
slab bits spell j ^ t) with the rank whose swapped bits spell j ^ t, which
sends its part j back; the received part lands where the sent one was.
Every part moves in chunks through two chunk buffers, so a rank needs its
slab plus two chunks, and the arithmetic and the data movement run in libps
(ps_shard_pack / ps_shard_unpack); this module arranges the calls and hands
each chunk to a communication callback:

  exchange(send, partner) -> the partner's chunk (the partner sends ours)

`torch_exchange` does it with torch.distributed point-to-point messages
(NCCL between GPUs, gloo between CPU processes); `libps_moves` gives the
pack / unpack callbacks on a CUDA slab.
"""
from __future__ import annotations

from . import ps_shard_pack, ps_shard_swap_plan, ps_shard_unpack


def set_bits(mask: int) -> list[int]:
    out, p = [], 0
    while mask >> p:
        if (mask >> p) & 1:
            out.append(p)
        p += 1
    return out


def swapped_bits(rank: int, s: int, rank_mask: int) -> int:
    """The value j that the swapped rank bits of `rank` spell (t-th lowest bit <-> t-th swapped position)."""
    j = 0
    for t, p in enumerate(set_bits(rank_mask)):
        j |= ((rank >> (p - s)) & 1) << t
    return j


def rank_with_bits(rank: int, s: int, rank_mask: int, j: int) -> int:
    """`rank` with its swapped bits replaced by the bits of j."""
    for t, p in enumerate(set_bits(rank_mask)):
        b = p - s
        rank = (rank & ~(1 << b)) | (((j >> t) & 1) << b)
    return rank


def exchange_rounds(rank: int, s: int, rank_mask: int):
    """(partner, part index) of rounds t = 1 .. 2^k - 1 of one exchange."""
    k = bin(rank_mask).count("1")
    own = swapped_bits(rank, s, rank_mask)
    return [(rank_with_bits(rank, s, rank_mask, own ^ t), own ^ t) for t in range(1, 1 << k)]


def run_sharded(n: int, m: int, rank: int, slab, x, z, phi, exchange, apply, pack, unpack, k_max: int | None = None,
                layout=None, chunk_bits: int | None = None):
    """Evolve this rank's slab through the sequence; returns (slab, layout).
    apply(slab, x, z, phi) -> slab;  pack(slab, slab_mask, first, count) -> chunk;
    unpack(chunk, slab_mask, first, slab) -> slab (packed ranges, see ps_shard_pack).
    chunk_bits: log2 of the amplitudes per message (default: a whole part)."""
    s = n - m
    steps, layout = ps_shard_swap_plan(n, m, m if k_max is None else k_max, rank, x, z, phi, layout)
    for st in steps:
        if st[0] == "window":
            if len(st[3]):
                slab = apply(slab, st[1], st[2], st[3])
            continue
        _, rank_mask, slab_mask = st
        k = bin(rank_mask).count("1")
        part = 1 << (s - k)
        chunk = part if chunk_bits is None else min(part, 1 << chunk_bits)
        for partner, j in exchange_rounds(rank, s, rank_mask):
            for c0 in range(0, part, chunk):
                first = j * part + c0
                got = exchange(pack(slab, slab_mask, first, chunk), partner)
                slab = unpack(got, slab_mask, first, slab)
    return slab, layout


def torch_exchange(dist):
    """One chunk each way with the partner as a batched isend / irecv pair."""
    def exchange(send, partner):
        import torch
        out = torch.empty_like(send)
        ops = [dist.P2POp(dist.isend, send.contiguous(), partner), dist.P2POp(dist.irecv, out, partner)]
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        return out
    return exchange


def libps_moves(s: int, dtype: int, stream=None):
    """pack / unpack callbacks for a CUDA slab tensor of 2^s amplitudes (libps kernels)."""
    import torch

    def _stream():
        return (stream if stream is not None else torch.cuda.current_stream()).cuda_stream

    def pack(slab, slab_mask, first, count):
        out = torch.empty(count, dtype=slab.dtype, device=slab.device)
        ps_shard_pack(s, dtype, slab_mask, first, count, slab.data_ptr(), out.data_ptr(), _stream())
        return out

    def unpack(chunk, slab_mask, first, slab):
        ps_shard_unpack(s, dtype, slab_mask, first, chunk.numel(), chunk.data_ptr(), slab.data_ptr(), _stream())
        return slab

    return pack, unpack
