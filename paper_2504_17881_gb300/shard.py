"""Sharded execution of a rotation sequence over 2^m ranks (see ps_shard_swap_plan).

Each rank holds one slab of 2^(n-m) amplitudes.  The plan alternates
windows, which every rank applies to its own slab with the single-GPU
kernels, and exchanges, which swap rank bits with slab bits: the slab is
packed into 2^k parts (ps_shard_pack), part j goes to the rank whose
swapped bits spell j, and the parts received are placed back
(ps_shard_unpack).  The arithmetic and the data movement run in libps; this
module arranges the calls and hands the parts to a communication callback:

  exchange(parts, partners) -> received parts, parts[j] sent to partners[j]
      and received[j] from partners[j] (partners[j] == rank: the own part)

`torch_exchange` does it with torch.distributed point-to-point messages
(NCCL between GPUs, gloo between CPU processes); `libps_moves` gives the
pack / unpack / apply callbacks on a CUDA slab.
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


def exchange_partners(rank: int, s: int, rank_mask: int) -> list[int]:
    """Rank receiving part j of an exchange over the rank positions of rank_mask
    (ascending): `rank` with bit t of j at the t-th swapped rank bit."""
    gbits = [p - s for p in set_bits(rank_mask)]
    out = []
    for j in range(1 << len(gbits)):
        r = rank
        for t, b in enumerate(gbits):
            r = (r & ~(1 << b)) | (((j >> t) & 1) << b)
        out.append(r)
    return out


def run_sharded(n: int, m: int, rank: int, slab, x, z, phi, exchange, apply, pack, unpack, k_max: int | None = None,
                layout=None):
    """Evolve this rank's slab through the sequence; returns (slab, layout).
    apply(slab, x, z, phi) -> slab;  pack(slab, slab_mask) -> parts (a sequence of 2^k);
    unpack(parts, slab_mask, slab) -> slab."""
    s = n - m
    steps, layout = ps_shard_swap_plan(n, m, m if k_max is None else k_max, rank, x, z, phi, layout)
    for st in steps:
        if st[0] == "window":
            if len(st[3]):
                slab = apply(slab, st[1], st[2], st[3])
        else:
            _, rank_mask, slab_mask = st
            parts = pack(slab, slab_mask)
            received = exchange(parts, exchange_partners(rank, s, rank_mask))
            slab = unpack(received, slab_mask, slab)
    return slab, layout


def torch_exchange(dist):
    """All parts of one exchange as batched point-to-point messages."""
    def exchange(parts, partners):
        import torch
        me = dist.get_rank()
        out = [None] * len(parts)
        ops = []
        for j, p in enumerate(partners):
            if p == me:
                out[j] = parts[j]
            else:
                out[j] = torch.empty_like(parts[j])
                ops.append(dist.P2POp(dist.isend, parts[j].contiguous(), p))
                ops.append(dist.P2POp(dist.irecv, out[j], p))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        return out
    return exchange


def libps_moves(s: int, dtype: int, stream=None):
    """pack / unpack callbacks for a CUDA slab tensor of 2^s amplitudes (libps kernels)."""
    import torch

    def _stream():
        return (stream if stream is not None else torch.cuda.current_stream()).cuda_stream

    def pack(slab, slab_mask):
        k = bin(slab_mask).count("1")
        out = torch.empty_like(slab)
        ps_shard_pack(s, dtype, slab_mask, slab.data_ptr(), out.data_ptr(), _stream())
        return list(out.view(1 << k, 1 << (s - k)).unbind(0))

    def unpack(parts, slab_mask, slab):
        buf = torch.cat([p.reshape(-1) for p in parts])
        ps_shard_unpack(s, dtype, slab_mask, buf.data_ptr(), slab.data_ptr(), _stream())
        return slab

    return pack, unpack
