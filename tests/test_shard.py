"""Sharded schedule over 2^m ranks (ps_shard_swap_plan, shard.run_sharded).

The schedule is checked against the oracle's single-state evolution three
ways: all ranks emulated in one process with a numpy model of the exchange
and the oracle applying each window (CPU), real gloo ranks exchanging parts
with torch.distributed (CPU, world sizes 2, 4 and 8), and all ranks emulated
on one GPU with the libps pack / unpack kernels and libps applying every
window (GPU).  The final state is in the plan's final layout; the tests map
it back to logical qubit order.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import paper_2504_17881_gb300 as ps
from paper_2504_17881_gb300 import inputs, shard


def sequence(n, seed):
    """Random strings (their X parts cut to at most 3 qubits, so that a slab of
    n - m >= 5 qubits can hold any one of them) plus JW-like terms, so X masks
    touch rank bits often."""
    xr, zr, pr = inputs.random_rotations(n, 40, seed=seed)
    rng = np.random.default_rng(seed + 7)
    for i in range(len(xr)):
        bits = [q for q in range(n) if (int(xr[i]) >> q) & 1]
        keep = rng.permutation(bits)[:3] if bits else []
        xr[i] = np.uint64(sum(1 << int(q) for q in keep))
    x, z, h = inputs.jw_hamiltonian(n, 30, seed=seed + 1)
    ang = rng.uniform(-1, 1, size=30)
    return (np.concatenate([xr, x]), np.concatenate([zr, z]), np.concatenate([pr, ang]))


# ------------------------------------------ a numpy model of the exchange

def _insert(c, j, pos):
    for t, p in enumerate(pos):
        c = ((c >> p) << (p + 1)) | (c & ((1 << p) - 1)) | (((j >> t) & 1) << p)
    return c


def _packed_at(slab, slab_mask, first, count):
    """Slab indices of packed indices first .. first + count - 1 (part j, amplitude c: bits of j at slab_mask)."""
    pos = shard.set_bits(slab_mask)
    k, s = len(pos), slab.size.bit_length() - 1
    idx = np.arange(first, first + count, dtype=np.int64)
    return _insert(idx & ((1 << (s - k)) - 1), idx >> (s - k), pos)


def np_pack(slab, slab_mask, first, count):
    return slab[_packed_at(slab, slab_mask, first, count)].copy()


def np_unpack(chunk, slab_mask, first, slab):
    out = slab.copy()
    out[_packed_at(slab, slab_mask, first, len(chunk))] = chunk
    return out


def to_logical(phys, layout):
    """Amplitude of logical index L sits at the physical index with bit layout[q] = bit q of L."""
    n = phys.size.bit_length() - 1
    P = np.arange(1 << n, dtype=np.int64)
    L = np.zeros_like(P)
    for q in range(n):
        L |= ((P >> int(layout[q])) & 1) << q
    out = np.empty_like(phys)
    out[L] = phys
    return out


def emulate(n, m, psi, x, z, phi, apply, pack, unpack, k_max, layout=None, chunk_bits=None):
    """All 2^m ranks in lockstep: windows on every slab; exchanges as the
    pairwise rounds of shard.exchange_rounds, chunk by chunk, every pair
    trading the chunks it packed.  psi is in the physical order of `layout`
    (identity when None)."""
    s, R = n - m, 1 << m
    slabs = [psi[r << s:(r + 1) << s].copy() for r in range(R)]
    plans = [ps.ps_shard_swap_plan(n, m, k_max, r, x, z, phi, layout) for r in range(R)]
    layout = plans[0][1]
    assert all(np.array_equal(p[1], layout) for p in plans)
    for t in range(len(plans[0][0])):
        st = plans[0][0][t]
        if st[0] == "window":
            slabs = [apply(slabs[r], *plans[r][0][t][1:]) if len(plans[r][0][t][3]) else slabs[r] for r in range(R)]
            continue
        _, rank_mask, slab_mask = st
        k = bin(rank_mask).count("1")
        part = 1 << (s - k)
        chunk = part if chunk_bits is None else min(part, 1 << chunk_bits)
        rounds = [shard.exchange_rounds(r, s, rank_mask) for r in range(R)]
        for q in range(len(rounds[0])):
            for r in range(R):
                partner, j = rounds[r][q]
                assert rounds[partner][q][0] == r  # the partner trades with r in the same round
            for c0 in range(0, part, chunk):
                sent = [pack(slabs[r], slab_mask, rounds[r][q][1] * part + c0, chunk) for r in range(R)]
                slabs = [unpack(sent[rounds[r][q][0]], slab_mask, rounds[r][q][1] * part + c0, slabs[r])
                         for r in range(R)]
    return np.concatenate(slabs), layout


def _emulate_from(n, m, phys, x, z, phi, layout):
    return emulate(n, m, phys, x, z, phi, lambda st, a, b, c: oracle.apply(st, a, b, c), np_pack, np_unpack, 2,
                   layout)


@pytest.mark.parametrize("n,m,k_max,chunk_bits", [(6, 1, 1, None), (7, 2, 1, None), (7, 2, 2, 2), (8, 3, 1, None),
                                                  (8, 3, 3, 1)])
def test_swap_plan_reproduces_single_state_evolution(n, m, k_max, chunk_bits):
    x, z, phi = sequence(n, 3 * n + m)
    psi = inputs.gaussian_state(n, 7)
    got, layout = emulate(n, m, psi, x, z, phi, lambda st, a, b, c: oracle.apply(st, a, b, c), np_pack, np_unpack,
                          k_max, chunk_bits=chunk_bits)
    ref = oracle.apply(psi, x, z, phi)
    assert np.max(np.abs(to_logical(got, layout) - ref)) < 1e-13


def test_swap_plan_structure_and_validation():
    n, m = 9, 3
    s = n - m
    x, z, phi = sequence(n, 5)
    for k_max in (1, 2, 3):
        steps, layout = ps.ps_shard_swap_plan(n, m, k_max, 5, x, z, phi)
        assert sorted(layout.tolist()) == list(range(n))
        total = 0
        for st in steps:
            if st[0] == "exchange":
                a, b = st[1], st[2]
                assert a >> s and not (a & ((1 << s) - 1)) and not (b >> s)
                assert 1 <= bin(a).count("1") == bin(b).count("1") <= m
            else:
                assert not np.any(st[1] >> np.uint64(s)) and not np.any(st[2] >> np.uint64(s))
                total += len(st[3])
        assert total == len(phi)
    # a second call continues from the first call's layout: the two together
    # still reproduce the single-state evolution
    psi = inputs.gaussian_state(n, 6)
    state = psi.copy()
    layout = None
    for lo, hi in ((0, 30), (30, len(phi))):
        part = (x[lo:hi], z[lo:hi], phi[lo:hi])
        state_log, layout = _emulate_from(n, m, state, *part, layout)
        state = state_log
    assert np.max(np.abs(to_logical(state, layout) - oracle.apply(psi, x, z, phi))) < 1e-13
    for bad in ((n, m, 0, 0), (n, 0, 1, 0), (n, m, m + 1, 0), (n, m, 1, 1 << m)):
        with pytest.raises(ps.PsError):
            ps.ps_shard_swap_plan(bad[0], bad[1], bad[2], bad[3], x, z, phi)
    with pytest.raises(ps.PsError):
        ps.ps_shard_swap_plan(n, m, 1, 0, [1 << n], [0], [0.1])
    with pytest.raises(ps.PsError):
        ps.ps_shard_swap_plan(n, m, 1, 0, x, z, phi, layout=[0] * n)
    # an X mask wider than the slab cannot be made local
    with pytest.raises(ps.PsError):
        ps.ps_shard_swap_plan(n, m, 1, 0, [(1 << (s + 1)) - 1], [0], [0.1])


def rotations_per_exchange(n, m, xs, zs, ph):
    steps, _ = ps.ps_shard_swap_plan(n, m, m, 0, xs, zs, ph)
    ex = [st for st in steps if st[0] == "exchange"]
    moved = sum(1.0 - 2.0 ** -bin(st[1]).count("1") for st in ex)
    return len(ph) / max(1, len(ex)), len(ph) / max(moved, 1e-9)


def test_headline_stream_rotations_per_exchange():
    """The n = 30 benchmark stream (10^4 JW-like terms, first 10^4 qDRIFT
    draws) spread over 2, 4 and 8 ranks: rotations per exchange, and per slab
    moved, well above one pairwise exchange per window of equal rank-bit X
    parts (7.6 at m = 2, 3.9 at m = 3 on this stream)."""
    n = 30
    x, z, h = inputs.jw_hamiltonian(n, 10_000, seed=3)
    xs, zs, ph = ps.Hamiltonian(n, x, z, h).qdrift_stream(1.0, 100_000, 4, first=0, count=10_000)
    per = {m: rotations_per_exchange(n, m, xs, zs, ph) for m in (1, 2, 3)}
    print({m: (round(a, 2), round(b, 2)) for m, (a, b) in per.items()})
    assert per[2][0] > 7.6 and per[3][0] > 3.9
    assert per[1][0] >= per[2][0] >= per[3][0]


# ------------------------------------------------------------ gloo ranks

def _free_port() -> int:
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _gloo_rank(rank, world, port, n, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m = world.bit_length() - 1
        s = n - m
        x, z, phi = sequence(n, 40 + n)
        psi = inputs.gaussian_state(n, 8)
        slab = torch.as_tensor(psi[rank << s:(rank + 1) << s].copy())

        def apply(st, a, b, c):
            return torch.as_tensor(oracle.apply(st.numpy(), a, b, c))

        def pack(st, mask, first, count):
            return torch.as_tensor(np_pack(st.numpy(), mask, first, count))

        def unpack(chunk, mask, first, st):
            return torch.as_tensor(np_unpack(chunk.numpy(), mask, first, st.numpy()))

        res, layout = shard.run_sharded(n, m, rank, slab, x, z, phi, shard.torch_exchange(dist), apply, pack, unpack,
                                        chunk_bits=2)
        out[rank] = (res.numpy(), layout.tolist())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4, 8])
def test_gloo_ranks_exchange_parts(world):
    n = 8
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_gloo_rank, args=(world, port, n, out), nprocs=world, join=True)
        got = np.concatenate([out[r][0] for r in range(world)])
        layout = out[0][1]
        assert all(out[r][1] == layout for r in range(world))
    x, z, phi = sequence(n, 40 + n)
    ref = oracle.apply(inputs.gaussian_state(n, 8), x, z, phi)
    assert np.max(np.abs(to_logical(got, layout) - ref)) < 1e-13


# ------------------------------------------------- ranks emulated on a GPU

@pytest.mark.gpu
@pytest.mark.parametrize("dtype,tol", [(torch.complex128, 1e-12), (torch.complex64, 1e-5)])
def test_ranks_emulated_on_one_gpu_with_libps(dtype, tol):
    """Eight ranks on one GPU: every window through libps's tile and pair
    kernels on the rank's slab (one StateVector per slab, so the carried scale
    is the same on every rank), every exchange through the pack / unpack
    kernels in chunks, the chunks routed between the ranks' device buffers."""
    n, m = 16, 3
    s = n - m
    x, z, h = inputs.jw_hamiltonian(n, 200, seed=51)
    xs, zs, ph = oracle.qdrift_stream(x, z, h, 0.8, 400, 5)
    psi = inputs.gaussian_state(n, 52)
    pdt = ps.PS_C64 if dtype == torch.complex64 else ps.PS_C128
    pack, unpack = shard.libps_moves(s, pdt)
    R = 1 << m
    svs = [ps.StateVector(s, tensor=torch.as_tensor(psi[r << s:(r + 1) << s]).to(dtype).cuda()) for r in range(R)]
    plans = [ps.ps_shard_swap_plan(n, m, m, r, xs, zs, ph) for r in range(R)]
    layout = plans[0][1]
    chunk = 1 << 9
    for t in range(len(plans[0][0])):
        st = plans[0][0][t]
        if st[0] == "window":
            for r in range(R):
                if len(plans[r][0][t][3]):
                    svs[r].apply_rotations(*plans[r][0][t][1:])
            continue
        _, rank_mask, slab_mask = st
        part = 1 << (s - bin(rank_mask).count("1"))
        rounds = [shard.exchange_rounds(r, s, rank_mask) for r in range(R)]
        for q in range(len(rounds[0])):
            for c0 in range(0, part, min(chunk, part)):
                cnt = min(chunk, part)
                sent = [pack(svs[r].tensor, slab_mask, rounds[r][q][1] * part + c0, cnt) for r in range(R)]
                for r in range(R):
                    unpack(sent[rounds[r][q][0]], slab_mask, rounds[r][q][1] * part + c0, svs[r].tensor)
    assert len({sv.scale() for sv in svs}) == 1
    got = to_logical(np.concatenate([sv.to_numpy() for sv in svs]), layout)
    ref = oracle.apply(psi, xs, zs, ph)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < tol
