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


def np_pack(slab, slab_mask):
    pos = shard.set_bits(slab_mask)
    k, s = len(pos), slab.size.bit_length() - 1
    idx = np.arange(1 << s, dtype=np.int64)
    at = _insert(idx & ((1 << (s - k)) - 1), idx >> (s - k), pos)
    return list(slab[at].reshape(1 << k, -1))


def np_unpack(parts, slab_mask, slab):
    pos = shard.set_bits(slab_mask)
    k, s = len(pos), slab.size.bit_length() - 1
    idx = np.arange(1 << s, dtype=np.int64)
    at = _insert(idx & ((1 << (s - k)) - 1), idx >> (s - k), pos)
    out = np.empty_like(slab)
    out[at] = np.concatenate(parts)
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


def emulate(n, m, psi, x, z, phi, apply, pack, unpack, k_max, layout=None):
    """All 2^m ranks in lockstep: windows on every slab, exchanges between them.
    psi is in the physical order of `layout` (identity when None)."""
    s, R = n - m, 1 << m
    slabs = [psi[r << s:(r + 1) << s].copy() for r in range(R)]
    plans = [ps.ps_shard_swap_plan(n, m, k_max, r, x, z, phi, layout) for r in range(R)]
    layout = plans[0][1]
    assert all(np.array_equal(p[1], layout) for p in plans)
    nsteps = len(plans[0][0])
    for t in range(nsteps):
        st = plans[0][0][t]
        if st[0] == "window":
            slabs = [apply(slabs[r], *plans[r][0][t][1:]) if len(plans[r][0][t][3]) else slabs[r] for r in range(R)]
        else:
            _, rank_mask, slab_mask = st
            parts = [pack(slabs[r], slab_mask) for r in range(R)]
            new = []
            for r in range(R):
                partners = shard.exchange_partners(r, s, rank_mask)
                # received[j] = part sent by partners[j] to r: that rank's part with index "r's swapped bits"
                mine = partners.index(r)
                new.append(unpack([parts[p][mine] for p in partners], slab_mask, slabs[r]))
            slabs = new
    return np.concatenate(slabs), layout


def _emulate_from(n, m, phys, x, z, phi, layout):
    return emulate(n, m, phys, x, z, phi, lambda st, a, b, c: oracle.apply(st, a, b, c), np_pack, np_unpack, 2,
                   layout)


@pytest.mark.parametrize("n,m,k_max", [(6, 1, 1), (7, 2, 1), (7, 2, 2), (8, 3, 1), (8, 3, 3)])
def test_swap_plan_reproduces_single_state_evolution(n, m, k_max):
    x, z, phi = sequence(n, 3 * n + m)
    psi = inputs.gaussian_state(n, 7)
    got, layout = emulate(n, m, psi, x, z, phi, lambda st, a, b, c: oracle.apply(st, a, b, c), np_pack, np_unpack,
                          k_max)
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

        def pack(st, mask):
            return [torch.as_tensor(p.copy()) for p in np_pack(st.numpy(), mask)]

        def unpack(parts, mask, st):
            return torch.as_tensor(np_unpack([p.numpy() for p in parts], mask, st.numpy()))

        res, layout = shard.run_sharded(n, m, rank, slab, x, z, phi, shard.torch_exchange(dist), apply, pack, unpack)
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
    """Every window through libps's tile and pair kernels on the rank's slab,
    every exchange through the pack / unpack kernels."""
    n, m = 16, 3
    s = n - m
    x, z, h = inputs.jw_hamiltonian(n, 200, seed=51)
    xs, zs, ph = ps.Hamiltonian(n, x, z, h).qdrift_stream(0.8, 400, 5)
    psi = inputs.gaussian_state(n, 52)
    pdt = ps.PS_C64 if dtype == torch.complex64 else ps.PS_C128
    pack, unpack = shard.libps_moves(s, pdt)
    states = {}

    def apply(st, a, b, c):
        sv = states.setdefault(st.data_ptr(), ps.StateVector(s, tensor=st))
        sv.apply_rotations(a, b, c)
        return st

    def gpu_pack(st, mask):
        # a windowed slab carries its own stored scale: fold it in before the amplitudes move
        sv = states.pop(st.data_ptr(), None)
        if sv is not None:
            st = torch.as_tensor(sv.to_numpy()).to(dtype).cuda()
        return pack(st, mask)

    R = 1 << m
    slabs = [torch.as_tensor(psi[r << s:(r + 1) << s]).to(dtype).cuda() for r in range(R)]
    plans = [ps.ps_shard_swap_plan(n, m, m, r, xs, zs, ph) for r in range(R)]
    layout = plans[0][1]
    for t in range(len(plans[0][0])):
        st = plans[0][0][t]
        if st[0] == "window":
            for r in range(R):
                if len(plans[r][0][t][3]):
                    slabs[r] = apply(slabs[r], *plans[r][0][t][1:])
        else:
            _, rank_mask, slab_mask = st
            parts = [gpu_pack(slabs[r], slab_mask) for r in range(R)]
            for r in range(R):
                partners = shard.exchange_partners(r, s, rank_mask)
                mine = partners.index(r)
                slabs[r] = unpack([parts[p][mine] for p in partners], slab_mask,
                                  torch.empty_like(parts[r][0]).repeat(len(partners)))
    out = []
    for r in range(R):
        sv = states.get(slabs[r].data_ptr())
        out.append(sv.to_numpy() if sv is not None else slabs[r].cpu().numpy().astype(np.complex128))
    got = to_logical(np.concatenate(out), layout)
    ref = oracle.apply(psi, xs, zs, ph)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < tol
