"""Sharded schedule over 2^m ranks (ps_shard_plan, shard.run_sharded).

The plan is checked against the oracle's single-state evolution three ways:
all ranks emulated in one process with the oracle applying each window
(CPU), real gloo ranks exchanging slabs with torch.distributed (CPU, world
sizes 2 and 4), and all ranks emulated on one GPU with libps applying each
window (GPU).
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
    """Random strings plus JW-like terms, so windows mix local and paired rotations."""
    xr, zr, pr = inputs.random_rotations(n, 40, seed=seed)
    x, z, h = inputs.jw_hamiltonian(n, 30, seed=seed + 1)
    ang = np.random.default_rng(seed).uniform(-1, 1, size=30)
    return (np.concatenate([xr, x]), np.concatenate([zr, z]), np.concatenate([pr, ang]))


def emulate(n, m, psi, x, z, phi, apply):
    """All 2^m ranks in lockstep; every window reads the slabs before it."""
    s = n - m
    R = 1 << m
    slabs = [psi[r << s:(r + 1) << s].copy() for r in range(R)]
    plans = [ps.ps_shard_plan(n, m, r, x, z, phi) for r in range(R)]
    assert all(len(p) == len(plans[0]) for p in plans)
    for w in range(len(plans[0])):
        new = []
        for r in range(R):
            partner, xl, zl, pl = plans[r][w]
            if partner < 0:
                new.append(apply(slabs[r], xl, zl, pl))
            else:
                both = apply(np.concatenate([slabs[r], slabs[partner]]), xl, zl, pl)
                new.append(both[:1 << s])
        slabs = new
    return np.concatenate(slabs)


@pytest.mark.parametrize("n,m", [(5, 1), (6, 2), (7, 3), (6, 0)])
def test_plan_reproduces_single_state_evolution(n, m):
    x, z, phi = sequence(n, 3 * n + m)
    psi = inputs.gaussian_state(n, 7)
    got = emulate(n, m, psi, x, z, phi, lambda st, a, b, c: oracle.apply(st, a, b, c))
    ref = oracle.apply(psi, x, z, phi)
    assert np.max(np.abs(got - ref)) < 1e-13


def test_plan_windows_and_validation():
    n, m = 6, 2
    s = n - m
    # three rotations pairing with top part 1, then a local one, then top part 2
    x = [1 << s, (1 << s) | 3, 5, 2 << s]
    z = [0, 1 << s, 2, 0]
    phi = [0.1, 0.2, 0.3, 0.4]
    plan = ps.ps_shard_plan(n, m, 1, x, z, phi)
    assert [p[0] for p in plan] == [1 ^ 1, 1 ^ 2]  # partners: rank ^ X
    assert [len(p[3]) for p in plan] == [3, 1]
    # the local masks of a paired rotation flip the local top bit
    assert int(plan[0][1][0]) == 1 << s
    with pytest.raises(ps.PsError):
        ps.ps_shard_plan(n, m, 4, x, z, phi)
    with pytest.raises(ps.PsError):
        ps.ps_shard_plan(n, n, 0, x, z, phi)
    with pytest.raises(ps.PsError):
        ps.ps_shard_plan(n, m, 0, [1 << n], [0], [0.1])


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

        res = shard.run_sharded(n, m, rank, slab, x, z, phi, shard.torch_exchange(dist), apply,
                                lambda own, other: torch.cat([own, other]), lambda both: both[:1 << s].clone())
        out[rank] = res.numpy()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_gloo_ranks_exchange_slabs(world):
    n = 7
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_gloo_rank, args=(world, port, n, out), nprocs=world, join=True)
        got = np.concatenate([out[r] for r in range(world)])
    x, z, phi = sequence(n, 40 + n)
    ref = oracle.apply(inputs.gaussian_state(n, 8), x, z, phi)
    assert np.max(np.abs(got - ref)) < 1e-13


@pytest.mark.gpu
@pytest.mark.parametrize("dtype,tol", [(torch.complex128, 1e-12), (torch.complex64, 1e-5)])
def test_ranks_emulated_on_one_gpu_with_libps(dtype, tol):
    # each window of each emulated rank runs through the library's kernels
    n, m = 14, 2
    x, z, h = inputs.jw_hamiltonian(n, 200, seed=51)
    xs, zs, ph = ps.Hamiltonian(n, x, z, h).qdrift_stream(0.8, 400, 5)
    psi = inputs.gaussian_state(n, 52)

    def apply(st, a, b, c):
        k = int(np.log2(st.size))
        sv = ps.StateVector(k, tensor=torch.as_tensor(st).to(dtype).cuda())
        sv.apply_rotations(a, b, c)
        return sv.to_numpy()

    got = emulate(n, m, psi, xs, zs, ph, apply)
    ref = oracle.apply(psi, xs, zs, ph)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < tol
