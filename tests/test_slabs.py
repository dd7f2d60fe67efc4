"""The z-slab exchange plan (hbe_slab_plan, a host function of libhbe) and its
execution between torch.distributed ranks, on CPU with gloo.

After one exchange every slab's two halo planes on each side must hold the
two grid planes beyond it: the neighbouring slab's planes, the other end of
the grid when periodic, zeros at a zero-Dirichlet wall (the zero ghost
layers of Eq. BC that an undivided grid reads there)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import __graft_entry__  # noqa: F401

H = 2


def slabs_mod():
    try:
        from paper_1803_01291_gb300 import slabs
        slabs.plan(8, 1, False)
    except (ImportError, OSError) as e:
        pytest.skip(f"libhbe not built: {e}")
    return slabs


def expected_halos(g, z0, nz, periodic):
    """Planes z0-2, z0-1 and z0+nz, z0+nz+1 of the global array g (wrapped
    or zero outside)."""
    N = g.shape[0]
    out = []
    for z in (z0 - 2, z0 - 1, z0 + nz, z0 + nz + 1):
        if 0 <= z < N:
            out.append(g[z])
        elif periodic:
            out.append(g[z % N])
        else:
            out.append(np.zeros_like(g[0]))
    return np.stack(out)


def split(g, nz):
    """Stored blocks (nz_i + 4 planes, halos zero) of the global array."""
    blocks, z0 = [], 0
    for n in nz:
        b = np.zeros((n + 2 * H,) + g.shape[1:])
        b[H:H + n] = g[z0:z0 + n]
        blocks.append(b)
        z0 += n
    return blocks


@pytest.mark.parametrize("N,k", [(16, 1), (16, 2), (17, 3), (20, 4), (8, 4)])
@pytest.mark.parametrize("periodic", [False, True])
def test_plan_fills_every_halo(N, k, periodic):
    slabs = slabs_mod()
    nz, copies = slabs.plan(N, k, periodic)
    assert sum(nz) == N and len(nz) == k and min(nz) >= 2 and max(nz) - min(nz) <= 1
    assert len(copies) == (2 * k if periodic else 2 * k - 2)
    rng = np.random.default_rng(N * 10 + k)
    g = rng.standard_normal((N, 5, 3))
    blocks = split(g, nz)
    for src, dst, sp, dp in copies:  # the transfers, as plain array copies
        assert H <= sp and sp + H <= nz[src] + H
        assert dp in (0, nz[dst] + H)
        blocks[dst][dp:dp + H] = blocks[src][sp:sp + H]
    z0 = 0
    for i, n in enumerate(nz):
        b = blocks[i]
        got = np.concatenate([b[:H], b[H + n:]])
        assert np.array_equal(got, expected_halos(g, z0, n, periodic)), (i, periodic)
        assert np.array_equal(b[H:H + n], g[z0:z0 + n])  # interiors untouched
        z0 += n


def test_plan_rejects_thin_slabs():
    slabs = slabs_mod()
    with pytest.raises(ValueError):
        slabs.plan(7, 4, False)
    with pytest.raises(ValueError):
        slabs.plan(16, 0, True)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, N, periodic, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1803_01291_gb300 import slabs
    nz, copies = slabs.plan(N, world, periodic)
    g = np.random.default_rng(7).standard_normal((N, 6, 4))
    z0 = sum(nz[:rank])
    local = torch.zeros((nz[rank] + 2 * H, 6, 4), dtype=torch.float64)
    local[H:H + nz[rank]] = torch.from_numpy(g[z0:z0 + nz[rank]])
    slabs.exchange_halos(local, rank, copies)
    b = local.numpy()
    ok = np.array_equal(np.concatenate([b[:H], b[H + nz[rank]:]]),
                        expected_halos(g, z0, nz[rank], periodic))
    ok = ok and np.array_equal(b[H:H + nz[rank]], g[z0:z0 + nz[rank]])
    q.put((rank, bool(ok)))
    dist.destroy_process_group()


@pytest.mark.parametrize("world,N", [(2, 12), (4, 19)])
@pytest.mark.parametrize("periodic", [False, True])
def test_exchange_between_gloo_ranks(world, N, periodic):
    slabs_mod()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, N, periodic, q))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    assert got == [(r, True) for r in range(world)]
