"""Host logic of the r* slab decomposition of one grid (no GPU): slab
geometry, the halo copy plan, and the distributed halo exchange as gloo
ranks.

The stand-in for the step has the step's reach and boundary behaviour: a
row-local operation in theta (the implicit angular stage) on every row but
the first and last of the array it is applied to (the step's boundary
rows), then a three-row stencil in r* after which those two rows are zero.
Slabs stepped halo - 1 steps at a time with their halo rows refreshed in
between must then reproduce every owned row of the whole-grid run bit for
bit, whatever the number of slabs, the halo width and the step count.
"""
import os
import socket

import numpy as np
import pytest

from paper_0909_4039_gb300 import slabs


def _stencil_step(u):
    """One stand-in step of a [2, rows, N] complex array; rows 0 and -1 -> 0."""
    out = np.zeros_like(u)
    c = 0.2 + 0.05j
    # row-local theta coupling on the non-boundary rows, then a three-row r* stencil
    v = u.copy()
    v[:, 1:-1] = u[:, 1:-1] + 0.1 * np.roll(u[:, 1:-1], 1, axis=2) - 0.1j * u[::-1, 1:-1]
    out[:, 1:-1] = v[:, 1:-1] + c * (v[:, :-2] - 2.0 * v[:, 1:-1] + v[:, 2:])
    return out


def _global(u0, n):
    u = u0.copy()
    for _ in range(n):
        u = _stencil_step(u)
    return u


def _u0(Nr, N, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.standard_normal((2, Nr, N)) + 1j * rng.standard_normal((2, Nr, N))
    u[:, 0] = u[:, -1] = 0.0
    return u


def test_slab_bounds_cover_the_grid_with_halos():
    for Nr, n, h in [(257, 3, 2), (100, 1, 1), (64, 4, 1), (1000, 7, 3)]:
        g = slabs.slab_bounds(Nr, n, h)
        assert g[0].a == 0 and g[-1].b == Nr
        assert all(x.b == y.a for x, y in zip(g[:-1], g[1:]))
        assert g[0].hl == 0 and g[-1].hr == 0
        assert all(x.hr == h for x in g[:-1]) and all(x.hl == h for x in g[1:])
        assert max(x.b - x.a for x in g) - min(x.b - x.a for x in g) <= 1
        for x in g:
            assert x.rows == x.b - x.a + x.hl + x.hr and x.g0 == x.a - x.hl
    with pytest.raises(ValueError):
        slabs.slab_bounds(5, 3, 2)
    with pytest.raises(ValueError):
        slabs.slab_bounds(100, 2, 0)


@pytest.mark.parametrize("Nr,nslabs,halo,steps", [(60, 3, 2, 7), (61, 3, 3, 9), (97, 4, 4, 10), (40, 2, 3, 5),
                                                  (50, 1, 2, 4)])
def test_slabs_with_halo_plan_reproduce_the_whole_grid(Nr, nslabs, halo, steps):
    u0 = _u0(Nr, 6, seed=Nr + 31 * halo)
    ref = _global(u0, steps)
    geoms = slabs.slab_bounds(Nr, nslabs, halo)
    plan = slabs.halo_plan(geoms, halo)
    parts = [u0[:, g.g0:g.g0 + g.rows].copy() for g in geoms]
    left = steps
    while left > 0:
        k = min(slabs.steps_per_exchange(halo), left)
        for _ in range(k):
            parts = [_stencil_step(p) for p in parts]
        for src, srows, dst, drows in plan:
            parts[dst][:, drows] = parts[src][:, srows]
        left -= k
    got = np.concatenate([p[:, slabs.local_rows(g)] for g, p in zip(geoms, parts)], axis=1)
    assert np.array_equal(got, ref)


def test_halo_plan_misses_a_stale_row_if_halo_is_too_thin():
    """The plan's invariant is load-bearing: with two halo rows but two steps
    between exchanges (one more than they allow) the slabs no longer
    reproduce the whole grid."""
    Nr, halo, steps = 60, 2, 6
    u0 = _u0(Nr, 6, seed=5)
    ref = _global(u0, steps)
    geoms = slabs.slab_bounds(Nr, 3, halo)
    plan = slabs.halo_plan(geoms, halo)
    parts = [u0[:, g.g0:g.g0 + g.rows].copy() for g in geoms]
    for _ in range(steps // 2):
        for _ in range(2):
            parts = [_stencil_step(p) for p in parts]
        for src, srows, dst, drows in plan:
            parts[dst][:, drows] = parts[src][:, srows]
    got = np.concatenate([p[:, slabs.local_rows(g)] for g, p in zip(geoms, parts)], axis=1)
    assert not np.array_equal(got, ref)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir, Nr, halo, steps):
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    geoms = slabs.slab_bounds(Nr, world, halo)
    g = geoms[rank]
    u0 = _u0(Nr, 5, seed=77)
    mine = torch.from_numpy(u0[:, g.g0:g.g0 + g.rows].copy())
    left = steps
    while left > 0:
        k = min(slabs.steps_per_exchange(halo), left)
        arr = mine.numpy()
        for _ in range(k):
            arr = _stencil_step(arr)
        mine = torch.from_numpy(arr.copy())
        slabs.exchange_halos_dist(mine, g, halo, rank, world)
        left -= k
    np.save(os.path.join(out_dir, f"slab{rank}.npy"), mine.numpy()[:, slabs.local_rows(g)])
    dist.destroy_process_group()


@pytest.mark.parametrize("world,halo", [(2, 3), (3, 2)])
def test_gloo_ranks_exchange_halos_and_reproduce_the_whole_grid(tmp_path, world, halo):
    import torch.multiprocessing as mp
    Nr, steps = 48, 7
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path), Nr, halo, steps), nprocs=world, join=True,
                       start_method="spawn")
    got = np.concatenate([np.load(tmp_path / f"slab{r}.npy") for r in range(world)], axis=1)
    assert np.array_equal(got, _global(_u0(Nr, 5, seed=77), steps))
