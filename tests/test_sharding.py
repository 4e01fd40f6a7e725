"""Host logic of multi-GPU batches: instance partition over ranks and the
waveform gather, run as world_size-2 gloo ranks on the CPU (no GPU)."""
import os
import socket

import numpy as np
import pytest

from paper_0909_4039_gb300 import inputs, sharding


def test_partition_covers_every_instance_once_and_balances():
    ws = inputs.batched_instances(64, seed=0)
    pts = [w.points for w in ws]
    for n in (1, 2, 3, 4, 8):
        parts = sharding.partition(pts, n)
        flat = sorted(k for p in parts for k in p)
        assert flat == list(range(64))
        loads = [sum(pts[k] for k in p) for p in parts]
        assert max(loads) - sum(pts) / n <= max(pts)          # LPT bound
        assert sharding.partition(pts, n) == parts             # same on every rank
    assert sharding.partition([5.0, 5.0, 5.0], 3) == [[0], [1], [2]]
    assert sharding.partition([1.0, 2.0, 3.0], 1) == [[0, 1, 2]]
    assert sharding.partition([], 4) == [[], [], [], []]
    with pytest.raises(ValueError):
        sharding.partition([1.0], 0)


def test_gather_without_process_group_is_local():
    assert sharding.gather_waveforms({3: "x"}) == {3: "x"}


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ws = inputs.batched_instances(64, seed=0)
    mine = sharding.local_instances([w.points for w in ws], rank, world)
    # a stand-in waveform per instance, a function of the instance only
    local = {k: np.arange(4, dtype=np.complex128) * (k + 1) + 1j * ws[k].m for k in mine}
    merged = sharding.gather_waveforms(local)
    np.save(os.path.join(out_dir, f"rank{rank}.npy"),
            np.array([len(mine), len(merged)] + sorted(merged), dtype=np.int64))
    ok = all(np.array_equal(merged[k], np.arange(4) * (k + 1) + 1j * ws[k].m) for k in range(64))
    np.save(os.path.join(out_dir, f"ok{rank}.npy"), np.array([ok]))
    # a second gather in which both ranks claim instance 0 must fail
    try:
        sharding.gather_waveforms({0: 1})
        dup = False
    except RuntimeError:
        dup = True
    np.save(os.path.join(out_dir, f"dup{rank}.npy"), np.array([dup]))
    dist.destroy_process_group()


def test_two_gloo_ranks_split_the_batch_and_gather_all_waveforms(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r0 = np.load(tmp_path / "rank0.npy")
    r1 = np.load(tmp_path / "rank1.npy")
    assert r0[0] + r1[0] == 64 and r0[0] > 0 and r1[0] > 0
    assert r0[1] == 64 and r1[1] == 64
    assert list(r0[2:]) == list(range(64)) and list(r1[2:]) == list(range(64))
    assert np.load(tmp_path / "ok0.npy")[0] and np.load(tmp_path / "ok1.npy")[0]
    assert np.load(tmp_path / "dup0.npy")[0] and np.load(tmp_path / "dup1.npy")[0]
