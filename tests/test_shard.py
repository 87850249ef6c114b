"""Sharding of a batch over ranks (CPU, gloo, world size 2): every element
runs on exactly one rank, the split balances atoms x steps, and the results
come back to rank 0 in the batch's order."""
import os

import numpy as np
import pytest
import torch.multiprocessing as tmp

import synth
from paper_1603_04628_gb300 import shard


def test_partition_covers_and_balances():
    els = synth.batch_uneven(64, steps=1000)
    for world in (1, 2, 3, 8):
        parts = shard.partition(els, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(els)))
        loads = [sum(shard.element_work(els[i]) for i in p) for p in parts]
        biggest = max(shard.element_work(e) for e in els)
        assert max(loads) - min(loads) <= biggest        # LPT bound
    with pytest.raises(ValueError):
        shard.partition(els, 0)


def _fake_result(el, i):
    return {"q": float(i) + el["h"], "q_se": 0.1, "p": 2.0, "p_se": 0.01, "T_meas": 1.1, "e_drift": 0.0,
            "n_fluid": i, "n_wall": 7, "status": 0}


def _worker(rank, world, port, els, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    parts = shard.partition(els, world)
    mine = parts[rank]
    local = [_fake_result(els[i], i) for i in mine]
    full = shard.gather_results(local, mine, len(els), dist)
    if rank == 0:
        np.save(out_path, np.array([[r["q"], r["n_fluid"]] for r in full]))
    dist.barrier()
    dist.destroy_process_group()


def test_gather_over_two_gloo_ranks(tmp_path):
    els = synth.batch_uneven(13, steps=100)
    out = str(tmp_path / "gathered.npy")
    port = 29500 + os.getpid() % 1000
    tmp.start_processes(_worker, args=(2, port, els, out), nprocs=2, join=True, start_method="spawn")
    got = np.load(out)
    expect = np.array([[i + e["h"], i] for i, e in enumerate(els)])
    np.testing.assert_allclose(got, expect)
