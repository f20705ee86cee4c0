"""Scene sharding over ranks: LPT partition properties and a world-size-2
gloo run on CPU (the per-rank compute is the FP64 oracle, so the multi-rank
host path - partition, barrier, max-over-ranks, gather - is exercised
without a GPU)."""
import os
import socket
import sys

import numpy as np
import pytest

from paper_2603_14634_gb300.shard import lpt_partition

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_lpt_partition_complete_disjoint_balanced():
    rng = np.random.default_rng(0)
    sizes = rng.integers(27, 7000, size=300)
    for world in (1, 2, 3, 8):
        parts = lpt_partition(sizes, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        loads = [int(sum(sizes[p])) for p in parts]
        assert max(loads) - min(loads) <= int(sizes.max())


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    from oracle import oracle as O
    from paper_2603_14634_gb300 import scenes
    from paper_2603_14634_gb300.shard import gather_to_rank0, lpt_partition, max_over_ranks
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rng = np.random.default_rng(3)
    scs = [scenes.batch_scene(rng, max_bodies=4) for _ in range(6)]
    mine = lpt_partition([s.num_particles for s in scs], world)[rank]
    dist.barrier()
    out = {}
    for i in mine:
        o = O.OracleScene(scs[i]).substep(1)
        out[i] = o.x.copy()
    t = max_over_ranks(float(rank + 1), dist)
    got = gather_to_rank0(out, dist)
    stepped = gather_to_rank0(list(mine), dist)
    if rank == 0:
        # every scene of the batch is stepped by exactly one rank
        flat = [i for part in stepped for i in part]
        assert sorted(flat) == list(range(len(scs))), flat
        merged = {}
        for part in got:
            merged.update(part)
        assert sorted(merged) == list(range(len(scs)))
        for i, sc in enumerate(scs):
            ref = O.OracleScene(sc).substep(1).x
            assert np.array_equal(merged[i], ref)
        assert t == float(world)
        open(os.path.join(out_dir, "ok"), "w").write("ok")
    dist.destroy_process_group()


def test_two_rank_gloo_sharding(tmp_path, orc):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    assert (tmp_path / "ok").exists()
