"""The N>1 path on CPU: two gloo ranks on 127.0.0.1.

* the benchmark's whole-job figures: max over ranks of the timings, sum of the
  work counts;
* replicated rendering: renders sharded over the ranks (each index on exactly
  one rank, loads balanced), rendered independently -- here by the FP64
  oracle on a few pixels -- and gathered on rank 0 identical to a
  single-process run;
* replicas with different render ids draw different random streams.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1912_06474_gb300 import replicas, scenes
    import oracle

    res = {}
    mx, sm = bench.reduce_over_ranks([10.0 * (rank + 1), 3.0 - rank], [100 + rank, 7])
    res["max"], res["sum"] = mx, sm

    sc = scenes.tiny_room(L=16, seed=0)
    specs = [scenes.RenderSpec(w, h, spp, 2, seed=0, camera=sc.camera)
             for w, h, spp in ((8, 8, 1), (16, 8, 2), (8, 4, 1), (12, 12, 1), (4, 4, 4))]
    for i, sp in enumerate(specs):
        sp.render_id = i
    mine = replicas.my_renders(specs, rank, world)
    res["mine"] = mine
    orc = oracle.Oracle(sc)
    local = {i: orc.render_pixels(specs[i], np.arange(8), n_threads=1)["xyz"] for i in mine}
    allimg = replicas.gather_images(local, len(specs))
    if rank == 0:
        np.save(os.path.join(out_dir, "gathered.npy"), np.stack(allimg))
    # a replica of render 0 with this rank's render id
    rep = scenes.RenderSpec(8, 8, 1, 2, seed=0, camera=sc.camera)
    rep.render_id = rank
    res["replica"] = orc.render_pixels(rep, np.arange(8), n_threads=1)["xyz"].tolist()
    np.save(os.path.join(out_dir, f"res{rank}.npy"), np.array(res, dtype=object), allow_pickle=True)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path, oracle_mod):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn",
                       join=True)
    res = [np.load(os.path.join(tmp_path, f"res{r}.npy"), allow_pickle=True).item() for r in range(world)]
    for r in res:
        assert r["max"] == [20.0, 3.0]
        assert r["sum"] == [201, 14]
    # each render on exactly one rank
    owned = sorted(res[0]["mine"] + res[1]["mine"])
    assert owned == [0, 1, 2, 3, 4]
    assert not set(res[0]["mine"]) & set(res[1]["mine"])
    # gathered images equal a single-process run of every render
    from paper_1912_06474_gb300 import scenes
    sc = scenes.tiny_room(L=16, seed=0)
    orc = oracle_mod.Oracle(sc)
    got = np.load(os.path.join(tmp_path, "gathered.npy"))
    for i, (w, h, spp) in enumerate(((8, 8, 1), (16, 8, 2), (8, 4, 1), (12, 12, 1), (4, 4, 4))):
        sp = scenes.RenderSpec(w, h, spp, 2, seed=0, camera=sc.camera)
        sp.render_id = i
        assert np.array_equal(got[i], orc.render_pixels(sp, np.arange(8), n_threads=1)["xyz"])
    # replicas with different render ids are different sample streams
    a, b = np.array(res[0]["replica"]), np.array(res[1]["replica"])
    assert not np.array_equal(a, b)


def test_shard_balance():
    from paper_1912_06474_gb300 import replicas
    rng = np.random.default_rng(0)
    costs = rng.choice([128 ** 2, 256 ** 2, 512 ** 2, 1024 ** 2], 64) * rng.choice([4, 16, 64], 64)
    for world in (1, 2, 3, 8):
        parts = replicas.shard_renders(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(64))
        loads = [int(sum(costs[i] for i in p)) for p in parts]
        # longest-first greedy: the heaviest rank is within one job of the mean
        assert max(loads) <= sum(loads) / world + max(costs)
