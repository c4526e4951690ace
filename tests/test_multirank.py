"""The host side of the multi-GPU path on CPU: two gloo ranks run the
benchmark's replica logic (barriers, the max of the ranks' timings, the
sharding of the serving stream and the merge of its results).  One process
per GPU with no data-path collective: each rank steps its own replica."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import torch.distributed as dist
    import bench
    d, r, w = bench._dist(backend="gloo")
    assert (r, w) == (rank, ws)
    res = {"max": bench._max_over_ranks(torch, d, 1.5 * (rank + 1), device="cpu"),
           "shard": bench._shard(range(7), rank, ws)}
    lat = [0.1 * (rank + 1), 0.2 * (rank + 1)]
    res["merged"] = bench._combine_serving(d, lat, 10.0 + rank, 100 * (rank + 1), rank + 1)
    d.barrier()
    dist.destroy_process_group()
    out.put((rank, res))


def test_two_gloo_ranks_replica_logic():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got[0]["max"] == got[1]["max"] == 3.0
    assert got[0]["shard"] == [0, 2, 4, 6] and got[1]["shard"] == [1, 3, 5]
    for r in (0, 1):
        lat, span, cvu, conv = got[r]["merged"]
        assert np.allclose(sorted(lat), [0.1, 0.2, 0.2, 0.4])
        assert span == 11.0 and cvu == 300 and conv == 3
