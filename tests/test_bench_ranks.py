"""Host logic of the multi-process bench on the CPU (gloo, world size 2):
every rank advances its own seeded replica (different droplet offsets), the
timed interval is the maximum over ranks and the work the sum."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    from paper_1509_07691_gb300 import synthetic as S
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, _ = bench.dist_info()
    ms, nf = bench.reduce_over_ranks(10.0 + rank, 100 * (rank + 1), "cpu")
    c = S.workload("oscillating256", seed=S.SEED + r)["geometry"]["c"]
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out, f"rank{rank}.json"), "w") as f:
        json.dump(dict(ws=ws, rank=r, ms=ms, nf=nf, c=list(c)), f)


def test_two_gloo_ranks(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    assert [r["ws"] for r in res] == [2, 2] and [r["rank"] for r in res] == [0, 1]
    assert all(r["ms"] == 11.0 and r["nf"] == 300.0 for r in res)
    assert res[0]["c"] != res[1]["c"]  # independent replicas
