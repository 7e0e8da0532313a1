"""The domain-decomposition face exchange on host ranks (gloo, 127.0.0.1): faces reach the
right neighbours, and a rank that leaves without sending becomes an error on its
neighbour's host within the timeout (no GPU is involved)."""
import json
import os
import socket
import time

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, scenario, outdir):
    import torch
    import torch.distributed as dist
    from paper_1904_08616_gb300.halo import HaloError, exchange_faces
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    result = {"rank": rank}
    try:
        to_prev = torch.full((16,), 100.0 * rank + 1, dtype=torch.float64)
        to_next = torch.full((16,), 100.0 * rank + 2, dtype=torch.float64)
        from_next = torch.zeros(16, dtype=torch.float64)
        from_prev = torch.zeros(16, dtype=torch.float64)
        if scenario == "leave" and rank == 1:
            result["left"] = True
            return
        t0 = time.time()
        try:
            exchange_faces(to_prev, to_next, from_next, from_prev, timeout_s=3.0)
            result["from_next"] = from_next.tolist()
            result["from_prev"] = from_prev.tolist()
        except HaloError as e:
            result["error"] = str(e)
        result["seconds"] = time.time() - t0
    finally:
        with open(os.path.join(outdir, f"r{rank}.json"), "w") as f:
            json.dump(result, f)
        if scenario != "leave":
            dist.destroy_process_group()


def _run(world, scenario, tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_worker, args=(r, world, port, scenario, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
        if p.is_alive():
            p.kill()
            p.join()
    return [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]


@pytest.mark.parametrize("world", [2, 3])
def test_faces_reach_their_neighbours(tmp_path, world):
    res = _run(world, "exchange", tmp_path)
    for r in res:
        rank = r["rank"]
        nxt, prv = (rank + 1) % world, (rank - 1) % world
        assert "error" not in r, r
        assert all(v == 100.0 * nxt + 1 for v in r["from_next"])     # the next rank's to_prev
        assert all(v == 100.0 * prv + 2 for v in r["from_prev"])     # the previous rank's to_next


def test_missing_neighbour_is_an_error(tmp_path):
    res = _run(2, "leave", tmp_path)
    assert res[1].get("left")
    assert "error" in res[0] and "rank 0" in res[0]["error"]
    assert res[0]["seconds"] < 30


def test_slab_dims():
    from paper_1904_08616_gb300.halo import slab_dims
    assert slab_dims((4, 4, 4, 8), 4) == (4, 4, 4, 2)
    with pytest.raises(ValueError):
        slab_dims((4, 4, 4, 6), 4)
