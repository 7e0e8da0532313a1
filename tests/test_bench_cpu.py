"""bench.py's whole-job figure on host ranks (gloo, 127.0.0.1): the slowest rank's time and
the units of all ranks; one rank without a process group reports its own."""
import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, outdir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, rate = bench.whole_job_rate(10.0 * (rank + 1), 1000 * (rank + 1), "cpu")
    with open(os.path.join(outdir, f"r{rank}.json"), "w") as f:
        json.dump({"ms": ms, "rate": rate}, f)
    dist.destroy_process_group()


def test_whole_job_rate_two_ranks(tmp_path):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for r in range(2):
        d = json.load(open(tmp_path / f"r{r}.json"))
        assert d["ms"] == 20.0                      # the slowest rank
        assert abs(d["rate"] - 3000 / 0.020) < 1e-6  # both ranks' units over that time


def test_whole_job_rate_one_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job_rate(4.0, 8000, "cpu") == (4.0, 8000 / 0.004)


def test_kernel_bytes_match_the_stored_formats():
    """The roofline's algorithmic bytes per site: K1 reads p and the four links and writes t;
    K2 reads t, p, r and psi and the links and writes psi and r (psi in FP32 beside scaled-FP16
    vectors); K3 reads r and p and writes p.  Spinor sites: FP32 96 B, scaled FP16 48 + 4 B,
    FP64 192 B; four 12-real links: FP32 192 B, FP16 96 B."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.kernel_bytes("mixed_f16") == {"K1": 52 + 96 + 52, "K2": 4 * 52 + 2 * 96 + 96, "K3": 3 * 52}
    assert bench.kernel_bytes("mixed_f32") == {"K1": 96 + 192 + 96, "K2": 6 * 96 + 192, "K3": 3 * 96}
    assert bench.kernel_bytes("f64")["K1"] == 192 + 576 + 192


def test_traffic_record_follows_the_kernel_sources(monkeypatch):
    """roofline.traffic comes from the committed ncu record only while the inner-loop kernel
    sources hash to the value it was captured on; any other hash gives None (no stale
    counters), and a role the record does not hold gives None."""
    sys.path.insert(0, ROOT)
    import bench
    rec = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
    monkeypatch.setattr(bench, "source_hash", lambda: rec["source_hash"])
    for role in ("K1", "K2"):
        assert bench.ncu_traffic(role) == rec["kernels"][role]["dram_bytes_per_launch_full_size"]
    assert bench.ncu_traffic("K9") is None
    monkeypatch.setattr(bench, "source_hash", lambda: "0" * 16)
    assert bench.ncu_traffic("K2") is None


def test_source_hash_covers_every_kernel_source(tmp_path, monkeypatch):
    """The hash changes when any one of the files the inner-loop kernels are built from
    changes, and only then."""
    import shutil
    sys.path.insert(0, ROOT)
    import bench
    src = os.path.join(ROOT, "paper_1904_08616_gb300", "csrc")
    dst = tmp_path / "paper_1904_08616_gb300" / "csrc"
    dst.mkdir(parents=True)
    for fn in bench.KERNEL_SOURCES:
        shutil.copy(os.path.join(src, fn), dst / fn)
    base = bench.source_hash()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.source_hash() == base
    for fn in bench.KERNEL_SOURCES:
        orig = (dst / fn).read_bytes()
        (dst / fn).write_bytes(orig + b"\n")
        assert bench.source_hash() != base, fn
        (dst / fn).write_bytes(orig)
    assert bench.source_hash() == base
