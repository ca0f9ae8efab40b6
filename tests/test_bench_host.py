"""Host logic of bench.py without a GPU: the multi-rank path on two gloo ranks
and the roofline's traffic record.

Under torchrun every rank solves its own problem (weak scaling, no collective
on the data path); the ranks only agree on the slowest time.  The reference
arm runs on rank 0 alone.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    slowest = bench.max_over_ranks(1.5 + rank, "cpu")
    w = bench.rank_workload(bench.inputs.WORKLOADS["sdmm64"], rank)
    out[rank] = (slowest, w.seed)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_agree_on_the_slowest_time_and_draw_independent_problems():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 2.5
    assert res[0][1] != res[1][1]


def test_reference_arm_prints_on_rank_zero_only(capsys, monkeypatch):
    import bench

    monkeypatch.setenv("RANK", "1")
    ns = type("Args", (), {"steps": 1, "warmup": 0, "gpus": 2})()
    bench.run_reference(ns, bench.inputs.WORKLOADS["sdmm64"])
    assert capsys.readouterr().out == ""


def test_traffic_record_follows_the_kernel_source(tmp_path, monkeypatch):
    """The roofline's DRAM traffic comes from a committed ncu record and turns
    to null when the kernel's source file no longer matches the record."""
    import hashlib

    import bench

    prof = tmp_path / "profiles"
    prof.mkdir()
    csrc = tmp_path / "paper_1307_4370_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "gridding.cu").write_text("kernel v1\n")
    sha = hashlib.sha256(b"kernel v1\n").hexdigest()
    (prof / "dram_traffic.txt").write_text(f"# comment\nsdmm256 grid 1234 {sha}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.dram_traffic("sdmm256", "grid") == 1234
    assert bench.dram_traffic("sdmm1024", "grid") is None
    assert bench.dram_traffic("sdmm256", "nosuch") is None
    (csrc / "gridding.cu").write_text("kernel v2\n")
    assert bench.dram_traffic("sdmm256", "grid") is None


def test_gram_algorithmic_bytes():
    """The roofline's algorithmic bytes of the Gram pass (G^T G per CG step):
    the grid read and the grid written (2 x (2n)^2 complex64 = 8Nc) and the
    frequencies once (8 B per visibility); for the 1024^2, M = 2^21 workload
    83,886,080 B, for 256^2, M = 65536, 4,718,592 B."""
    import bench
    from paper_1307_4370_gb300 import inputs

    assert bench.algorithmic_bytes(inputs.WORKLOADS["sdmm1024"])["gram"] == 83886080
    assert bench.algorithmic_bytes(inputs.WORKLOADS["sdmm256"])["gram"] == 4718592
