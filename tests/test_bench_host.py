"""Host logic of bench.py: multi-rank (replica) runs on CPU with gloo at
world size 2 (the step time is the maximum over ranks and the reported
value counts the points of every rank), and the rule that the roofline's
DRAM traffic is reported only for the kernel source it was measured on."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, world)  # rank 1 is the slow one
        value = bench.whole_job_value(world, 1000, ms / 1000.0)
        out.put((rank, ms, value))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]
    assert res[0][2] == pytest.approx(2 * 1000 / 0.015)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_value(1, 100, 0.5) == 200.0


def test_traffic_is_reported_only_for_the_source_it_was_measured_on(tmp_path, monkeypatch):
    """The roofline's DRAM traffic comes from a committed ncu summary and is
    dropped (null) once the kernel source differs from the one measured."""
    import hashlib
    import json
    sys.path.insert(0, ROOT)
    import bench
    src = tmp_path / "kern.cu"
    src.write_text("// kernel v1\n")
    (tmp_path / "profiles").mkdir()
    entry = {"source": "kern.cu", "sha256": hashlib.sha256(src.read_bytes()).hexdigest(),
             "bytes_per_element": 24.5, "launches_per_step": 20}
    (tmp_path / "profiles" / "dram_traffic.json").write_text(json.dumps({"sort_pass": entry}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_for("sort_pass") == pytest.approx(24.5)
    assert bench.traffic_for("level_pass") is None
    src.write_text("// kernel v2\n")
    assert bench.traffic_for("sort_pass") is None
