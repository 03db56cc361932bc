"""The N > 1 path of bench.py on the CPU: two gloo ranks (one process per
GPU in a real run; replicas with no data-path collective) exercise the
barrier, the slowest-rank timing and the whole-job rate, and the reference
arm runs on rank 0 only."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    import torch.distributed as dist
    w, r, local = bench.dist_setup(backend="gloo")
    steps = 5
    my_ms = 10.0 * (r + 1)                      # rank 1 is the slower replica
    bench.barrier(w, cuda=False)
    slowest = bench.max_over_ranks(w, my_ms, device="cpu")
    out.put((r, w, local, slowest, bench.whole_job_rate(w, steps, slowest)))
    bench.barrier(w, cuda=False)
    dist.destroy_process_group()


def test_two_gloo_ranks_slowest_rank_and_whole_job_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    assert [r[2] for r in res] == [0, 1]
    # every rank sees the slowest replica's 20 ms; 2 ranks x 5 solves in 20 ms
    assert all(r[3] == pytest.approx(20.0) for r in res)
    assert all(r[4] == pytest.approx(500.0) for r in res)


def test_single_process_rate_and_reference_arm_only_on_rank_zero(monkeypatch):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1, 12.5) == 12.5
    assert bench.whole_job_rate(1, 50, 1000.0) == pytest.approx(50.0)
    # a non-zero rank of the reference arm returns at once, without work or output
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps = 1
        warmup = 0
    called = []
    monkeypatch.setattr(bench, "cpu_oracle_baseline", lambda *a, **k: called.append(1))
    assert bench.run_reference(Args()) == 0
    assert not called


def test_replica_launch_spawns_or_refuses_on_a_mismatch():
    """`bench.py --gpus N` without a launcher starts N processes itself
    (torch.distributed.run, 127.0.0.1), runs in place under a launcher whose
    WORLD_SIZE is N, and exits with an error when the two differ."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_launch(1, {}) == ("run", None)
    how, cmd = bench.replica_launch(4, {})
    assert how == "spawn"
    assert cmd[1:3] == ["-m", "torch.distributed.run"]
    assert "--nproc-per-node=4" in cmd and "127.0.0.1" in cmd
    assert cmd[cmd.index("--master-addr") + 1] == "127.0.0.1"
    assert bench.replica_launch(2, {"WORLD_SIZE": "2"}) == ("run", None)
    how, msg = bench.replica_launch(8, {"WORLD_SIZE": "1"})
    assert how == "error" and "WORLD_SIZE=1" in msg


def test_roofline_bytes_and_recorded_traffic(monkeypatch):
    """The mode form's algorithmic bytes per launch, and the DRAM traffic of a
    committed ncu summary reported only while its kernel sources hash to the
    value written beside it."""
    import bench
    field, mc, nz = 128 * 128 * 1024 * 4, 400, 1024
    b = bench.mode_alg_bytes(128, 128, 1024, mc, 2)
    assert b["mode_project"] == field + 2 * mc * nz * 4
    assert b["mode_z"] == 2 * mc * nz * 4 + mc * (nz + 1) * 4 + mc * nz * 4
    assert b["mode_back"] == mc * nz * 4 + field
    monkeypatch.setattr(bench, "source_hash", lambda k: "0000000000000000")
    assert bench.recorded_traffic("mode_project") is None
    path = bench.os.path.join(bench.ROOT, "profiles", bench.PROFILE_FILES["mode_project"])
    text = open(path).read()
    recorded = text.split("mode_project_source_sha256: `")[1].split("`")[0]
    monkeypatch.setattr(bench, "source_hash", lambda k: recorded)
    assert bench.recorded_traffic("mode_project") > 0
