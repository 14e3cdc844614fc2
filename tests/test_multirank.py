"""Host-side multi-process logic of the benchmark on CPU (gloo, world size 2):
the step has no exchange between boxes, so N GPUs run N independent replicas;
only the timing rule (barrier, max over ranks) crosses processes."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    bench.init_dist(world, "gloo")
    w, r, lr = bench.dist_env()
    bench.barrier(world)
    slowest = bench.max_over_ranks(10.0 + rank, world)
    # replicas draw their initial conditions from different seeds
    from paper_2410_20501_gb300 import inputs
    noise = inputs.white_noise(4, bench.SEED + r)
    q.put((r, w, lr, slowest, float(noise.sum())))
    dist.destroy_process_group()


def test_replicas_max_over_ranks_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    assert all(o[1] == world for o in out)
    assert all(o[3] == 11.0 for o in out)
    assert out[0][4] != out[1][4]


def test_reference_arm_nonzero_ranks_do_nothing(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setenv("RANK", "0")
    called = []
    monkeypatch.setattr(bench, "oracle_sample", lambda steps: (called.append(steps) or (1.0, 1.0, "x")))

    class A:
        steps, warmup, gpus = 2, 3, 1
    assert bench.run_reference(A()) == 0
    line = capsys.readouterr().out.strip()
    import json
    d = json.loads(line)
    assert d["impl"] == "reference" and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0
    assert called == [2]
