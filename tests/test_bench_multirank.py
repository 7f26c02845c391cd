"""bench.py's multi-rank host logic with two gloo ranks on CPU: every rank solves its own
system (replicas); the job's throughput is the summed targets over the slowest rank."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    d = bench.Dist()
    try:
        assert d.pg is not None and d.pg.get_backend() == "gloo"
        d.barrier()
        # rank 1 is the slow one
        agg = bench.aggregate(10.0 + 30.0 * rank, 1000 + rank, d)
        q.put((rank, agg))
    finally:
        d.close()


def test_two_gloo_ranks_aggregate():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = dict(q.get(timeout=5) for _ in range(world))
    for r in range(world):
        assert res[r]["ms_per_step"] == pytest.approx(40.0)
        assert res[r]["total_targets"] == pytest.approx(2001)
        assert res[r]["targets_per_s"] == pytest.approx(2001 / 0.040)


def test_single_process_aggregate():
    import bench
    d = bench.Dist()
    assert d.world == 1 and d.pg is None
    agg = bench.aggregate(20.0, 500, d)
    assert agg["targets_per_s"] == pytest.approx(500 / 0.02)


def test_reference_arm_line(capsys):
    """`bench.py --impl reference` on CPU: one JSON line with the contract's keys, the oracle
    timed on a bounded sample (a small system here), no device traffic in its e2e."""
    import json

    import bench
    bench.main(["--impl", "reference", "--n", "20000", "--steps", "1", "--warmup", "3"])
    line = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")][-1]
    d = json.loads(line)
    assert d["impl"] == "reference" and d["unit"] == "targets/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 3
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert isinstance(cb["cpu_model"], str) and cb["sample"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
