"""The multi-process (replica) path of bench.py on the host: two gloo ranks
on CPU.  One process per GPU runs an independent replica (the path does not
shard), so the only cross-rank steps are the barrier around the timed region
and the maximum of the ranks' times; the whole-job value counts every rank's
units over the slowest rank's time.  The reference arm runs on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        bench._barrier(ws)
        local_s = [0.25, 0.75][rank]  # the ranks' own timed seconds
        slowest = bench._reduce_max(local_s, ws)
        value = bench._whole_job(1000.0, ws, slowest)
        bench._barrier(ws)
        q.put((rank, slowest, value))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_count_every_rank():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, value in out:
        assert slowest == 0.75  # every rank sees the slowest rank's time
        assert value == pytest.approx(2 * 1000.0 / 0.75)  # both ranks' units


def _reference_arm(rank, ws):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank),
               MASTER_ADDR="127.0.0.1")
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--gpus", str(ws), "--steps", "1", "--warmup", "3"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_on_rank_0_only():
    r1 = _reference_arm(1, 2)
    assert r1.returncode == 0, r1.stderr
    assert r1.stdout.strip() == ""
    r0 = _reference_arm(0, 2)
    assert r0.returncode == 0, r0.stderr
    lines = [x for x in r0.stdout.splitlines() if x.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["value"] > 0
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_ensemble_members_are_sharded_by_cell_count():
    """The ensemble leg under several ranks: every member on exactly one rank,
    the ranks' cell counts within one largest member of each other, the
    same partition on every call."""
    sys.path.insert(0, ROOT)
    import bench
    from workloads import heat as H
    probs = H.config3_members(512)
    cells = [p.Nr * p.Nz for p in probs]
    for ws in (1, 2, 3, 8):
        parts = bench.shard_members(cells, ws)
        assert parts == bench.shard_members(cells, ws)
        flat = sorted(i for part in parts for i in part)
        assert flat == list(range(len(cells)))
        loads = [sum(cells[i] for i in part) for part in parts]
        assert max(loads) - min(loads) <= max(cells)
        assert all(part == sorted(part) for part in parts)


def _ens_rank(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        act, ms = [(1000, 2.0), (3000, 5.0)][rank]  # the ranks' own active cells and step time
        q.put((rank, bench._reduce_sum(act, ws), bench._reduce_max(ms, ws)))
    finally:
        dist.destroy_process_group()


def test_sharded_ensemble_counts_every_rank_over_the_slowest_time():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_ens_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, act, ms in out:
        assert act == 4000 and ms == 5.0
