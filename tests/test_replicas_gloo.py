"""Multi-process replicas on CPU (gloo, world size 2): job sharding, the
slowest-rank timing and the gathering of per-job results, as bench.py and the
serving loop use them with one process per GPU."""
from __future__ import annotations

import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import json

    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle as O
        from paper_1804_07250_gb300 import replicas as R

        jobs = list(range(11))
        mine = R.shard(jobs, rank, world)
        # each job: a short oracle chain keyed by its own stream id
        results = {}
        for j in mine:
            st = O.aztec(4)
            O.sweeps(O.DOMINO, st, seed=3, stream=R.replica_stream_id(j, 0, 1), k=5, t_scalar=1 << 31)
            results[j] = O.state_hash(st)
        slowest = R.max_over_ranks(10.0 + rank, dist)
        gathered = R.gather_results(results, dist)
        with open(os.path.join(out_dir, "r%d.json" % rank), "w") as f:
            json.dump({"mine": mine, "slowest": slowest,
                       "gathered": [{str(k): int(v) for k, v in g.items()} for g in gathered],
                       "sid": [R.replica_stream_id(7, r, world) for r in range(world)]}, f)
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas(tmp_path):
    import json

    import torch.multiprocessing as mp

    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    out = [json.load(open(tmp_path / ("r%d.json" % r))) for r in range(world)]
    # every job on exactly one rank
    assert sorted(out[0]["mine"] + out[1]["mine"]) == list(range(11))
    assert not set(out[0]["mine"]) & set(out[1]["mine"])
    # the job time is the slowest rank's, seen by every rank
    assert out[0]["slowest"] == out[1]["slowest"] == 11.0
    # every rank sees all results; a job's result depends on the job only
    import oracle as O
    for o in out:
        merged = {}
        for g in o["gathered"]:
            merged.update(g)
        assert sorted(int(k) for k in merged) == list(range(11))
        st = O.aztec(4)
        O.sweeps(O.DOMINO, st, seed=3, stream=4, k=5, t_scalar=1 << 31)
        assert merged["4"] == O.state_hash(st)
    assert len(set(out[0]["sid"])) == world


def test_single_process_fallbacks():
    from paper_1804_07250_gb300 import replicas as R
    assert R.shard([1, 2, 3], 0, 1) == [1, 2, 3]
    assert R.max_over_ranks(2.5) == 2.5
    assert R.gather_results({"a": 1}) == [{"a": 1}]
    assert R.replica_stream_id(5, 0, 1) == 5
    with pytest.raises(ValueError):
        R.shard([1], 2, 2)


def test_bench_starts_its_own_ranks():
    # `bench.py --gpus 2` started as one process re-runs itself as two ranks
    # (torch.distributed.run on 127.0.0.1); the dry run needs no GPU: each
    # rank samples its own replica and rank 0 reports both
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    env["CUDA_VISIBLE_DEVICES"] = ""
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--gpus", "2", "--dry-run"],
                       capture_output=True, text=True, env=env, timeout=300, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    out = json.loads(lines[0])
    assert out["n_gpus"] == 2 and out["ranks_seen"] == 2 and out["distinct_streams"] == 2


def _liveness_worker(rank, world, port, out_dir, lost_rank):
    # three steps of a replica chain; after each, the rank records the step
    # and waits (3 s at most) for every other rank to record it before going on
    import datetime
    import json
    import time

    import torch.distributed as dist

    store = dist.TCPStore("127.0.0.1", port, world, rank == 0, timeout=datetime.timedelta(seconds=60))
    dist.init_process_group("gloo", store=store, rank=rank, world_size=world)
    import oracle as O
    from paper_1804_07250_gb300 import replicas as R

    st = O.aztec(6)
    done, lost, total, waited = 0, None, None, 0.0
    try:
        for step in range(3):
            if rank == lost_rank and step == 1:
                raise RuntimeError("injected failure before the end of step 1")
            O.sweeps(O.DOMINO, st, seed=9, stream=R.replica_stream_id(0, rank, world), sweep0=5 * step, k=5,
                     t_scalar=1 << 31)
            done = step + 1
            R.heartbeat(store, rank, step)
            t0 = time.monotonic()
            try:
                R.wait_peers(store, world, step, timeout_s=3.0)
            finally:
                waited = time.monotonic() - t0
        total = R.max_over_ranks(float(done), dist)   # the collective after the last step
    except R.PeerLost as e:
        lost = {"step": e.step, "ranks": e.ranks}
    except RuntimeError:
        if rank == lost_rank:
            os._exit(3)   # the failed rank leaves without touching the group again
        raise
    with open(os.path.join(out_dir, "live%d.json" % rank), "w") as f:
        json.dump({"done": done, "lost": lost, "total": total, "waited": waited, "hash": int(O.state_hash(st))}, f)
    if lost is None:
        dist.destroy_process_group()
    os._exit(0)


@pytest.mark.parametrize("lost_rank", [None, 1])
def test_lost_rank_is_found_between_steps(tmp_path, lost_rank):
    # a rank that fails between steps is found by the others on the host,
    # through the shared store, within the liveness limit: they stop before
    # the next collective (none waits for the lost rank) and keep their own
    # results; with no failure every step and the final collective complete
    import json
    import multiprocessing

    import oracle as O

    world, port = 2, _free_port()
    ctx = multiprocessing.get_context("spawn")
    procs = [ctx.Process(target=_liveness_worker, args=(r, world, port, str(tmp_path), lost_rank))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    codes = [p.exitcode for p in procs]
    for p in procs:
        if p.exitcode is None:
            p.kill()
    assert codes[0] == 0, codes
    out0 = json.load(open(tmp_path / "live0.json"))
    st = O.aztec(6)
    O.sweeps(O.DOMINO, st, seed=9, stream=0, k=5 * out0["done"], t_scalar=1 << 31)
    assert out0["hash"] == O.state_hash(st)       # the survivor's chain is exact
    if lost_rank is None:
        assert codes == [0, 0]
        assert out0["done"] == 3 and out0["lost"] is None and out0["total"] == 3.0
    else:
        assert codes[1] == 3
        assert out0["done"] == 2 and out0["total"] is None
        assert out0["lost"] == {"step": 1, "ranks": [1]}
        assert 2.5 < out0["waited"] < 30.0        # found at the limit, not by a hang
