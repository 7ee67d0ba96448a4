"""The N > 1 path on the CPU with world_size 2 gloo ranks: a star join
sharded by node 0's cover rows and merged by one all-reduce equals the
unsharded oracle result, and bench.py under torchrun prints one JSON line
from rank 0 only (the reference arm, which runs on the host)."""

import json
import os
import socket
import subprocess
import sys


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import oracle
    from paper_2301_10841_gb300 import datagen as G
    from paper_2301_10841_gb300 import shard

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    fact, dims = G.star_schema(n_fact=30_000, dims=(500, 800, 1200, 2000), s=1.1, seed=9)
    lo, hi = shard.row_range(len(fact["cols"][0]), rank, world)
    part = {"name": "F", "cols": [c[lo:hi] for c in fact["cols"]]}
    q = G.star_query(part, dims, theta=400_000_000)
    c, m, _ = oracle.binary_join(q, min_vars=[4, 5, 6, 7])
    total, mins = shard.merge(c, m)
    if rank == 0:
        with open(out, "w") as f:
            json.dump({"count": total, "mins": mins}, f)
    dist.destroy_process_group()


def test_sharded_star_join_merges_to_the_whole(tmp_path):
    import multiprocessing as mp

    sys.path.insert(0, ROOT)
    import oracle
    from paper_2301_10841_gb300 import datagen as G

    oracle.build()
    out = str(tmp_path / "merged.json")
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    fact, dims = G.star_schema(n_fact=30_000, dims=(500, 800, 1200, 2000), s=1.1, seed=9)
    c, m, _ = oracle.binary_join(G.star_query(fact, dims, theta=400_000_000), min_vars=[4, 5, 6, 7])
    with open(out) as f:
        got = json.load(f)
    assert (got["count"], got["mins"]) == (c, m)


def _merge_edges_main(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    from paper_2301_10841_gb300 import shard

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    got = {}
    # A true MIN of 2^31 - 1 on one rank, no result row on the other.
    c, m = (5, [2**31 - 1, -3]) if rank == 0 else (0, [None, None])
    got["int32_max"] = shard.merge(c, m)
    # Counts above 2^63 (uint64): their sum still fits.
    got["big"] = shard.merge(2**63 - 1 + rank, [rank])
    # A sum of 2^64 does not fit.
    try:
        shard.merge(2**63, [0])
        got["overflow"] = False
    except OverflowError:
        got["overflow"] = True
    if rank == 0:
        with open(out, "w") as f:
            json.dump(got, f)
    dist.destroy_process_group()


def test_merge_keeps_int32_max_and_uint64_counts(tmp_path):
    """The merge's edge cases: a MIN equal to 2^31 - 1 is a value, not "no
    row"; counts above 2^63 merge exactly; a total of 2^64 is an overflow."""
    import multiprocessing as mp

    out = str(tmp_path / "edges.json")
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_merge_edges_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    with open(out) as f:
        got = json.load(f)
    assert got["int32_max"] == [5, [2**31 - 1, -3]]
    assert got["big"] == [2**64 - 1, [0]]
    assert got["overflow"] is True


def test_bench_reference_arm_two_ranks():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
