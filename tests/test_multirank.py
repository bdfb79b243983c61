"""The N > 1 path of the benchmark on CPU: two gloo ranks launched by torchrun. Each rank
takes its own queries (disjoint seeds, weak scaling) and the only exchange is the job's
time (slowest rank) and work (sum over ranks)."""
import json
import os
import socket
import subprocess
import sys
import textwrap

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import json, sys
    sys.path.insert(0, {root!r})
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo")
    r = dist.get_rank()
    ms, units = bench.combine_ranks(10.0 * (r + 1), 100 * (r + 1), device="cpu")
    g, pats = bench.workload(r, 6, "c2")
    edges = [sorted(p.edges()) for p in pats]
    got = [None, None]
    dist.all_gather_object(got, edges)
    rank, world, local = bench.dist_env()
    with open(sys.argv[1] + "/rank%d.json" % r, "w") as f:  # one file per rank: no interleaved output
        json.dump({{"rank": r, "env": [rank, world, local], "ms": ms, "units": units, "n": len(pats),
                   "disjoint": all(e not in got[1 - r] for e in edges)}}, f)
    dist.destroy_process_group()
""")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_shard_queries_and_combine_time_and_work(tmp_path):
    script = tmp_path / "child.py"
    script.write_text(CHILD.format(root=ROOT))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), str(script), str(tmp_path)]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=300, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [json.loads((tmp_path / f"rank{r}.json").read_text()) for r in range(2)]
    assert sorted(x["rank"] for x in lines) == [0, 1]
    for x in lines:
        assert x["ms"] == 20.0 and x["units"] == 300.0  # max of 10, 20 and sum of 100, 200
        assert x["env"][:2] == [x["rank"], 2] and x["n"] == 6
        assert x["disjoint"]  # no query of one rank is a query of the other


def test_single_process_keeps_its_own_numbers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(12.5, 7, device="cpu") == (12.5, 7.0)


SHARD_CHILD = textwrap.dedent("""
    import json, sys
    sys.path.insert(0, {root!r})
    import numpy as np
    import torch.distributed as dist
    import bench
    import oracle
    from paper_2508_21287_gb300 import binding as B
    from paper_2508_21287_gb300 import inputs as I
    dist.init_process_group("gloo")
    r, n = dist.get_rank(), dist.get_world_size()
    out = []
    for g, p, motifs in ((I.heavy_hex(3, 4), I.path(9), [4]), (I.grid(5, 5), I.cycle(8), [104, 106]),
                         (I.heavy_hex(2, 3), I.sub_patch(I.heavy_hex(2, 3), 14, 3), [4])):
        # the shard vertex: the first slice's first pattern vertex of the paper-order plan
        # (the host planner; no GPU)
        v0 = B.dm_decompose(p.n, p.row_ptr, p.col_idx, motifs)[0]["slice"][0]
        rows = oracle.enumerate(g, p).rows
        mine = rows[rows[:, v0] % n == r]
        cnt, cs = bench.combine_counts(len(mine), oracle.checksum(mine), device="cpu")
        whole = oracle.enumerate(g, p, rows=False)
        out.append([cnt == whole.count, cs == whole.checksum, int(len(mine)), int(whole.count)])
    with open(sys.argv[1] + "/shard%d.json" % r, "w") as f:
        json.dump(out, f)
    dist.destroy_process_group()
""")


def test_two_gloo_ranks_shard_r0_and_sum_counts_and_checksums(tmp_path):
    # R_0 sharding: each rank takes the embeddings whose shard vertex maps to its residue
    # (the partition dm_match_shard applies to the first table), and the only exchange is one
    # exact 2 x u64 sum; it must give the whole count and checksum (here from the oracle)
    from paper_2508_21287_gb300 import build
    build.build()
    import oracle
    oracle.build()
    script = tmp_path / "shard.py"
    script.write_text(SHARD_CHILD.format(root=ROOT))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), str(script), str(tmp_path)]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=300, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    res = [json.loads((tmp_path / f"shard{r}.json").read_text()) for r in range(2)]
    for case in zip(*res):
        for eq_count, eq_sum, part, whole in case:
            assert eq_count and eq_sum
        assert sum(c[2] for c in case) == case[0][3]  # the shards partition the set
        assert all(0 < c[2] < c[3] for c in case)     # and both shards are non-empty


def test_combine_counts_wraps_mod_2_64_in_one_process():
    sys.path.insert(0, ROOT)
    import bench
    big = (1 << 64) - 5
    assert bench.combine_counts(7, big, device="cpu") == (7, big)
