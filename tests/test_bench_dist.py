"""bench.py's multi-rank plumbing on CPU with the gloo backend (world size
2): the max-over-ranks timing and the reference arm under torchrun."""
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


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        v = bench.max_over_ranks(1.5 + rank, dist, world)
        out.put((rank, v))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=5) for _ in range(2))
    assert got == {0: 2.5, 1: 2.5}


def test_reference_arm_two_ranks():
    """torchrun with two CPU ranks: rank 0 times the oracle and prints the
    one JSON line; rank 1 exits 0 without output."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "2", "--warmup", "3"]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["steps"] == 2
    assert d["unit"] == "MLUPS" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_lpt_partition_balance():
    """bench.py's longest-processing-time bin packing of the batch's node
    counts: every lattice in exactly one bin, the largest load within 4/3 of
    the lower bound max(total / bins, largest item)."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_1202_0442_gb300 import synth
    sizes = [w.nodes for w in synth.batch()]
    for m in (1, 2, 3, 4, 8):
        bins = bench.lpt_partition(sizes, m)
        assert sorted(k for b in bins for k in b) == list(range(len(sizes)))
        loads = [sum(sizes[k] for k in b) for b in bins]
        lower = max(sum(sizes) / m, max(sizes))
        assert max(loads) <= 4 / 3 * lower
    # 5 -> bin 0, 4 -> bin 1, 3 -> bin 1 (load 4), 3 -> bin 0 (5), 3 -> bin 1 (7)
    assert bench.lpt_partition([5, 4, 3, 3, 3], 2) == [[0, 3], [1, 2, 4]]
