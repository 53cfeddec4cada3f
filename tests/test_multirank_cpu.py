"""World-size-2 tests of the multi-rank path on CPU (gloo), no GPU.

Frames are independent of one another (Sec. "Parallelization": every farm node
selects its own frames), so N ranks each select a disjoint batch and nothing is
exchanged on the data path.  The only collectives are the timing barrier and the
max-over-ranks reduction of the timed duration.  These tests check, with the
oracle standing in for each rank's selection:
  * each rank draws its own batch (disjoint seeds) deterministically;
  * sharding changes no decision: the ranks' decisions are those of one process
    selecting all shards as one batch;
  * the timing reduction gives every rank the slowest rank's time;
  * the reference arm under torchrun prints one line, from rank 0 only.
"""
from __future__ import annotations

import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N_FRAMES = 300


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from oracle import oracle as O
    from paper_2206_11535_gb300 import gen
    d = bench.make_batch(N_FRAMES, rank)
    c = O.make_config(gen.load_config())
    keep, reason = O.select_frames(c, d["hits"], d["off"], 1)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, torch.device("cpu"), world)
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), hits=d["hits"], off=d["off"], keep=keep, reason=reason,
             ms=np.float64(ms))
    dist.barrier()
    dist.destroy_process_group()


def test_shards_are_independent_and_exact(tmp_path):
    import torch.multiprocessing as mp
    from oracle import oracle as O
    from paper_2206_11535_gb300 import gen
    O.build()
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    r = [np.load(tmp_path / f"rank{k}.npz") for k in range(world)]
    # the slowest rank's time on every rank
    assert [float(x["ms"]) for x in r] == [15.0, 15.0]
    # disjoint draws: the two shards differ, and rank 0's is the single-GPU batch
    assert r[0]["hits"].size != r[1]["hits"].size or not np.array_equal(r[0]["hits"], r[1]["hits"])
    import bench
    d0 = bench.make_batch(N_FRAMES, 0)
    assert np.array_equal(d0["hits"], r[0]["hits"]) and np.array_equal(d0["off"], r[0]["off"])
    # one process selecting the concatenated shards gives the ranks' decisions
    hits = np.concatenate([x["hits"] for x in r])
    off = np.concatenate([r[0]["off"], r[1]["off"][1:] + r[0]["off"][-1]])
    c = O.make_config(gen.load_config())
    keep, reason = O.select_frames(c, hits, off, 2)
    assert np.array_equal(reason, np.concatenate([x["reason"] for x in r]))
    assert np.array_equal(keep, np.concatenate([x["keep"] for x in r]))


def test_reference_arm_under_torchrun_prints_once():
    env = dict(os.environ, PYTHONPATH=ROOT)
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--frames", str(N_FRAMES)]
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [x for x in p.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["n_gpus"] == 2 and out["value"] > 0
    assert out["cpu_baseline"]["kind"] == "oracle" and out["e2e"]["h2d_bytes_per_step"] == 0


if __name__ == "__main__":
    sys.exit(pytest.main([__file__, "-q"]))
