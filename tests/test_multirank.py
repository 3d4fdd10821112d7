"""Host logic of the multi-process benchmark path, on CPU with two gloo ranks.

Signals are independent (eq. 3 separates over the columns of B), so with N
processes each rank solves its own batch against the shared dictionary and the
only cross-rank steps are the barrier around the timed region and the max over
ranks of the elapsed time.  These tests run that logic as two processes on
127.0.0.1: the ranks agree on the dictionary, hold disjoint signals, reduce
their timings to the slowest rank, and only rank 0 runs the reference arm."""
import contextlib
import io
import os
import socket
import sys
import types

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    from paper_1302_5010_gb300 import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        P = bench.rank_problem(synth, "c1", rank, p=6)
        Pt = bench.rank_problem(synth, "c1", rank, p=6, seed_shift=9000)
        a_sum = torch.tensor([float(np.sum(P.At, dtype=np.float64))], dtype=torch.float64)
        sums = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(sums, a_sum)
        Bs = [torch.zeros(P.B.shape, dtype=torch.float32) for _ in range(world)]
        dist.all_gather(Bs, torch.from_numpy(P.B))
        # the slowest rank sets the time
        slow = bench.max_over_ranks(1.0 + 2.0 * rank, dist, torch.device("cpu"))
        rate = bench.aggregate_rate(world, P.p, 5, slow)
        # the reference arm prints on rank 0 only
        buf = io.StringIO()
        args = types.SimpleNamespace(config="c1", ref_signals=1, steps=1, warmup=0)
        with contextlib.redirect_stdout(buf):
            if rank != 0:
                bench.run_reference(args, rank, world)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"),
                 sums=np.array([float(t) for t in sums]), B=np.stack([b.numpy() for b in Bs]),
                 Btrain=Pt.B, slow=slow, rate=rate, printed=len(buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [np.load(tmp_path / f"rank{k}.npz") for k in range(world)]
    # one dictionary on every rank
    assert r[0]["sums"][0] == r[0]["sums"][1]
    # disjoint signals: rank batches differ, and differ from the training stream
    B = r[0]["B"]
    assert B[0].shape == (6, 256)
    assert not np.allclose(B[0], B[1])
    for k in range(world):
        assert not np.allclose(r[k]["Btrain"], B[k])
    # max over ranks seen identically by both ranks
    assert r[0]["slow"] == r[1]["slow"] == 3.0
    assert r[0]["rate"] == pytest.approx(2 * 6 * 5 / 3.0)
    assert int(r[1]["printed"]) == 0


def test_single_process_helpers():
    sys.path.insert(0, ROOT)
    import bench
    from paper_1302_5010_gb300 import synth
    assert bench.max_over_ranks(2.5, None, None) == 2.5
    assert bench.aggregate_rate(1, 256, 10, 2.0) == 1280.0
    P0 = bench.rank_problem(synth, "c1", 0, p=3)
    Pref = synth.make_config("c1", p=3)
    np.testing.assert_array_equal(P0.B, Pref.B)
    np.testing.assert_array_equal(P0.At, Pref.At)
