"""The multi-GPU form of the bench (replicas only, no collective on the data path) on CPU with
two gloo ranks: the job's time is the slowest rank's, the whole-job rate counts every rank's
replica, each rank draws its own replica from its seed, and the reference arm runs on rank 0
only (the other ranks exit without work or output)."""
import contextlib
import io
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    from paper_2210_05547_gb300 import inputs as I
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, world)
    rate = bench.job_rate(world, 1000, 4, ms)
    cfg = I.sbli_case(64, 32, seed=rank)             # the replica a rank runs
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        rc = bench.reference_arm(_Args(), rank, world) if rank != 0 else 0
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as fh:
        json.dump({"ms": ms, "rate": rate, "mach": cfg["mach"], "ref_rc": rc,
                   "ref_out": buf.getvalue()}, fh)


class _Args:
    steps = 1
    warmup = 0
    gpus = 2


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    r = [json.load(open(tmp_path / f"rank{k}.json")) for k in range(2)]
    assert r[0]["ms"] == r[1]["ms"] == 15.0                    # the slower rank's time
    assert r[0]["rate"] == pytest.approx(2 * 1000 * 3 * 4 / 0.015 / 1e6)
    assert r[0]["mach"] != r[1]["mach"]                         # independent replicas
    assert r[1]["ref_rc"] == 0 and r[1]["ref_out"] == ""       # non-zero ranks: no work, no line


def test_oracle_baseline_on_every_host_core():
    """The CPU baseline's all-cores leg: one spawned single-threaded process per host core runs
    one warmed oracle RK3 step of a small sample; the host rate is the processes' work over the
    slowest step, so it exceeds the one-core rate and stays below cores x the one-core rate x 1.5.
    A leg that cannot finish says why instead of vanishing from the bench line."""
    sys.path.insert(0, ROOT)
    import bench
    one, _, _ = bench.oracle_step_rate(48, 24)
    every = bench.oracle_all_cores(48, 24, deadline_s=240.0)
    assert "unavailable" not in every, every
    nproc = every["cores"]
    assert nproc == max(1, min(64, len(os.sched_getaffinity(0))))
    assert every["slowest_s"] > 0.0
    assert every["value"] > 0.5 * one and every["value"] < 1.5 * nproc * one
    late = bench.oracle_all_cores(48, 24, deadline_s=0.0)
    assert "deadline" in late["unavailable"]
