"""The N > 1 host logic of bench.py on CPU: two gloo ranks (world size 2)
check the max-over-ranks timing, the barrier, the whole-job value and that
only rank 0 prints the reference arm's line."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import argparse

    import torch.distributed as dist

    import bench

    w, r, _ = bench.dist_setup(False)
    assert (w, r) == (world, rank)
    bench.barrier(w)
    # each rank's own time; every rank must see the slowest one
    t = bench.max_over_ranks(10.0 + 5.0 * rank, w)
    value = bench.job_value(1000, 4, t, w)
    bench.barrier(w)
    dist.destroy_process_group()
    # the reference arm: rank 0 alone runs and prints
    os.environ["MASTER_PORT"] = str(port + 1)
    args = argparse.Namespace(workload="small_gf8", warmup=1, steps=1)
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
        json.dump({"t": t, "value": value, "ref_out": buf.getvalue()}, f)


def test_two_gloo_ranks(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    assert res[0]["t"] == res[1]["t"] == 15.0
    # 2 ranks x 4 steps x 1000 B over 15 ms
    assert res[0]["value"] == pytest.approx(2 * 4 * 1000 / 0.015 / 1e9)
    lines = [ln for ln in res[0]["ref_out"].splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
    assert res[1]["ref_out"] == ""
