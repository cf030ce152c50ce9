"""The multi-process path of bench.py on CPU: two gloo ranks on 127.0.0.1 run
the same helpers the GPU bench uses under torchrun (setup from the
environment, barrier, max over ranks, whole-job rate); the reference arm's
non-zero ranks return without work.  No GPU needed."""
from __future__ import annotations

import importlib.util
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    sys.path.insert(0, ROOT)
    spec.loader.exec_module(mod)
    return mod


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    os.environ["CUDA_VISIBLE_DEVICES"] = ""
    bench = load_bench()
    import torch.distributed as dist
    w, r, local = bench.dist_setup(None)
    assert (w, r, local) == (world, rank, rank) and dist.get_backend() == "gloo"
    bench.barrier(w)
    slowest = bench.max_over_ranks(10.0 + 5.0 * rank, w)  # per-rank step times in ms
    rate = bench.aggregate_rate(1_000_000, slowest, w)
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(f"{slowest} {rate}\n")
    bench.barrier(w)
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_rank(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, free_port(), str(tmp_path)), nprocs=world, join=True)
    got = [tuple(map(float, (tmp_path / f"rank{r}.txt").read_text().split())) for r in range(world)]
    assert got[0] == got[1]
    slowest, rate = got[0]
    assert slowest == 15.0
    assert rate == pytest.approx(world * 1_000_000 / 0.015 / 1e9)


def test_single_process_defaults():
    bench = load_bench()
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        os.environ.pop(k, None)
    assert bench.dist_setup(None) == (1, 0, 0)
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.aggregate_rate(2_000_000, 2.0, 1) == pytest.approx(1.0)


def test_reference_arm_other_ranks_do_no_work():
    bench = load_bench()
    assert bench.run_reference(None, 2, 1) is None  # rank 1 of 2 returns at once
