"""Host-side logic of bench.py that needs no GPU: the whole-job aggregation over ranks (world size 2 on gloo,
one process per rank as under torchrun), the reference arm's rank rule, and the M2L translation count used for
the M2L roofline (pinned to the per-level interaction-list totals of a full tree)."""
import argparse
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

torch = pytest.importorskip("torch")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, totals, out_dir):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, value = bench.whole_job(totals[rank], 10, 1 << 20, world, dist)
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(f"{ms!r} {value!r}\n")
    finally:
        dist.destroy_process_group()


def test_whole_job_takes_the_slowest_rank_gloo_world2(tmp_path):
    import torch.multiprocessing as mp

    totals = [10.0, 12.5]  # ms over 10 steps on each rank
    mp.spawn(_rank_main, args=(2, _free_port(), totals, str(tmp_path)), nprocs=2, join=True)
    got = [tuple(float(t) for t in open(tmp_path / f"r{r}.txt").read().split()) for r in range(2)]
    for ms, value in got:  # every rank sees the same maximum
        assert ms == pytest.approx(1.25)
        assert value == pytest.approx(2 * (1 << 20) / 1.25e-3 / 1e6)


def test_whole_job_single_rank():
    ms, value = bench.whole_job(7.0, 7, 1000, 1)
    assert ms == 1.0 and value == pytest.approx(1.0)


def test_reference_arm_runs_on_rank0_only():
    args = argparse.Namespace(workload="uniform_1m", steps=1, warmup=0)
    assert bench.run_reference(args, rank=1, world=2) is None


class _W:
    pass


@pytest.mark.parametrize("depth,total", [(2, 156), (3, 156 + 1116), (4, 156 + 1116 + 5628),
                                         (5, 156 + 1116 + 5628 + 25020),
                                         (6, 156 + 1116 + 5628 + 25020 + 105276)])
def test_m2l_translations_full_tree(depth, total):
    """One particle per leaf: every box non-empty, so the count is the full tree's interaction-list total."""
    w = _W()
    w.depth, w.domain = depth, (0.0, 0.0, 1.0)
    n = 1 << depth
    g = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(g, g)
    w.x, w.y = X.ravel(), Y.ravel()
    assert bench.m2l_translations(w) == total


def test_m2l_translations_skip_empty_boxes():
    """Particles in the left half only: level-2 boxes in columns 2, 3 are empty; brute force over box pairs."""
    w = _W()
    w.depth, w.domain = 3, (0.0, 0.0, 1.0)
    n = 8
    g = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(g[: n // 2], g)
    w.x, w.y = X.ravel(), Y.ravel()
    want = 0
    for l in (2, 3):
        m = 1 << l
        occ = lambda bx, by: 0 <= bx < m and 0 <= by < m and bx < m // 2  # noqa: E731
        for by in range(m):
            for bx in range(m):
                if not occ(bx, by):
                    continue
                for sy in range(m):
                    for sx in range(m):
                        near = abs(sx - bx) <= 1 and abs(sy - by) <= 1
                        parents_adjacent = abs(sx // 2 - bx // 2) <= 1 and abs(sy // 2 - by // 2) <= 1
                        if occ(sx, sy) and not near and parents_adjacent:
                            want += 1
    assert bench.m2l_translations(w) == want
