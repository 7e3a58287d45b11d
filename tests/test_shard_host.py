"""Host logic of the sharded evaluation (paper §3-§4: parts own level-k subtrees, share the root tree through the
level-k multipoles, and exchange one layer of neighbouring boxes) on 2 and 4 gloo ranks, CPU only.

The CUDA library is replaced by a stand-in with the same two calls whose results are simple functions of what a
part is given, so every check is exact: its "multipoles" are the circulation sum of each level-k box and its
"velocity" at a particle is (the box's circulation from the arrays it was handed, the number of particles it was
handed in that box). A correct split gives every particle to exactly one part, hands each part every particle of
its own boxes and of the boxes touching them (nothing else), and makes the summed arrays the global ones."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")

from paper_1008_2410_gb300 import shard  # noqa: E402

DOMAIN = (0.0, 0.0, 1.0)
LEVEL = 3


class StandIn:
    """The library's two sharding calls, replaced by exactly checkable functions of their inputs."""

    def __init__(self, p: int = 4):
        self.p = p
        self.received = None

    def level_multipoles(self, x, y, g, level):
        ix, iy = shard.level_boxes(x, y, DOMAIN, level)
        b = iy * (1 << level) + ix
        nb = 1 << (2 * level)
        M = torch.zeros((nb, self.p, 2), dtype=torch.float64)
        M[:, 0, 0] = torch.zeros(nb, dtype=torch.float64).index_add_(0, b, g)
        return M, torch.bincount(b, minlength=nb).to(torch.int64)

    def velocity_level(self, x, y, g, level, M, cnt):
        self.received = (x.clone(), y.clone())
        ix, iy = shard.level_boxes(x, y, DOMAIN, level)
        b = iy * (1 << level) + ix
        local = torch.bincount(b, minlength=1 << (2 * level)).to(torch.float64)
        return M[b, 0, 0].clone(), local[b]


def _data(n=3000, seed=5):
    r = np.random.default_rng(seed)
    # uneven density: a dense blob and a uniform background
    m = n // 2
    x = np.concatenate([np.clip(0.3 + 0.05 * r.standard_normal(m), 0, 0.999), r.random(n - m)])
    y = np.concatenate([np.clip(0.7 + 0.05 * r.standard_normal(m), 0, 0.999), r.random(n - m)])
    g = r.standard_normal(n)
    return x, y, g


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        x, y, g = (torch.from_numpy(a) for a in _data())
        n = x.numel()
        idx = torch.arange(n, dtype=torch.int64)
        sl = slice(rank * n // world, (rank + 1) * n // world)  # each rank starts with an arbitrary share
        f = StandIn()
        res = shard.velocity_sharded(f, shard.DistComm(), x[sl], y[sl], g[sl], idx[sl], DOMAIN, LEVEL)
        rx, ry = f.received
        np.savez(os.path.join(out_dir, f"r{rank}.npz"), index=res["index"].numpy(), u=res["u"].numpy(),
                 v=res["v"].numpy(), rx=rx.numpy(), ry=ry.numpy(), own=res["own"], halo=res["halo"])
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_sharded_split_gloo(tmp_path, world):
    import torch.multiprocessing as mp

    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    x, y, g = _data()
    n = x.size
    xt, yt = torch.from_numpy(x), torch.from_numpy(y)
    ix, iy = shard.level_boxes(xt, yt, DOMAIN, LEVEL)
    ns = 1 << LEVEL
    box = (iy * ns + ix).numpy()
    hist = np.bincount(box, minlength=ns * ns)
    circ = np.zeros(ns * ns)
    np.add.at(circ, box, g)
    owner = shard.owners(torch.from_numpy(hist), LEVEL, world).numpy()
    seen = np.zeros(n, dtype=int)
    for r in range(world):
        d = np.load(tmp_path / f"r{r}.npz")
        idx = d["index"]
        seen[idx] += 1
        assert np.all(owner[box[idx]] == r)                     # a part gets exactly the particles it owns
        assert np.array_equal(d["u"], circ[box[idx]])           # the summed level-k arrays are the global ones
        assert np.array_equal(d["v"], hist[box[idx]])           # ... and its own boxes arrived whole
        # what it was handed: its own boxes and those touching them (corners included), nothing else
        want = np.zeros(ns * ns, dtype=bool)
        og = (owner == r).reshape(ns, ns)
        for by in range(ns):
            for bx in range(ns):
                if og[max(by - 1, 0):by + 2, max(bx - 1, 0):bx + 2].any():
                    want[by * ns + bx] = True
        rix, riy = shard.level_boxes(torch.from_numpy(d["rx"]), torch.from_numpy(d["ry"]), DOMAIN, LEVEL)
        got_boxes = (riy * ns + rix).numpy()
        assert np.all(want[got_boxes])
        assert len(got_boxes) == hist[want].sum()
        assert int(d["own"]) + int(d["halo"]) == len(got_boxes)
    assert np.all(seen == 1)
    # owners: contiguous in Morton order and balanced to within one box's particles
    loads = [hist[owner == r].sum() for r in range(world)]
    assert max(loads) - min(loads) <= 2 * hist.max()


def test_owner_rule_and_halo_on_a_small_grid():
    hist = torch.ones(16, dtype=torch.int64)  # level 2, 16 boxes of one particle each
    own = shard.owners(hist, 2, 4)
    # four parts over 16 equal boxes in Morton order: the four quadrants
    assert own.reshape(4, 4).tolist() == [[0, 0, 1, 1], [0, 0, 1, 1], [2, 2, 3, 3], [2, 2, 3, 3]]
    ix = torch.tensor([0, 1, 2, 3, 2, 3])
    iy = torch.tensor([0, 0, 0, 0, 2, 3])
    # part 0 owns the lower-left quadrant: boxes in column 2 or row 2 touch it; (3, 0) and (3, 3) do not
    assert shard.halo_mask(ix, iy, own, 0, 2).tolist() == [False, False, True, False, True, False]
