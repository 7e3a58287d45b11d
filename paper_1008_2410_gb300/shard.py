"""One FMM evaluation split over P parts by space (§3-§4 of the paper: each of P processes owns the subtrees below
a level k of the quadtree; the coarse levels above k, the "root tree", are formed from every process's level-k
multipoles, and each process's near field needs the particles of the leaves next to its own).

Host logic only: every step of the evaluation runs in the CUDA library (fmm_level_multipoles, fmm_velocity_level);
this module decides which part owns which level-k boxes, moves particles and the level-k arrays between parts,
and assembles the results. Parts talk through a small interface (``all_reduce_sum``, ``all_gather``, ``rank``,
``size``):

* ``DistComm``  -- torch.distributed, one process per part (gloo for CPU tensors, NCCL for CUDA tensors);
* ``ThreadComm`` -- P threads of one process (one FMM handle per thread), so the split can be run and checked on
  a single GPU: the threads only meet on the host, after synchronising their own work, never inside a kernel.

Per part, with its share of the input particles (any split; together the parts hold every particle once):

1. level-k box of each particle (the library's leaf rule at level k, explicit root square); the global box
   histogram (all-reduce); owners: contiguous runs of boxes in Morton order holding about N / P particles each;
2. particles move to the part that owns their box (an all-gather here: the simple exchange, not the cheapest);
   a part also keeps, as sources only, the particles of the level-k boxes adjacent to its own (the halo);
3. level-k multipoles and counts of its own particles (fmm_level_multipoles), summed over parts (all-reduce): the
   root tree's input;
4. fmm_velocity_level on own + halo particles with that sum in place of level k: exact at its own particles (the
   interaction lists below level k and the adjacent leaves lie inside own + halo boxes).
"""
from __future__ import annotations

import threading

import torch


def level_boxes(x: torch.Tensor, y: torch.Tensor, domain, level: int) -> tuple[torch.Tensor, torch.Tensor]:
    """(ix, iy) of each particle's box at `level`: floor((c - c0) * (2^level / S)) in IEEE double, clamped to
    [0, 2^level - 1], the library's leaf rule (the box at level k of the leaf at depth L is that leaf shifted by
    L - k, since 2^L / S and 2^k / S differ by a power of two)."""
    x0, y0, side = (float(v) for v in domain)
    ns = 1 << level
    scale = float(ns) / side
    ix = torch.floor((x - x0) * scale).clamp_(0, ns - 1).to(torch.int64)
    iy = torch.floor((y - y0) * scale).clamp_(0, ns - 1).to(torch.int64)
    return ix, iy


def morton(ix: torch.Tensor, iy: torch.Tensor) -> torch.Tensor:
    """Morton index (bits of ix on even positions, iy on odd ones) of box coordinates below 2^16."""
    def spread(v):
        v = v & 0xFFFF
        v = (v | (v << 8)) & 0x00FF00FF
        v = (v | (v << 4)) & 0x0F0F0F0F
        v = (v | (v << 2)) & 0x33333333
        v = (v | (v << 1)) & 0x55555555
        return v
    return spread(ix) | (spread(iy) << 1)


def owners(hist: torch.Tensor, level: int, parts: int) -> torch.Tensor:
    """Owner part of every level-`level` box (row-major grid, as `hist`): boxes taken in Morton order and cut into
    `parts` contiguous runs of about equal particle counts (part q takes the boxes whose Morton-order prefix count
    starts in [q N / P, (q + 1) N / P))."""
    ns = 1 << level
    iy, ix = torch.meshgrid(torch.arange(ns), torch.arange(ns), indexing="ij")
    order = torch.argsort(morton(ix.reshape(-1), iy.reshape(-1)))
    h = hist.to("cpu", torch.int64)[order]
    total = int(h.sum())
    before = torch.cumsum(h, 0) - h  # particles of the boxes before, in Morton order
    part = torch.clamp((before * parts) // max(total, 1), max=parts - 1)
    own = torch.empty(ns * ns, dtype=torch.int64)
    own[order] = part
    return own


def halo_mask(ix: torch.Tensor, iy: torch.Tensor, own_grid: torch.Tensor, rank: int, level: int) -> torch.Tensor:
    """True for particles whose level-k box is not owned by `rank` but touches (shares a side or a corner with) a
    box it owns."""
    ns = 1 << level
    g = own_grid.reshape(ns, ns).to(ix.device) == rank  # [iy][ix]
    near = torch.zeros_like(g)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            sh = torch.zeros_like(g)
            ys, yd = (slice(max(dy, 0), ns + min(dy, 0)), slice(max(-dy, 0), ns + min(-dy, 0)))
            xs, xd = (slice(max(dx, 0), ns + min(dx, 0)), slice(max(-dx, 0), ns + min(-dx, 0)))
            sh[yd, xd] = g[ys, xs]  # sh[b] = owned(b + (dx, dy))
            near |= sh
    return near[iy, ix] & ~g[iy, ix]


class DistComm:
    """torch.distributed collectives (the process group must be initialised)."""

    def __init__(self):
        import torch.distributed as dist

        self.dist = dist
        self.rank = dist.get_rank()
        self.size = dist.get_world_size()

    def all_reduce_sum(self, t: torch.Tensor) -> torch.Tensor:
        t = t.clone()
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM)
        return t

    def all_gather(self, t: torch.Tensor) -> torch.Tensor:
        """Concatenation over parts of 1-D tensors of any lengths (padded to the longest for the collective)."""
        n = torch.tensor([t.numel()], dtype=torch.int64, device=t.device)
        ns = [torch.zeros_like(n) for _ in range(self.size)]
        self.dist.all_gather(ns, n)
        m = max(int(v) for v in ns)
        pad = torch.zeros(m, dtype=t.dtype, device=t.device)
        pad[: t.numel()] = t
        outs = [torch.empty_like(pad) for _ in range(self.size)]
        self.dist.all_gather(outs, pad)
        return torch.cat([o[: int(k)] for o, k in zip(outs, ns)])


class ThreadComm:
    """Collectives among `size` threads of one process; ``for_rank(r)`` gives each thread its view."""

    def __init__(self, size: int, timeout: float = 120.0):
        self.size = size
        self._bar = threading.Barrier(size, timeout=timeout)  # a failed part breaks it instead of hanging the rest
        self._slots = [None] * size

    def for_rank(self, rank: int) -> "_ThreadRank":
        return _ThreadRank(self, rank)


class _ThreadRank:
    def __init__(self, hub: ThreadComm, rank: int):
        self.hub, self.rank, self.size = hub, rank, hub.size

    def _exchange(self, t: torch.Tensor) -> list:
        if t.is_cuda:
            torch.cuda.current_stream(t.device).synchronize()  # this part's work is done before others read it
        self.hub._slots[self.rank] = t
        self.hub._bar.wait()
        got = list(self.hub._slots)
        self.hub._bar.wait()  # every part has read the slots before they are reused
        return got

    def all_reduce_sum(self, t: torch.Tensor) -> torch.Tensor:
        got = self._exchange(t)
        out = torch.zeros_like(t)
        for g in got:  # the same order in every part
            out += g.to(t.device)
        return out

    def all_gather(self, t: torch.Tensor) -> torch.Tensor:
        return torch.cat([g.to(t.device) for g in self._exchange(t)])


def velocity_sharded(fmm, comm, x: torch.Tensor, y: torch.Tensor, gamma: torch.Tensor, index: torch.Tensor,
                     domain, level: int) -> dict:
    """This part's share of one sharded evaluation (module docstring, steps 1-4).

    fmm: this part's handle (``api.FMM``, uniform tree, explicit root square `domain`, depth >= level >= 2);
    x, y, gamma: this part's input particles (float64, on the handle's device); index: their global indices
    (int64). Returns {"index", "u", "v"} for the particles this part owns (the union over parts is every particle
    once), plus "own" and "halo" counts."""
    dev = x.device
    nb = 1 << (2 * level)
    ix, iy = level_boxes(x, y, domain, level)
    hist = torch.bincount(iy * (1 << level) + ix, minlength=nb).to(torch.int64)
    hist = comm.all_reduce_sum(hist)
    own_grid = owners(hist, level, comm.size)
    # redistribution: every particle to its box's owner; the halo as sources only
    ax, ay, ag, ai = (comm.all_gather(t) for t in (x, y, gamma, index))
    bx, by = level_boxes(ax, ay, domain, level)
    mine = own_grid.to(dev)[by * (1 << level) + bx] == comm.rank
    halo = halo_mask(bx, by, own_grid, comm.rank, level)
    ox, oy, og, oi = ax[mine], ay[mine], ag[mine], ai[mine]
    # root tree input: level-k multipoles and counts of every part's own particles
    M, cnt = fmm.level_multipoles(ox.contiguous(), oy.contiguous(), og.contiguous(), level)
    M = comm.all_reduce_sum(M)
    cnt = comm.all_reduce_sum(cnt)
    sx = torch.cat([ox, ax[halo]]).contiguous()
    sy = torch.cat([oy, ay[halo]]).contiguous()
    sg = torch.cat([og, ag[halo]]).contiguous()
    u, v = fmm.velocity_level(sx, sy, sg, level, M, cnt)
    n_own = ox.numel()
    return {"index": oi, "u": u[:n_own], "v": v[:n_own], "own": n_own, "halo": int(halo.sum())}
