"""Seeded synthetic vortex-particle workloads.

The only module both the CUDA path's tests/bench and the CPU oracle's tests draw inputs from. It holds no
step of the FMM: it only draws positions and circulations (numpy PCG64, seed = 1008241 + workload index)
and states the tree parameters of each workload. The paper (M. G. Knepley, "Removing the Barrier to
Scalability in Parallel FMM", §2) uses no dataset; these stand-ins have the shapes of its vortex-method
setting: Gaussian blobs of core sigma on a quadtree with about 64 particles per leaf.

Workloads:
  lattice_lamb_oseen  N = 128^2 lattice in [-1, 1]^2, gamma_i = h^2 omega(x_i) of a Lamb-Oseen vortex
                      (Gamma = 1, core 0.2), sigma = 2h, depth 4, p = 12
  uniform_1m          N = 2^20 uniform in [0, 1)^2, gamma ~ N(0, 1)/N, sigma = 0.5/sqrt(N), depth 7, p = 17
  patches_16m         N = 2^24 from 8 Gaussian patches (std 0.05, centres U[0.2, 0.8]^2, circulations +-1),
                      depth 9, p = 20, sigma = 0.5/sqrt(N)
  batched_64          64 systems, N_k log-uniform in [4096, 262144], uniform, gamma ~ N(0, 1)/N_k,
                      sigma_k = 0.5/sqrt(N_k), depth_k = round(log4(N_k / 64)), p = 14
  adjoint_1m          uniform_1m positions; target velocities from gamma + 0.01 N(0, 1)/N
  two_scale           small adaptive-tree test field: a dense blob (std 0.02), a uniform background and three
                      isolated points, so that leaves sit on many levels
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 1008241


def rng(index: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + index))


@dataclass
class Workload:
    name: str
    x: np.ndarray
    y: np.ndarray
    gamma: np.ndarray
    sigma: float
    depth: int
    p: int
    domain: tuple[float, float, float]
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.x.size)


def lamb_oseen_vorticity(x, y, circulation: float = 1.0, core: float = 0.2):
    """omega(r) = Gamma / (pi r_c^2) exp(-r^2 / r_c^2) (Lamb-Oseen vortex at the origin)."""
    r2 = x * x + y * y
    return circulation / (math.pi * core * core) * np.exp(-r2 / (core * core))


def lattice_lamb_oseen(side: int = 128, depth: int = 4, p: int = 12) -> Workload:
    """Lattice x = -1 + (i + 1/2) h in [-1, 1]^2, h = 2/side, gamma = h^2 omega(x), sigma = 2h."""
    h = 2.0 / side
    c = -1.0 + (np.arange(side) + 0.5) * h
    X, Y = np.meshgrid(c, c, indexing="xy")
    x, y = X.ravel().copy(), Y.ravel().copy()
    g = h * h * lamb_oseen_vorticity(x, y)
    return Workload("lattice_lamb_oseen", x, y, g, 2.0 * h, depth, p, (-1.0, -1.0, 2.0),
                    {"h": h, "circulation": 1.0, "core": 0.2})


def uniform(n: int, seed_index: int = 1, depth: int | None = None, p: int = 17, sigma: float | None = None,
            name: str = "uniform") -> Workload:
    """n uniform points in [0, 1)^2, gamma ~ N(0, 1)/n, sigma = 0.5/sqrt(n), ~64 particles per leaf."""
    r = rng(seed_index)
    x = r.random(n)
    y = r.random(n)
    g = r.standard_normal(n) / max(n, 1)
    if depth is None:
        depth = max(0, int(round(math.log(max(n, 1) / 64.0, 4)))) if n > 64 else 0
    if sigma is None:
        sigma = 0.5 / math.sqrt(max(n, 1))
    return Workload(name, x, y, g, sigma, depth, p, (0.0, 0.0, 1.0))


def uniform_1m() -> Workload:
    return uniform(1 << 20, seed_index=1, depth=7, p=17, name="uniform_1m")


def patches(n: int, seed_index: int = 2, depth: int = 9, p: int = 20, npatch: int = 8, std: float = 0.05,
            name: str = "patches") -> Workload:
    """Mixture of npatch Gaussian patches; draws outside [0, 1)^2 are redrawn. Half the patches carry
    circulation +1 and half -1 (seeded order); every particle of a patch carries Gamma_patch / (n / npatch)."""
    r = rng(seed_index)
    centres = 0.2 + 0.6 * r.random((npatch, 2))
    signs = np.array([1.0] * (npatch // 2) + [-1.0] * (npatch - npatch // 2))
    r.shuffle(signs)
    per = n // npatch
    counts = np.full(npatch, per)
    counts[: n - per * npatch] += 1
    xs, ys, gs = [], [], []
    for k in range(npatch):
        m = int(counts[k])
        px = np.empty(m)
        py = np.empty(m)
        todo = np.arange(m)
        while todo.size:
            px[todo] = centres[k, 0] + std * r.standard_normal(todo.size)
            py[todo] = centres[k, 1] + std * r.standard_normal(todo.size)
            bad = (px[todo] < 0.0) | (px[todo] >= 1.0) | (py[todo] < 0.0) | (py[todo] >= 1.0)
            todo = todo[bad]
        xs.append(px)
        ys.append(py)
        gs.append(np.full(m, signs[k] / (n / npatch)))
    x = np.concatenate(xs)
    y = np.concatenate(ys)
    g = np.concatenate(gs)
    perm = r.permutation(n)
    return Workload(name, x[perm].copy(), y[perm].copy(), g[perm].copy(), 0.5 / math.sqrt(n), depth, p,
                    (0.0, 0.0, 1.0), {"centres": centres, "signs": signs})


def patches_16m() -> Workload:
    return patches(1 << 24, seed_index=2, depth=9, p=20, name="patches_16m")


@dataclass
class Batch:
    name: str
    systems: list[Workload]
    p: int

    @property
    def offsets(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum([s.n for s in self.systems])]).astype(np.int64)


def batched(nsys: int = 64, nmin: int = 4096, nmax: int = 262144, p: int = 14, seed_index: int = 3) -> Batch:
    """nsys independent uniform systems, N_k = round(exp(U[ln nmin, ln nmax])), depth_k = round(log4(N_k/64))."""
    r = rng(seed_index)
    systems = []
    for k in range(nsys):
        n = int(round(math.exp(r.uniform(math.log(nmin), math.log(nmax)))))
        x = r.random(n)
        y = r.random(n)
        g = r.standard_normal(n) / n
        depth = int(round(math.log(n / 64.0, 4)))
        systems.append(Workload(f"sys{k}", x, y, g, 0.5 / math.sqrt(n), depth, p, (0.0, 0.0, 1.0)))
    return Batch("batched_64", systems, p)


def adjoint_target_gamma(w: Workload, seed_index: int = 5, scale: float = 0.01) -> np.ndarray:
    """Perturbed circulations gamma + scale * N(0, 1)/N used to make the target velocities u*."""
    r = rng(seed_index)
    return w.gamma + scale * r.standard_normal(w.n) / w.n


def sample_targets(n: int, count: int, seed_index: int = 7) -> np.ndarray:
    """Seeded sorted subsample of target indices (without replacement)."""
    r = rng(seed_index)
    count = min(count, n)
    return np.sort(r.choice(n, size=count, replace=False)).astype(np.int64)


def clustered(n: int, seed_index: int = 11, sigma: float | None = None, depth: int = 4, p: int = 14) -> Workload:
    """Small clustered test field: 70% of points in one tight blob, the rest uniform."""
    r = rng(seed_index)
    m = int(0.7 * n)
    x = np.concatenate([np.clip(0.3 + 0.03 * r.standard_normal(m), 0.0, 0.999999), r.random(n - m)])
    y = np.concatenate([np.clip(0.6 + 0.03 * r.standard_normal(m), 0.0, 0.999999), r.random(n - m)])
    g = r.standard_normal(n) / n
    if sigma is None:
        sigma = 0.5 / math.sqrt(n)
    return Workload("clustered", x, y, g, sigma, depth, p, (0.0, 0.0, 1.0))


def two_scale(n: int, seed_index: int = 21) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Dense blob (60%, std 0.02 around (0.31, 0.62)), uniform background and three isolated points, clipped to
    [0, 0.999]: leaves of an adaptive tree on many levels, with non-empty W and X lists. Returns (x, y, gamma)."""
    r = rng(seed_index)
    m = int(0.6 * n)
    x = np.concatenate([0.31 + 0.02 * r.standard_normal(m), r.random(n - m - 3), [0.9, 0.91, 0.05]])
    y = np.concatenate([0.62 + 0.02 * r.standard_normal(m), r.random(n - m - 3), [0.1, 0.1, 0.95]])
    x, y = np.clip(x, 0.0, 0.999), np.clip(y, 0.0, 0.999)
    g = r.standard_normal(n) / n
    return x, y, g
