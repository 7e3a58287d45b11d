"""The paper's complexity model (§3, Table 1, §4) for the 2D vortex-blob FMM, in flop units (rate r = 1).

T = a N/P + b log_4 P + c N/(B P) + d N B/P (the Greengard-Gropp form used in §3), with t expansion terms:
  a = 16t - 15,  b = (84 - 48t + 571t^2)/3,  c = (128 - 48t + 844t^2)/3,  d = 198      (Table 1)
  B_opt = sqrt(c/d)                                                                    (§4)
  full overlap of the root-tree bottleneck by near-field work:  B >= (b/d) P L_root / N (§4)
Used to report algorithmic work and the overlap bound next to measured times (the bench reports B_opt and the
minimum leaf occupancy for overlap beside the occupancy it runs).
"""
from __future__ import annotations

import math

P2P_FLOPS_PER_PAIR = 22  # §3: 9 flops per complex division, 1 per exponential, per ordered pair


def coefficients(t: int) -> dict:
    """Table 1 coefficients times the flop rate r."""
    return {
        "a": 16 * t - 15,
        "b": (84 - 48 * t + 571 * t * t) / 3.0,
        "c": (128 - 48 * t + 844 * t * t) / 3.0,
        "d": 198.0,
    }


def b_opt(t: int) -> float:
    """Optimal particles per leaf, sqrt(c/d) (§4)."""
    k = coefficients(t)
    return math.sqrt(k["c"] / k["d"])


def overlap_ratio(t: int) -> float:
    """b/d: the near-field work that covers one level of the root tree, per particle-per-leaf (§4)."""
    k = coefficients(t)
    return k["b"] / k["d"]


def min_leaf_occupancy_for_overlap(t: int, N: float, P: float, L_root: float | None = None) -> float:
    """Smallest B for which near-field work hides the root-tree bottleneck: (b/d) P L_root / N, with
    L_root = log_4 P by default (§4)."""
    if L_root is None:
        L_root = math.log(P, 4)
    return overlap_ratio(t) * P * L_root / N


def min_particles_per_process(t: int, P: float, B: float) -> float:
    """Memory-scalable regime: N/P >= (b/d) log_4 P / B (§4)."""
    return overlap_ratio(t) * math.log(P, 4) / B


def near_pairs_uniform(B: int, L: int) -> int:
    """Ordered near-field pairs of a full uniform tree with B particles per leaf at depth L (§3, W_direct/22)."""
    return (4 * (4 * B * B - B) + (2 ** (L + 2) - 8) * (6 * B * B - B)
            + (4 ** L - 2 ** (L + 2) + 4) * (9 * B * B - B))


def flops(N: int, B: float, L: int, t: int, near_pairs: int | None = None) -> dict:
    """Algorithmic flops of one evaluation by the paper's per-stage counts (§3): P2M (8t+3)/particle,
    L2P (8t+2)/particle, sum 2/particle, M2M 4(2+2t^2+4t(t-1)) per parent, M2L 27(2+17t^2) per cell,
    L2L 4(2+10t^2) per cell, and 22 per near-field pair."""
    if near_pairs is None:
        near_pairs = near_pairs_uniform(int(round(B)), L)
    up = sum(4 ** l for l in range(2, L)) * 4 * (2 + 2 * t * t + 4 * t * (t - 1))
    m2l = sum(4 ** l for l in range(2, L + 1)) * 27 * (2 + 17 * t * t)
    l2l = sum(4 ** l for l in range(3, L + 1)) * 4 * (2 + 10 * t * t)
    return {
        "p2m": (8 * t + 3) * N,
        "l2p": (8 * t + 2) * N,
        "sum": 2 * N,
        "m2m": up,
        "m2l": m2l,
        "l2l": l2l,
        "p2p": P2P_FLOPS_PER_PAIR * near_pairs,
    }
