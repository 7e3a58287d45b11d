"""Pins of the oracle's adaptive quadtree (uneven densities, the paper's closing section): the U, V, W, X lists
deliver every leaf pair exactly once; on inputs whose adaptive tree is uniform the adaptive FMM equals the
uniform oracle FMM; as p grows it converges geometrically to the exact split sum (K_sigma between adjacent
leaves, point vortex otherwise); a tree of one or four leaves is the direct sum of Eq. 7; P2L is the
expansion of 1/(z - z_j)."""
import math

import numpy as np
import pytest

import fmm_inputs
import oracle


def rel_l2(a, b):
    return float(np.sqrt(np.sum((a[0] - b[0]) ** 2 + (a[1] - b[1]) ** 2) / np.sum(b[0] ** 2 + b[1] ** 2)))


def two_scale(n, seed):
    return fmm_inputs.two_scale(n, seed)


def brute_near_pairs(x, y, L, B):
    """Ordered pairs (i, j != i) whose adaptive leaves touch, by brute force over particles in numpy: a particle's
    leaf is its box at the first level whose box holds at most B particles (or at level L); the leaves' closed
    squares are compared in depth-L cells. Unit square domain."""
    ix = np.minimum(np.floor(np.asarray(x) * 2**L), 2**L - 1).astype(np.int64)
    iy = np.minimum(np.floor(np.asarray(y) * 2**L), 2**L - 1).astype(np.int64)
    lev = np.full(ix.size, L)
    done = np.zeros(ix.size, bool)
    for l in range(L + 1):
        key = (ix >> (L - l)) * (1 << l) + (iy >> (L - l))
        _, inv, cnt = np.unique(key, return_inverse=True, return_counts=True)
        stop = (cnt[inv] <= B) & ~done
        lev[stop] = l
        done |= stop
    sh = L - lev
    x0, y0 = (ix >> sh) << sh, (iy >> sh) << sh
    x1, y1 = x0 + (1 << sh) - 1, y0 + (1 << sh) - 1
    adj = ((x0[:, None] <= x1[None, :] + 1) & (x0[None, :] <= x1[:, None] + 1) &
           (y0[:, None] <= y1[None, :] + 1) & (y0[None, :] <= y1[:, None] + 1))
    return int(adj.sum()) - ix.size


@pytest.mark.parametrize("case", ["two_scale", "patches", "one_blob_at_max_depth", "coincident", "default_domain"])
def test_lists_deliver_every_leaf_pair_once(case):
    dom = (0.0, 0.0, 1.0)
    if case == "two_scale":
        x, y, _ = two_scale(3000, 21)
        L, B = 8, 16
    elif case == "patches":
        w = fmm_inputs.patches(4096, seed_index=22, std=0.05)
        x, y = w.x, w.y
        L, B = 8, 24
    elif case == "one_blob_at_max_depth":  # leaves at the maximum depth hold more than B
        r = fmm_inputs.rng(23)
        x = np.concatenate([0.5 + 1e-3 * r.random(300), r.random(200)])
        y = np.concatenate([0.25 + 1e-3 * r.random(300), r.random(200)])
        L, B = 5, 8
    elif case == "coincident":
        r = fmm_inputs.rng(24)
        x = np.concatenate([np.full(50, 0.7), r.random(400)])
        y = np.concatenate([np.full(50, 0.2), r.random(400)])
        L, B = 7, 10
    else:
        x, y, _ = two_scale(2000, 25)
        x, y, dom = x * 3.0 - 1.0, y * 3.0 + 2.0, None
        L, B = 7, 12
    bad, s = oracle.adaptive_lists_check(x, y, L, B, domain=dom)
    assert bad == 0, s
    assert s["maxV"] <= 27
    assert s["U"] >= s["leaves"]
    if case in ("two_scale", "one_blob_at_max_depth", "coincident"):
        assert s["near_pairs"] == brute_near_pairs(x, y, L, B)
    if case in ("two_scale", "patches", "default_domain"):
        assert s["W"] > 0 and s["X"] > 0 and s["W"] == s["X"], s  # X is W transposed
        assert s["deepest"] >= 5


def test_uniform_tree_equals_uniform_oracle():
    """A 32 x 32 lattice with B = 16: every level-3 box holds 16 particles, so the adaptive tree is the uniform
    depth-3 tree and the adaptive lists reduce to the uniform ones (U = 3 x 3 neighbours, V = interaction list,
    W = X = empty)."""
    h = 1.0 / 32
    gx, gy = np.meshgrid((np.arange(32) + 0.5) * h, (np.arange(32) + 0.5) * h)
    x, y = gx.ravel(), gy.ravel()
    g = fmm_inputs.rng(26).standard_normal(x.size) / x.size
    sigma = 0.75 * h
    bad, s = oracle.adaptive_lists_check(x, y, 6, 16, domain=(0.0, 0.0, 1.0))
    assert bad == 0 and s["leaves"] == 64 and s["W"] == 0 and s["X"] == 0 and s["deepest"] == 3
    ua = oracle.adaptive_fmm(x, y, g, sigma, 6, 16, 12, domain=(0.0, 0.0, 1.0))
    uu, vu, _ = oracle.fmm(x, y, g, sigma, 3, 12, domain=(0.0, 0.0, 1.0))
    assert rel_l2(ua, (uu, vu)) < 1e-13


def test_converges_to_split_sum_geometrically():
    x, y, g = two_scale(2500, 27)
    sigma = 2e-3
    ref = oracle.adaptive_split_direct(x, y, g, sigma, 8, 16, domain=(0.0, 0.0, 1.0))
    errs = []
    for p in (4, 8, 12, 16, 20):
        errs.append(rel_l2(oracle.adaptive_fmm(x, y, g, sigma, 8, 16, p, domain=(0.0, 0.0, 1.0)), ref))
    # worst-case ratio per term of the W / X / V expansions is at most 0.55; require a clear geometric decay
    for a, b in zip(errs, errs[1:]):
        assert b < 0.25 * a, errs
    assert errs[-1] < 1e-7, errs


def test_near_and_far_parts_add_up():
    x, y, g = two_scale(1200, 28)
    both = oracle.adaptive_fmm(x, y, g, 3e-3, 7, 12, 10, domain=(0.0, 0.0, 1.0))
    near = oracle.adaptive_fmm(x, y, g, 3e-3, 7, 12, 10, domain=(0.0, 0.0, 1.0), parts="near")
    far = oracle.adaptive_fmm(x, y, g, 3e-3, 7, 12, 10, domain=(0.0, 0.0, 1.0), parts="far")
    assert rel_l2((near[0] + far[0], near[1] + far[1]), both) < 1e-15


@pytest.mark.parametrize("L,B", [(0, 4), (1, 4), (6, 10000)])
def test_shallow_tree_is_the_direct_sum(L, B):
    """One leaf (depth 0, or B >= n) or four mutually adjacent leaves (depth 1): every pair is near."""
    x, y, g = two_scale(600, 29)
    sigma = 0.05
    a = oracle.adaptive_fmm(x, y, g, sigma, L, B, 8, domain=(0.0, 0.0, 1.0))
    d = oracle.direct(x, y, g, sigma)
    assert rel_l2(a, d) < 1e-14


def test_p2l_is_the_expansion_of_a_point_charge():
    zj, c, z, q = 0.9 + 0.4j, 0.1 + 0.05j, 0.25 - 0.1j, 0.3 - 0.7j
    exact = q / (z - zj)
    ratio = abs(z - c) / abs(zj - c)
    for p in (5, 10, 20, 40):
        b = oracle.p2l([zj.real], [zj.imag], [q], c, p)
        w = sum(b[k] * (z - c) ** k for k in range(p))
        assert abs(w - exact) <= 1.01 * abs(q) * ratio ** p / (abs(zj - c) - abs(z - c)) + 1e-15
    b = oracle.p2l([zj.real], [zj.imag], [q], c, 40)
    assert abs(sum(b[k] * (z - c) ** k for k in range(40)) - exact) < 1e-14
