"""GPU parity of the adaptive quadtree (U, V, W, X lists) against the oracle's adaptive FMM on the same seeded
inputs: the FP64 form within 1e-12 relative L2 (same tree, same truncation, FP64 both sides), the precision form
(FP32 expansions and near field) within 1e-6. The full-size clustered workload (2^24 particles from 8 Gaussian
patches) is checked on sampled targets against the direct sum of Eq. 7, within the truncation and far-field-tail
bound the oracle's pins measure (1e-5)."""
import numpy as np
import pytest

import fmm_inputs as fi
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-6


def rel_l2(a, b):
    a = np.concatenate([np.ravel(t) for t in a])
    b = np.concatenate([np.ravel(t) for t in b])
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1008_2410_gb300 import api, build

    build.build()
    return api


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def gpu_adaptive(api, x, y, g, sigma, L, B, p, domain=(0.0, 0.0, 1.0), mode="full", graph=False,
                 precision="fp64"):
    f = api.FMM(L, p, sigma, precision=precision, domain=domain, graph=graph, leaf_capacity=B)
    fn = {"full": f.velocity, "near": f.velocity_near, "far": f.velocity_far}[mode]
    u, v = fn(dev(x), dev(y), dev(g))
    f.sync()
    return u.cpu().numpy(), v.cpu().numpy()


def blob_at_max_depth():
    r = fi.rng(23)
    x = np.concatenate([0.5 + 1e-3 * r.random(300), r.random(200)])
    y = np.concatenate([0.25 + 1e-3 * r.random(300), r.random(200)])
    return x, y, r.standard_normal(500) / 500


def tight_blob():
    """A cluster of 300 points in a 2e-4 square plus a sparse background: refinement down to the maximum depth 12."""
    r = fi.rng(38)
    x = np.concatenate([0.6 + 2e-4 * r.random(300), r.random(200)])
    y = np.concatenate([0.3 + 2e-4 * r.random(300), r.random(200)])
    return x, y, r.standard_normal(500) / 500


def coincident():
    r = fi.rng(24)
    x = np.concatenate([np.full(50, 0.7), r.random(400)])
    y = np.concatenate([np.full(50, 0.2), r.random(400)])
    return x, y, r.standard_normal(450) / 450


CASES = [
    ("two_scale3000_L8_B16_p14", lambda: fi.two_scale(3000, 21), 2e-3, 8, 16, 14, (0.0, 0.0, 1.0)),
    ("two_scale_bbox_L7_B12_p10", lambda: fi.two_scale(2000, 25), 3e-3, 7, 12, 10, None),
    ("patches8192_L9_B32_p20", lambda: (lambda w: (w.x, w.y, w.gamma))(fi.patches(8192, seed_index=22)), 5e-4, 9,
     32, 20, (0.0, 0.0, 1.0)),
    ("blob_at_max_depth_L5_B8_p12", blob_at_max_depth, 1e-3, 5, 8, 12, (0.0, 0.0, 1.0)),
    ("coincident_L7_B10_p12", coincident, 1e-3, 7, 10, 12, (0.0, 0.0, 1.0)),
    ("ragged_B1_L6_p8", lambda: fi.two_scale(777, 30), 2e-3, 6, 1, 8, (0.0, 0.0, 1.0)),
    ("p1_L7_B12", lambda: fi.two_scale(1500, 35), 2e-3, 7, 12, 1, (0.0, 0.0, 1.0)),
    ("p24_L8_B16", lambda: fi.two_scale(2000, 36), 2e-3, 8, 16, 24, (0.0, 0.0, 1.0)),
    ("p32_L8_B16", lambda: fi.two_scale(2000, 37), 2e-3, 8, 16, 32, (0.0, 0.0, 1.0)),
    ("depth12_tight_blob_B4_p12", lambda: tight_blob(), 2e-5, 12, 4, 12, (0.0, 0.0, 1.0)),
]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name,make,sigma,L,B,p,dom", CASES, ids=[c[0] for c in CASES])
def test_adaptive_matches_oracle(api, name, make, sigma, L, B, p, dom, precision):
    x, y, g = make()
    ref = oracle.adaptive_fmm(x, y, g, sigma, L, B, p, domain=dom)
    got = gpu_adaptive(api, x, y, g, sigma, L, B, p, domain=dom, precision=precision)
    assert rel_l2(got, ref) < (TOL64 if precision == "fp64" else TOL32)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("mode", ["near", "far"])
def test_adaptive_parts_match_oracle(api, mode, precision):
    x, y, g = fi.two_scale(2500, 27)
    ref = oracle.adaptive_fmm(x, y, g, 2e-3, 8, 16, 12, domain=(0.0, 0.0, 1.0), parts=mode)
    got = gpu_adaptive(api, x, y, g, 2e-3, 8, 16, 12, mode=mode, precision=precision)
    assert rel_l2(got, ref) < (TOL64 if precision == "fp64" else TOL32)


@pytest.mark.parametrize("L,B", [(0, 4), (1, 4), (6, 100000)])
def test_adaptive_shallow_tree_is_direct_sum(api, L, B):
    x, y, g = fi.two_scale(600, 29)
    got = gpu_adaptive(api, x, y, g, 0.05, L, B, 8)
    assert rel_l2(got, oracle.direct(x, y, g, 0.05)) < TOL64


def test_adaptive_uniform_tree_matches_uniform_path(api):
    """A 64 x 64 lattice with B = 16: the adaptive tree is the uniform depth-4 tree, so the adaptive path and the
    uniform FP64 path compute the same sum."""
    h = 1.0 / 64
    gx, gy = np.meshgrid((np.arange(64) + 0.5) * h, (np.arange(64) + 0.5) * h)
    x, y = gx.ravel(), gy.ravel()
    g = fi.rng(26).standard_normal(x.size) / x.size
    a = gpu_adaptive(api, x, y, g, 0.75 * h, 8, 16, 12)
    f = api.FMM(4, 12, 0.75 * h, precision="fp64", domain=(0.0, 0.0, 1.0))
    u, v = f.velocity(dev(x), dev(y), dev(g))
    f.sync()
    assert rel_l2(a, (u.cpu().numpy(), v.cpu().numpy())) < TOL64


def test_adaptive_graph_replay_is_deterministic(api):
    x, y, g = fi.two_scale(5000, 31)
    f = api.FMM(9, 16, 1e-3, precision="fp64", domain=(0.0, 0.0, 1.0), graph=True, leaf_capacity=24)
    xd, yd, gd = dev(x), dev(y), dev(g)
    outs = []
    for _ in range(3):
        u, v = f.velocity(xd, yd, gd)
        f.sync()
        outs.append((u.cpu().numpy().copy(), v.cpu().numpy().copy()))
    assert all(np.array_equal(outs[0][k], o[k]) for o in outs[1:] for k in range(2))
    ref = oracle.adaptive_fmm(x, y, g, 1e-3, 9, 24, 16, domain=(0.0, 0.0, 1.0))
    assert rel_l2(outs[0], ref) < TOL64
    assert f.params()["leaf_capacity"] == 24


def test_adaptive_rejects_batched_adjoint_and_outside_points(api):
    from paper_1008_2410_gb300 import _lib

    x, y, g = fi.two_scale(1000, 32)
    f = api.FMM(6, 10, 1e-3, domain=(0.0, 0.0, 1.0), leaf_capacity=16)
    with pytest.raises(_lib.FMMError):
        f.adjoint(dev(x), dev(y), dev(g), dev(g), dev(g))
    xo = x.copy()
    xo[5] = 1.5
    with pytest.raises(_lib.FMMError):
        f.velocity(dev(xo), dev(y), dev(g))
        f.sync()


def test_adaptive_advect_midpoint_step(api):
    """One Runge-Kutta 2 (midpoint) step of Eq. 3 on the adaptive tree, against the same step composed from the
    oracle's adaptive FMM (the tree is rebuilt from the bounding box at each stage on both sides)."""
    x, y, g = fi.two_scale(1500, 33)
    sigma, dt, L, B, p = 2e-3, 0.02, 7, 12, 12
    u1, v1 = oracle.adaptive_fmm(x, y, g, sigma, L, B, p)
    xm, ym = x + 0.5 * dt * u1, y + 0.5 * dt * v1
    u2, v2 = oracle.adaptive_fmm(xm, ym, g, sigma, L, B, p)
    f = api.FMM(L, p, sigma, precision="fp64", leaf_capacity=B)
    xd, yd = dev(x), dev(y)
    f.advect(xd, yd, dev(g), dt, 1, order=2)
    f.sync()
    assert rel_l2((xd.cpu().numpy() - x, yd.cpu().numpy() - y), (dt * u2, dt * v2)) < 1e-11


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_adaptive_pair_count_matches_oracle_lists(api, precision):
    """Ordered near pairs counted by the near-field kernel equal the oracle's count over its U lists."""
    x, y, g = fi.two_scale(3000, 21)
    _, sizes = oracle.adaptive_lists_check(x, y, 8, 16, domain=(0.0, 0.0, 1.0))
    f = api.FMM(8, 8, 2e-3, precision=precision, domain=(0.0, 0.0, 1.0), leaf_capacity=16)
    f.set_count_pairs(True)
    f.velocity(dev(x), dev(y), dev(g))
    assert f.pair_count() == sizes["near_pairs"] > 0


@pytest.mark.slow
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_adaptive_patches_16m_sampled_against_direct_sum(api, precision):
    """The clustered 2^24 workload at maximum depth 11, B = 48, p = 20, explicit unit square, as the bench runs it
    (graph replay): 256 sampled targets against Eq. 7 over all 2^24 sources."""
    w = fi.patches_16m()
    u, v = gpu_adaptive(api, w.x, w.y, w.gamma, w.sigma, 11, 48, w.p, domain=w.domain, precision=precision,
                        graph=True)
    t = fi.sample_targets(w.n, 256, seed_index=8)
    du, dv = oracle.direct(w.x, w.y, w.gamma, w.sigma, targets=t)
    assert rel_l2((u[t], v[t]), (du, dv)) < 1e-5


@pytest.mark.parametrize("pinned", [False, True])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_adaptive_host_entry_matches_device(api, pinned, precision):
    """fmm_velocity_host on the adaptive tree (inputs copied in, outputs copied out) gives the device path's
    result bit for bit."""
    x, y, g = fi.two_scale(4000, 34)
    dom = (0.0, 0.0, 1.0)
    f = api.FMM(9, 14, 1e-3, precision=precision, domain=dom, leaf_capacity=24)
    ud, vd = f.velocity(dev(x), dev(y), dev(g))
    f.sync()
    hx, hy, hg = (torch.from_numpy(np.ascontiguousarray(a)) for a in (x, y, g))
    if pinned:
        hx, hy, hg = hx.pin_memory(), hy.pin_memory(), hg.pin_memory()
    uh, vh = f.velocity_host(hx, hy, hg)
    assert np.array_equal(ud.cpu().numpy(), np.asarray(uh)) and np.array_equal(vd.cpu().numpy(), np.asarray(vh))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_adaptive_empty_and_single_particle(api, precision):
    """n = 0 is a no-op; one particle feels no velocity (K_sigma(0) = 0, nothing else to interact with)."""
    f = api.FMM(8, 12, 1e-3, precision=precision, domain=(0.0, 0.0, 1.0), leaf_capacity=16)
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    u0, v0 = f.velocity(e, e, e)
    f.sync()
    assert u0.numel() == 0 and v0.numel() == 0
    one = lambda a: dev(np.array([a]))
    u1, v1 = f.velocity(one(0.3), one(0.7), one(1.0))
    f.sync()
    assert float(u1.abs().max()) == 0.0 and float(v1.abs().max()) == 0.0


def test_adaptive_autotune_picks_a_capacity(api):
    """fmm_autotune on an adaptive handle keeps the fastest of the listed leaf capacities (and a maximum depth in
    range), and the tuned handle still matches the oracle at the chosen parameters."""
    x, y, g = fi.two_scale(20000, 39)
    f = api.FMM(9, 12, 1e-3, precision="mixed", domain=(0.0, 0.0, 1.0), leaf_capacity=64)
    tuned = f.autotune(dev(x), dev(y), dev(g), 8, 9)
    assert tuned["leaf_capacity"] in (16, 24, 32, 48, 64, 96, 128) and 8 <= tuned["depth"] <= 9
    u, v = f.velocity(dev(x), dev(y), dev(g))
    f.sync()
    ref = oracle.adaptive_fmm(x, y, g, 1e-3, tuned["depth"], tuned["leaf_capacity"], 12, domain=(0.0, 0.0, 1.0))
    assert rel_l2((u.cpu().numpy(), v.cpu().numpy()), ref) < TOL32
