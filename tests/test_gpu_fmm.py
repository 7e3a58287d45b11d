"""GPU parity tests: the CUDA path (through the C ABI) against the FP64 CPU oracle on the same seeded inputs.

Tolerances: plain FP64 form within 1e-12 relative L2 of the oracle FMM at the same depth and p; precision
form within 1e-6 relative L2 of the oracle FMM (FP32 arithmetic against FP64, same truncation); integer
results (pair counts) exact.
"""
import math

import numpy as np
import pytest

import fmm_inputs as fi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-6


def rel_l2(a, b):
    a = np.concatenate([np.ravel(t) for t in a])
    b = np.concatenate([np.ravel(t) for t in b])
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1008_2410_gb300 import api, build

    build.build()
    return api


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def run(lib, w, precision="fp64", domain="explicit", graph=False, mode="full", tile=None, m2l_engine=None):
    f = lib.FMM(w.depth, w.p, w.sigma, precision=precision, domain=w.domain if domain == "explicit" else None,
                graph=graph, m2l_engine=m2l_engine)
    if tile:
        f.set_p2p_tile(*tile)
    x, y, g = dev(w.x), dev(w.y), dev(w.gamma)
    fn = {"full": f.velocity, "near": f.velocity_near, "far": f.velocity_far}[mode]
    u, v = fn(x, y, g)
    f.sync()
    return u.cpu().numpy(), v.cpu().numpy(), f


CASES = [
    ("uniform5k_d3_p10", lambda: fi.uniform(5000, seed_index=31, depth=3, p=10)),
    ("uniform40k_d5_p17", lambda: fi.uniform(40000, seed_index=32, depth=5, p=17)),
    ("ragged12345_d4_p20", lambda: fi.uniform(12345, seed_index=33, depth=4, p=20)),
    ("clustered20k_d5_p14", lambda: fi.clustered(20000, depth=5, p=14)),
    ("lattice_lamb_oseen_d4_p12", lambda: fi.lattice_lamb_oseen()),
    ("depth2_p8", lambda: fi.uniform(3000, seed_index=34, depth=2, p=8)),
    ("depth1", lambda: fi.uniform(1500, seed_index=35, depth=1, p=8)),
    ("depth0", lambda: fi.uniform(700, seed_index=36, depth=0, p=8)),
    ("p1_d3", lambda: fi.uniform(2000, seed_index=37, depth=3, p=1)),
    ("p32_d3", lambda: fi.uniform(2000, seed_index=38, depth=3, p=32)),
    ("patches64k_d6_p20", lambda: fi.patches(1 << 16, seed_index=39, depth=6, p=20)),
    # leaves 3 sigma wide: most particles sit in a boundary band, so the near field tests most neighbour sources
    ("wide_bands_d5", lambda: fi.uniform(20000, seed_index=41, depth=5, p=14, sigma=0.0105)),
    # leaves narrower than two band widths: no band order, every source tested
    ("no_bands_d6", lambda: fi.uniform(20000, seed_index=42, depth=6, p=14, sigma=0.01)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_fp64_matches_oracle_fmm(lib, oracle, name, make):
    w = make()
    u, v, _ = run(lib, w)
    uo, vo, _ = oracle.fmm(w.x, w.y, w.gamma, w.sigma, w.depth, w.p, domain=w.domain)
    assert rel_l2((u, v), (uo, vo)) < TOL64
    scale = max(np.abs(uo).max(), np.abs(vo).max())
    assert max(np.abs(u - uo).max(), np.abs(v - vo).max()) < 1e-11 * scale


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_mixed_matches_oracle_fmm(lib, oracle, name, make):
    w = make()
    uo, vo, _ = oracle.fmm(w.x, w.y, w.gamma, w.sigma, w.depth, w.p, domain=w.domain)
    for coarse in (4, -1):
        f = lib.FMM(w.depth, w.p, w.sigma, precision="mixed", domain=w.domain, coarse_level=coarse)
        u, v = f.velocity(dev(w.x), dev(w.y), dev(w.gamma))
        f.sync()
        assert rel_l2((u.cpu().numpy(), v.cpu().numpy()), (uo, vo)) < TOL32, coarse


@pytest.mark.parametrize("domain", ["explicit", "bbox"])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_mixed_symmetric_near_field_matches_oracle(lib, oracle, name, make, domain):
    """Tile 128: each adjacent pair evaluated once and applied to both particles (depth 0 and 1 have leaves wider
    than the one-float bound and go through the target-side kernel; with the bounding-box rule both kernels
    are launched)."""
    w = make()
    dom = w.domain if domain == "explicit" else None
    uo, vo, _ = oracle.fmm(w.x, w.y, w.gamma, w.sigma, w.depth, w.p, domain=dom)
    f = lib.FMM(w.depth, w.p, w.sigma, precision="mixed", domain=dom)
    f.set_p2p_tile(128, 4)
    u, v = f.velocity(dev(w.x), dev(w.y), dev(w.gamma))
    f.sync()
    assert rel_l2((u.cpu().numpy(), v.cpu().numpy()), (uo, vo)) < TOL32


@pytest.mark.parametrize("tile", [(64, 4), (64, 2), (256, 4), (256, 2), (32, 4), (32, 2), (128, 4), (128, 2), (192, 4),
                                  (192, 2)])
def test_mixed_tile_shapes(lib, oracle, tile):
    w = fi.clustered(30000, depth=4, p=12)  # dense leaves: several target chunks and source tiles per leaf
    uo, vo, _ = oracle.fmm(w.x, w.y, w.gamma, w.sigma, w.depth, w.p, domain=w.domain)
    u, v, _ = run(lib, w, precision="mixed", tile=tile)
    assert rel_l2((u, v), (uo, vo)) < TOL32


def test_default_domain_bbox_rule(lib, oracle):
    w = fi.clustered(9000, depth=4, p=12)
    u, v, _ = run(lib, w, domain=None)
    uo, vo, _ = oracle.fmm(w.x, w.y, w.gamma, w.sigma, w.depth, w.p, domain=None)
    assert rel_l2((u, v), (uo, vo)) < TOL64


@pytest.mark.parametrize("precision,tol", [("fp64", TOL64), ("mixed", TOL32)])
def test_near_and_far_halves(lib, oracle, precision, tol):
    w = fi.uniform(20000, seed_index=40, depth=4, p=14)
    un, vn, _ = run(lib, w, precision=precision, mode="near")
    uf, vf, _ = run(lib, w, precision=precision, mode="far")
    uon, von, _ = oracle.fmm(w.x, w.y, w.gamma, w.sigma, w.depth, w.p, domain=w.domain, parts="near")
    uof, vof, _ = oracle.fmm(w.x, w.y, w.gamma, w.sigma, w.depth, w.p, domain=w.domain, parts="far")
    assert rel_l2((un, vn), (uon, von)) < tol
    assert rel_l2((uf, vf), (uof, vof)) < tol


M2L_CASES = [
    ("p1_d3", lambda: fi.uniform(2000, seed_index=37, depth=3, p=1)),
    ("p8_d2", lambda: fi.uniform(3000, seed_index=34, depth=2, p=8)),
    ("p10_d3", lambda: fi.uniform(5000, seed_index=31, depth=3, p=10)),
    ("p14_d4", lambda: fi.uniform(20000, seed_index=40, depth=4, p=14)),
    ("p17_d5", lambda: fi.uniform(40000, seed_index=32, depth=5, p=17)),
    ("ragged12345_d4_p20", lambda: fi.uniform(12345, seed_index=33, depth=4, p=20)),
    ("p24_d3", lambda: fi.uniform(4000, seed_index=41, depth=3, p=24)),
    ("p32_d3", lambda: fi.uniform(2000, seed_index=38, depth=3, p=32)),
    ("clustered20k_d5_p14", lambda: fi.clustered(20000, depth=5, p=14)),  # empty boxes: zero source rows
    ("patches64k_d6_p20", lambda: fi.patches(1 << 16, seed_index=39, depth=6, p=20)),  # several tiles a level
    ("d8_p6", lambda: fi.uniform(200000, seed_index=42, depth=8, p=6)),  # levels <= 7 and level 8 split by engine
]


@pytest.mark.parametrize("engine", ["tensor", "cuda_cores"])
@pytest.mark.parametrize("name,make", M2L_CASES, ids=[c[0] for c in M2L_CASES])
def test_far_field_by_m2l_engine(lib, oracle, engine, name, make):
    """The far field alone (P2M, M2M, M2L, L2L, L2P) of the precision form against the oracle's far part, with
    the FP32 M2L levels on the tensor cores (3xTF32) and on the CUDA cores."""
    w = make()
    f = lib.FMM(w.depth, w.p, w.sigma, precision="mixed", domain=w.domain, m2l_engine=engine)
    u, v = f.velocity_far(dev(w.x), dev(w.y), dev(w.gamma))
    f.sync()
    uo, vo, _ = oracle.fmm(w.x, w.y, w.gamma, w.sigma, w.depth, w.p, domain=w.domain, parts="far")
    assert rel_l2((u.cpu().numpy(), v.cpu().numpy()), (uo, vo)) < TOL32


def test_pair_count_exact(lib, oracle):
    w = fi.lattice_lamb_oseen()
    f = lib.FMM(w.depth, w.p, w.sigma, domain=w.domain)
    f.set_count_pairs(True)
    f.velocity(dev(w.x), dev(w.y), dev(w.gamma))
    assert f.pair_count() == 8650752
    w = fi.clustered(15000, depth=5, p=8)
    f = lib.FMM(w.depth, w.p, w.sigma, domain=w.domain)
    f.set_count_pairs(True)
    f.velocity(dev(w.x), dev(w.y), dev(w.gamma))
    _, _, npairs = oracle.fmm(w.x, w.y, w.gamma, w.sigma, w.depth, 2, domain=w.domain, parts="near")
    assert f.pair_count() == npairs


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_deterministic_and_graph_replay_identical(lib, precision):
    w = fi.clustered(25000, depth=5, p=12)
    x, y, g = dev(w.x), dev(w.y), dev(w.gamma)
    f = lib.FMM(w.depth, w.p, w.sigma, precision=precision, domain=w.domain)
    u1, v1 = f.velocity(x, y, g)
    u2, v2 = f.velocity(x, y, g)
    fg = lib.FMM(w.depth, w.p, w.sigma, precision=precision, domain=w.domain, graph=True)
    if precision == "mixed":  # also the symmetric near field (reactions summed in a fixed order)
        fs = lib.FMM(w.depth, w.p, w.sigma, precision=precision, domain=w.domain)
        fs.set_p2p_tile(128, 4)
        us1, vs1 = fs.velocity(x, y, g)
        us2, vs2 = fs.velocity(x, y, g)
        torch.cuda.synchronize()
        assert torch.equal(us1, us2) and torch.equal(vs1, vs2)
    u3, v3 = fg.velocity(x, y, g)
    u4, v4 = fg.velocity(x, y, g)  # replay
    torch.cuda.synchronize()
    for a, b in ((u1, u2), (v1, v2), (u1, u3), (v1, v3), (u1, u4), (v1, v4)):
        assert torch.equal(a, b)


@pytest.mark.parametrize("pinned", [False, True])
@pytest.mark.parametrize("domain", ["explicit", "bbox"])
def test_host_entry_point_equals_device(lib, pinned, domain):
    """Host buffers (pageable: copied; page-locked with an explicit square: read in place by the key kernel)
    give the device entry point's bits."""
    w = fi.uniform(30000, seed_index=41, depth=5, p=12)
    f = lib.FMM(w.depth, w.p, w.sigma, precision="mixed", domain=w.domain if domain == "explicit" else None)
    u, v = f.velocity(dev(w.x), dev(w.y), dev(w.gamma))
    hx, hy, hg = (torch.from_numpy(a) for a in (w.x, w.y, w.gamma))
    uo, vo = torch.empty(w.n, dtype=torch.float64), torch.empty(w.n, dtype=torch.float64)
    if pinned:
        hx, hy, hg, uo, vo = (t.pin_memory() for t in (hx, hy, hg, uo, vo))
    for _ in range(2):
        uh, vh = f.velocity_host(hx, hy, hg, uo, vo)
        assert torch.equal(u.cpu(), uh) and torch.equal(v.cpu(), vh)


def test_edge_cases(lib, oracle):
    from paper_1008_2410_gb300._lib import FMMError

    f = lib.FMM(3, 8, 0.01, domain=(0.0, 0.0, 1.0))
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    u, v = f.velocity(e, e, e)
    assert u.numel() == 0
    # one particle: no other particle acts on it
    one = dev([0.3])
    u, v = f.velocity(one, one, one)
    f.sync()
    assert u.item() == 0.0 and v.item() == 0.0
    # coincident particles, points on leaf edges and on the square's upper edge, an empty system of leaves
    x = np.array([0.25, 0.25, 0.5, 0.125, 1.0, 0.0, 0.999999, 0.6])
    y = np.array([0.25, 0.25, 0.5, 0.875, 1.0, 0.0, 0.000001, 0.6])
    g = np.array([1.0, -2.0, 0.5, 0.3, 0.7, -0.1, 0.2, 0.9])
    for prec, tol in (("fp64", TOL64), ("mixed", TOL32)):
        f2 = lib.FMM(3, 8, 0.01, precision=prec, domain=(0.0, 0.0, 1.0))
        u, v = f2.velocity(dev(x), dev(y), dev(g))
        f2.sync()
        uo, vo, _ = oracle.fmm(x, y, g, 0.01, 3, 8, domain=(0.0, 0.0, 1.0))
        assert rel_l2((u.cpu().numpy(), v.cpu().numpy()), (uo, vo)) < tol
    # every particle in one leaf
    w = fi.uniform(3000, seed_index=42, depth=3, p=8)
    xs, ys = 0.1 + 0.01 * w.x, 0.1 + 0.01 * w.y
    u, v, _ = run(lib, fi.Workload("one_leaf", xs, ys, w.gamma, 1e-3, 3, 8, (0.0, 0.0, 1.0)))
    uo, vo, _ = oracle.fmm(xs, ys, w.gamma, 1e-3, 3, 8, domain=(0.0, 0.0, 1.0))
    assert rel_l2((u, v), (uo, vo)) < TOL64
    # a point outside the explicit square and a NaN are reported as FMM_EINVAL, and the handle stays usable
    for bad in ([0.5, 1.5], [0.5, float("nan")]):
        f3 = lib.FMM(3, 8, 0.01, domain=(0.0, 0.0, 1.0))
        f3.velocity(dev(bad), dev([0.5, 0.5]), dev([1.0, 1.0]))
        with pytest.raises(FMMError) as ei:
            f3.sync()
        assert ei.value.status == 1
        u, v = f3.velocity(dev([0.2, 0.4]), dev([0.5, 0.5]), dev([1.0, 1.0]))
        f3.sync()
    with pytest.raises(FMMError):
        lib.FMM(13, 8, 0.01)
    with pytest.raises(FMMError):
        lib.FMM(3, 33, 0.01)
    with pytest.raises(FMMError):
        lib.FMM(3, 8, -1.0)


def test_batched_systems_match_single_evaluations(lib, oracle):
    b = fi.batched(nsys=6, nmin=500, nmax=20000, p=10, seed_index=43)
    off = b.offsets
    x = np.concatenate([s.x for s in b.systems])
    y = np.concatenate([s.y for s in b.systems])
    g = np.concatenate([s.gamma for s in b.systems])
    depths = [s.depth for s in b.systems]
    sigmas = [s.sigma for s in b.systems]
    doms = [s.domain for s in b.systems]
    # the precision form with either M2L engine (the tensor-core kernel indexes its tiles per system and level)
    for prec, tol, eng in (("fp64", TOL64, None), ("mixed", TOL32, "cuda_cores"), ("mixed", TOL32, "tensor")):
        f = lib.FMM(3, b.p, 0.01, precision=prec, graph=True, m2l_engine=eng)
        u, v = f.velocity_batched(off, dev(x), dev(y), dev(g), depths=depths, sigmas=sigmas, domains=doms)
        f.sync()
        u, v = u.cpu().numpy(), v.cpu().numpy()
        for k, s in enumerate(b.systems):
            uo, vo, _ = oracle.fmm(s.x, s.y, s.gamma, s.sigma, s.depth, b.p, domain=s.domain)
            sl = slice(off[k], off[k + 1])
            assert rel_l2((u[sl], v[sl]), (uo, vo)) < tol, (prec, eng, k)
    # bounding-box rule per system, and an empty system in the middle
    off2 = np.array([0, off[1], off[1], off[2]])
    f = lib.FMM(3, b.p, 0.01)
    n2 = off[2]
    u, v = f.velocity_batched(off2, dev(x[:n2]), dev(y[:n2]), dev(g[:n2]), depths=[depths[0], 2, depths[1]],
                              sigmas=[sigmas[0], 1.0, sigmas[1]])
    f.sync()
    u, v = u.cpu().numpy(), v.cpu().numpy()
    for k, sys_k in ((0, 0), (2, 1)):
        s = b.systems[sys_k]
        uo, vo, _ = oracle.fmm(s.x, s.y, s.gamma, s.sigma, s.depth, b.p, domain=None)
        sl = slice(off2[k], off2[k + 1])
        assert rel_l2((u[sl], v[sl]), (uo, vo)) < TOL64


def test_adjoint_matches_oracle(lib, oracle):
    w = fi.uniform(6000, seed_index=44, depth=4, p=12)
    rs = np.random.default_rng(9)
    gu, gv = rs.normal(size=w.n), rs.normal(size=w.n)
    f = lib.FMM(w.depth, w.p, w.sigma, domain=w.domain)
    dg, dx, dy = f.adjoint(dev(w.x), dev(w.y), dev(w.gamma), dev(gu), dev(gv))
    f.sync()
    og, ox, oy = oracle.fmm_adjoint(w.x, w.y, w.gamma, w.sigma, w.depth, w.p, gu, gv, domain=w.domain)
    assert rel_l2((dg.cpu().numpy(),), (og,)) < 1e-11
    assert rel_l2((dx.cpu().numpy(), dy.cpu().numpy()), (ox, oy)) < 1e-10


@pytest.mark.parametrize("name,make,tol", [
    ("uniform6000_d4_p12", lambda: fi.uniform(6000, seed_index=44, depth=4, p=12), 1e-6),
    ("clustered20k_d5_p14", lambda: fi.clustered(20000, depth=5, p=14), 5e-6),
    ("lattice_lamb_oseen", lambda: fi.lattice_lamb_oseen(), 1e-6),
])
def test_adjoint_fp32_near_field_matches_oracle(lib, oracle, name, make, tol):
    """fmm_set_adjoint_precision(FMM_MIXED): the near-field part of the adjoint in FP32 (series for the small-r
    factors of K_sigma and its derivative) against the oracle's transposed stages; dense leaves (the clustered case)
    carry the largest FP32 coordinate rounding."""
    w = make()
    rs = np.random.default_rng(9)
    gu, gv = rs.normal(size=w.n), rs.normal(size=w.n)
    f = lib.FMM(w.depth, w.p, w.sigma, domain=w.domain)
    f.set_adjoint_precision("mixed")
    dg, dx, dy = f.adjoint(dev(w.x), dev(w.y), dev(w.gamma), dev(gu), dev(gv))
    f.sync()
    og, ox, oy = oracle.fmm_adjoint(w.x, w.y, w.gamma, w.sigma, w.depth, w.p, gu, gv, domain=w.domain)
    assert rel_l2((dg.cpu().numpy(),), (og,)) < tol
    assert rel_l2((dx.cpu().numpy(), dy.cpu().numpy()), (ox, oy)) < 2 * tol


def test_autograd_function_finite_differences(lib):
    w = fi.uniform(3000, seed_index=45, depth=3, p=14)
    f = lib.FMM(w.depth, w.p, w.sigma, domain=w.domain)
    x = dev(w.x).requires_grad_(True)
    y = dev(w.y).requires_grad_(True)
    g = dev(w.gamma).requires_grad_(True)
    ustar = dev(np.zeros(w.n))
    u, v = lib.fmm_velocity(x, y, g, f)
    L = 0.5 * ((u - ustar) ** 2).sum() + 0.5 * (v**2).sum()
    L.backward()

    def loss(xx, yy, gg):
        uu, vv = f.velocity(xx, yy, gg)
        return float(0.5 * (uu**2).sum() + 0.5 * (vv**2).sum())

    rs = np.random.default_rng(10)
    for j in rs.choice(w.n, 5, replace=False):
        # position step 1e-6: smaller steps drown the difference in the rounding of the evaluation itself
        for arr, grad, h in ((g, g.grad, 1e-6 / w.n), (x, x.grad, 1e-6), (y, y.grad, 1e-6)):
            base = arr.detach().clone()
            p_, m_ = base.clone(), base.clone()
            p_[j] += h
            m_[j] -= h
            args_p = [x.detach(), y.detach(), g.detach()]
            args_m = [x.detach(), y.detach(), g.detach()]
            idx = 0 if arr is x else (1 if arr is y else 2)
            args_p[idx], args_m[idx] = p_, m_
            fd = (loss(*args_p) - loss(*args_m)) / (2 * h)
            an = grad[j].item()
            assert abs(fd - an) <= 1e-5 * max(abs(an), 1e-6 * float(grad.abs().max())), (idx, j, fd, an)


def test_autograd_direct_limit_matches_torch_direct_sum(lib):
    """Depth 1 (every pair near): gradients equal autograd through a torch FP64 Eq. 7 sum at N = 4096."""
    w = fi.uniform(4096, seed_index=46, depth=1, p=8)
    f = lib.FMM(1, 8, w.sigma, domain=w.domain)
    x = dev(w.x).requires_grad_(True)
    y = dev(w.y).requires_grad_(True)
    g = dev(w.gamma).requires_grad_(True)
    u, v = lib.fmm_velocity(x, y, g, f)
    ustar = dev(np.random.default_rng(11).normal(size=w.n) * 1e-3)
    L = 0.5 * ((u - ustar) ** 2).sum() + 0.5 * (v**2).sum()
    L.backward()
    xr = dev(w.x).requires_grad_(True)
    yr = dev(w.y).requires_grad_(True)
    gr = dev(w.gamma).requires_grad_(True)
    a = xr[:, None] - xr[None, :]
    b = yr[:, None] - yr[None, :]
    eye = torch.eye(w.n, dtype=torch.bool, device="cuda")
    r2 = torch.where(eye, torch.ones_like(a), a * a + b * b)
    fk = torch.where(eye, torch.zeros_like(a), -torch.expm1(-r2 / (2 * w.sigma**2)) / (2 * math.pi * r2))
    ur = torch.sum(gr[None, :] * (-b) * fk, dim=1)
    vr = torch.sum(gr[None, :] * a * fk, dim=1)
    Lr = 0.5 * ((ur - ustar) ** 2).sum() + 0.5 * (vr**2).sum()
    Lr.backward()
    for got, ref in ((g.grad, gr.grad), (x.grad, xr.grad), (y.grad, yr.grad)):
        assert float((got - ref).norm() / ref.norm()) < 1e-11


def test_stage_times_launch_count_and_autotune(lib):
    w = fi.uniform(50000, seed_index=47, depth=5, p=12)
    f = lib.FMM(w.depth, w.p, w.sigma, precision="mixed", domain=w.domain)
    f.set_timing(True)
    x, y, g = dev(w.x), dev(w.y), dev(w.gamma)
    n0 = f.kernel_launches()
    f.velocity(x, y, g)
    t = f.stage_times()
    assert len(t) == 8 and all(v >= 0 for v in t) and t[6] > 0
    assert f.kernel_launches() > n0 + 8
    prm = f.autotune(x, y, g, 4, 6)
    assert 4 <= prm["depth"] <= 6
    assert prm["p2p_threads"] in (32, 64, 128, 192, 256) and prm["p2p_targets_per_thread"] in (2, 4)
    assert prm["m2l_engine"] in ("tensor", "cuda_cores")


@pytest.mark.slow
def test_batched_64_systems_full_size_sampled_parity(lib, oracle):
    """The full batched workload: 64 uniform systems of 4096 .. 262144 particles (4.5 M in all), each at its own
    depth round(log4(N_k / 64)), p = 14, one graph launch per stage, in both forms; 128 sampled targets per system
    against the oracle FMM of that system."""
    b = fi.batched()
    off = b.offsets
    x = np.concatenate([s.x for s in b.systems])
    y = np.concatenate([s.y for s in b.systems])
    g = np.concatenate([s.gamma for s in b.systems])
    kw = dict(depths=[s.depth for s in b.systems], sigmas=[s.sigma for s in b.systems],
              domains=[s.domain for s in b.systems])
    res = {}
    for prec in ("fp64", "mixed"):
        f = lib.FMM(b.systems[0].depth, b.p, b.systems[0].sigma, precision=prec, graph=True)
        xd, yd, gd = dev(x), dev(y), dev(g)
        u, v = f.velocity_batched(off, xd, yd, gd, **kw)
        f.velocity_batched(off, xd, yd, gd, u=u, v=v, **kw)  # a replay of the captured graph
        f.sync()
        res[prec] = (u.cpu().numpy(), v.cpu().numpy())
        f.close()
    for k, sy in enumerate(b.systems):
        t = fi.sample_targets(sy.n, 128, seed_index=100 + k)
        uo, vo, _ = oracle.fmm(sy.x, sy.y, sy.gamma, sy.sigma, sy.depth, b.p, domain=sy.domain, targets=t)
        for prec, tol in (("fp64", TOL64), ("mixed", TOL32)):
            u, v = res[prec]
            assert rel_l2((u[off[k]:off[k + 1]][t], v[off[k]:off[k + 1]][t]), (uo, vo)) < tol, (prec, k)


@pytest.mark.slow
def test_adjoint_full_size_config5_loss(lib, oracle):
    """The adjoint at 2^20 uniform particles (depth 7, p = 17) for the loss L = 1/2 |u - u*|^2, u* the FMM velocity
    of the perturbed circulations: dL/dgamma, dL/dx, dL/dy against the oracle's transposed stages."""
    w = fi.uniform_1m()
    gs = fi.adjoint_target_gamma(w)
    f = lib.FMM(w.depth, w.p, w.sigma, precision="fp64", domain=w.domain)
    x, y, g = dev(w.x), dev(w.y), dev(w.gamma)
    us, vs = f.velocity(x, y, dev(gs))
    u, v = f.velocity(x, y, g)
    gu, gv = u - us, v - vs
    dg, dx, dy = f.adjoint(x, y, g, gu, gv)
    f.sync()
    og, ox, oy = oracle.fmm_adjoint(w.x, w.y, w.gamma, w.sigma, w.depth, w.p, gu.cpu().numpy(), gv.cpu().numpy(),
                                    domain=w.domain)
    assert rel_l2((dg.cpu().numpy(),), (og,)) < 1e-11
    assert rel_l2((dx.cpu().numpy(), dy.cpu().numpy()), (ox, oy)) < 1e-10


def test_suggested_depth_reaches_eq7_on_the_gpu(lib, oracle):
    """§2: the expansions carry the point-vortex kernel, so the FMM misses the Gaussian tail of pairs beyond adjacent
    leaves. On the Lamb-Oseen lattice the GPU evaluation at fmm_suggest_depth's depth (3 for a tail tolerance of
    1e-12: leaves 8 sigma wide) matches the direct sum of Eq. 7 to 1e-12 in the FP64 form (p = 30) and to 1e-6 in
    the precision form, while at depth 4 (leaves 4 sigma wide) it stays tail-limited above 1e-7."""
    w = fi.lattice_lamb_oseen()
    d = lib.suggest_depth(w.n, w.sigma, w.domain[2], tail_tol=1e-12)
    assert d == 3
    t = fi.sample_targets(w.n, 512)
    ud, vd = oracle.direct(w.x, w.y, w.gamma, w.sigma, targets=t)
    x, y, g = dev(w.x), dev(w.y), dev(w.gamma)
    errs = {}
    for depth, prec in ((d, "fp64"), (d, "mixed"), (4, "fp64")):
        f = lib.FMM(depth, 30, w.sigma, precision=prec, domain=w.domain)
        u, v = f.velocity(x, y, g)
        f.sync()
        errs[(depth, prec)] = rel_l2((u.cpu().numpy()[t], v.cpu().numpy()[t]), (ud, vd))
    assert errs[(d, "fp64")] < 1e-12
    assert errs[(d, "mixed")] < TOL32
    assert errs[(4, "fp64")] > 1e-7


@pytest.mark.parametrize("leaf_capacity", [0, 24])
def test_default_engine_and_stage_events_in_graph_replays(lib, leaf_capacity):
    """A fresh handle runs the FP32 M2L levels on the CUDA cores; with graphs on, the stage events are graph nodes,
    so a far-only replay reports its fork-to-join span (the sweep alone) and a near-only replay none of it."""
    w = fi.clustered(30000, depth=6, p=12) if leaf_capacity else fi.uniform(50000, seed_index=48, depth=5, p=12)
    f = lib.FMM(w.depth, w.p, w.sigma, precision="mixed", domain=w.domain, graph=True, leaf_capacity=leaf_capacity)
    assert f.params()["m2l_engine"] == "cuda_cores"
    f.set_timing(True)
    x, y, g = dev(w.x), dev(w.y), dev(w.gamma)
    u, v = torch.empty_like(x), torch.empty_like(x)
    for _ in range(2):  # capture, then replay
        f.velocity_far(x, y, g, u, v)
    t = f.stage_times()
    assert len(t) == 8 and t[7] > 0 and t[6] >= t[7]
    if not leaf_capacity:  # uniform tree: no near-field kernel between the fork and the join's event nodes
        assert t[1] < 0.5 * t[7]
    for _ in range(2):
        f.velocity_near(x, y, g, u, v)
    t = f.stage_times()
    assert len(t) == 8 and t[1] > 0 and t[2] == 0 and t[3] == 0
    for _ in range(2):
        f.velocity(x, y, g, u, v)
    t = f.stage_times()
    assert all(t[k] > 0 for k in ((0, 1, 2, 3, 6, 7) if leaf_capacity else (0, 1, 2, 3, 4, 6, 7)))
    f.sync()


@pytest.mark.parametrize("precision,tol,case", [("fp64", TOL64, "lattice"), ("fp64", TOL64, "narrow"),
                                                ("mixed", TOL32, "narrow")])
def test_far_tail_matches_oracle(lib, oracle, precision, tol, case):
    """The regularised far-field correction: the GPU evaluation with it equals the oracle FMM plus the oracle's
    brute-force correction, and the correction alone (with minus without) equals the oracle's. On the lattice
    (leaves 4 sigma wide, one ring) the correction is 1.6e-7 of the velocity and at p = 20 it takes the FMM from
    that gap to Eq. 7 down to truncation; on leaves 1.5 sigma wide (three rings) it is 2.5 per cent of the velocity,
    large enough to check the precision form's FP32 correction (and the FMM then meets Eq. 7 to 3.5e-7 instead of
    2.5e-2)."""
    if case == "lattice":
        w, rings = fi.lattice_lamb_oseen(), 1
    else:
        w, rings = fi.uniform(20000, seed_index=44, depth=5, p=14, sigma=1.0 / 32 / 1.5), 3
    x, y, g = dev(w.x), dev(w.y), dev(w.gamma)
    f = lib.FMM(w.depth, w.p, w.sigma, precision=precision, domain=w.domain)
    u0, v0 = f.velocity(x, y, g)
    f.set_far_tail(rings)
    u1, v1 = f.velocity(x, y, g)
    f.sync()
    uo, vo, _ = oracle.fmm(w.x, w.y, w.gamma, w.sigma, w.depth, w.p, domain=w.domain)
    ut, vt = oracle.far_tail(w.x, w.y, w.gamma, w.sigma, w.depth, rings, domain=w.domain)
    got = (u1.cpu().numpy(), v1.cpu().numpy())
    assert rel_l2(got, (uo + ut, vo + vt)) < tol
    dcorr = (got[0] - u0.cpu().numpy(), got[1] - v0.cpu().numpy())
    assert rel_l2(dcorr, (ut, vt)) < (1e-9 if precision == "fp64" else 1e-4)
    if case == "lattice":
        ud, vd = oracle.direct(w.x, w.y, w.gamma, w.sigma)
        f20 = lib.FMM(w.depth, 20, w.sigma, precision="fp64", domain=w.domain)
        a0 = f20.velocity(x, y, g)
        f20.set_far_tail(1)
        a1 = f20.velocity(x, y, g)
        f20.sync()
        e0 = rel_l2((a0[0].cpu().numpy(), a0[1].cpu().numpy()), (ud, vd))
        e1 = rel_l2((a1[0].cpu().numpy(), a1[1].cpu().numpy()), (ud, vd))
        assert e1 < e0 / 10


def test_far_tail_rejected_where_not_built(lib):
    """The correction runs on the uniform tree's forward evaluation only: the adaptive tree, the adjoint and the
    level exchange refuse a handle with it on, and the handle works again once it is off."""
    w = fi.uniform(3000, seed_index=43, depth=3, p=10)
    x, y, g = dev(w.x), dev(w.y), dev(w.gamma)
    fa = lib.FMM(6, w.p, w.sigma, precision="mixed", domain=w.domain, leaf_capacity=32)
    fa.set_far_tail(1)
    with pytest.raises(RuntimeError):
        fa.velocity(x, y, g)
    fa.set_far_tail(0)
    fa.velocity(x, y, g)
    fa.sync()
    f = lib.FMM(w.depth, w.p, w.sigma, precision="fp64", domain=w.domain)
    f.set_far_tail(1)
    with pytest.raises(RuntimeError):
        f.adjoint(x, y, g, torch.ones_like(x), torch.ones_like(x))
    with pytest.raises(RuntimeError):
        f.level_multipoles(x, y, g, 2)
    f.set_far_tail(0)
    f.adjoint(x, y, g, torch.ones_like(x), torch.ones_like(x))
    f.sync()


def test_near_field_only_stage_events(lib):
    """Timing mode "near" (the bench's timed steps): only the near field's two events are graph nodes, so stage 1
    reads the near field and every other stage reads 0; the results equal an untimed evaluation's bit for bit."""
    w = fi.uniform(50000, seed_index=48, depth=5, p=12)
    f = lib.FMM(w.depth, w.p, w.sigma, precision="mixed", domain=w.domain, graph=True)
    x, y, g = dev(w.x), dev(w.y), dev(w.gamma)
    u0, v0 = f.velocity(x, y, g)
    f.set_timing("near")
    u, v = torch.empty_like(x), torch.empty_like(x)
    for _ in range(2):  # capture, then replay
        f.velocity(x, y, g, u, v)
    t = f.stage_times()
    assert len(t) == 8 and t[1] > 0 and all(t[k] == 0 for k in (0, 2, 3, 4, 5, 6, 7))
    assert torch.equal(u, u0) and torch.equal(v, v0)
    f.sync()


@pytest.mark.slow
@pytest.mark.parametrize("precision,graph,engine", [("mixed", True, None), ("fp64", True, None),
                                                    ("mixed", True, "tensor")])
def test_uniform_1m_sampled_parity(lib, oracle, precision, graph, engine):
    """The 2^20-particle uniform workload (depth 7, p = 17) in the launch configuration the bench times,
    checked at 2048 sampled targets against the oracle FMM; also with the FP32 M2L levels on the tensor cores
    (full 256-position tiles at level 7 and the largest K bucket)."""
    w = fi.uniform_1m()
    u, v, _ = run(lib, w, precision=precision, graph=graph, m2l_engine=engine)
    t = fi.sample_targets(w.n, 2048)
    uo, vo, _ = oracle.fmm(w.x, w.y, w.gamma, w.sigma, w.depth, w.p, domain=w.domain, targets=t)
    assert rel_l2((u[t], v[t]), (uo, vo)) < (TOL64 if precision == "fp64" else TOL32)


@pytest.mark.slow
def test_patches_16m_sampled_parity(lib, oracle):
    """The 2^24-particle 8-patch workload (depth 9, p = 20), precision form, at 512 sampled targets."""
    w = fi.patches_16m()
    u, v, _ = run(lib, w, precision="mixed", graph=True)
    t = fi.sample_targets(w.n, 512)
    uo, vo, _ = oracle.fmm(w.x, w.y, w.gamma, w.sigma, w.depth, w.p, domain=w.domain, targets=t)
    assert rel_l2((u[t], v[t]), (uo, vo)) < TOL32


# ---------------------------------------------------------------------------------------- Eq. 3 (advection)


def _advect_case():
    w = fi.uniform(20000, seed_index=82, depth=4, p=14)
    return w


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-6)])
def test_advect_matches_oracle(lib, oracle, order, precision, tol):
    """Runge-Kutta steps of the particles (Eq. 3) with FMM velocities: displacement against the oracle's same
    scheme, bounding-box root square recomputed at every stage on both sides."""
    w = _advect_case()
    u0, v0, _ = oracle.fmm(w.x, w.y, w.gamma, w.sigma, w.depth, w.p, domain=None)
    dt = 0.05 * w.sigma / float(np.hypot(u0, v0).max())
    nsteps = 3
    xo, yo = oracle.advect(w.x, w.y, w.gamma, w.sigma, w.depth, w.p, dt, nsteps, order=order, domain=None)
    f = lib.FMM(w.depth, w.p, w.sigma, precision=precision)
    x, y, g = dev(w.x), dev(w.y), dev(w.gamma)
    f.advect(x, y, g, dt, nsteps, order)
    f.sync()
    dx, dy = x.cpu().numpy() - w.x, y.cpu().numpy() - w.y
    assert rel_l2((dx, dy), (xo - w.x, yo - w.y)) < tol
    if precision == "fp64":  # linear impulse: sum gamma_i u_i = 0 at every stage
        assert abs(np.dot(w.gamma, dx)) < 1e-12 * np.dot(np.abs(w.gamma), np.abs(dx))
        assert abs(np.dot(w.gamma, dy)) < 1e-12 * np.dot(np.abs(w.gamma), np.abs(dy))


def test_advect_lamb_oseen_lattice_and_graph_replay(lib, oracle):
    """The Lamb-Oseen lattice in its explicit square [-1, 1]^2 (FP64 form) follows the oracle's RK4 steps; a
    graph-replayed handle gives the same bits as an eager one."""
    w = fi.lattice_lamb_oseen()
    dt, nsteps = 0.01, 2
    xo, yo = oracle.advect(w.x, w.y, w.gamma, w.sigma, w.depth, w.p, dt, nsteps, order=4, domain=w.domain)
    outs = []
    for graph in (False, True):
        f = lib.FMM(w.depth, w.p, w.sigma, domain=w.domain, graph=graph)
        x, y, g = dev(w.x), dev(w.y), dev(w.gamma)
        f.advect(x, y, g, dt, nsteps, 4)
        f.sync()
        outs.append((x, y))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    dx, dy = outs[0][0].cpu().numpy() - w.x, outs[0][1].cpu().numpy() - w.y
    assert rel_l2((dx, dy), (xo - w.x, yo - w.y)) < 1e-10


def test_advect_rejects_bad_arguments(lib):
    w = fi.uniform(100, seed_index=83, depth=2, p=8)
    f = lib.FMM(w.depth, w.p, w.sigma)
    x, y, g = dev(w.x), dev(w.y), dev(w.gamma)
    from paper_1008_2410_gb300._lib import FMMError

    for args in ((0.1, 1, 3), (0.1, -1, 2), (float("nan"), 1, 2)):
        with pytest.raises(FMMError):
            f.advect(x, y, g, *args)
    f.advect(x, y, g, 0.1, 0, 2)  # zero steps: nothing happens
    assert torch.equal(x, dev(w.x))


# ---------------------------------------------------------------------------------------- failure reporting


def test_bounded_wait_timeout_reaches_the_host_and_the_handle_recovers(lib):
    """The bounded device wait (the one guarding every bulk copy of the near field) is made to run out on a
    barrier that nothing completes: fmm_sync returns FMM_ETIMEOUT, and the same handle then evaluates correctly."""
    from paper_1008_2410_gb300 import _lib

    w = fi.uniform(4000, seed_index=49, depth=3, p=10)
    f = lib.FMM(w.depth, w.p, w.sigma, precision="mixed", domain=w.domain)
    x, y, g = dev(w.x), dev(w.y), dev(w.gamma)
    u0, v0 = f.velocity(x, y, g)
    f.sync()
    f.selftest_timeout(4096)
    with pytest.raises(_lib.FMMError) as err:
        f.sync()
    assert err.value.status == _lib.FMM_ETIMEOUT
    f.sync()  # reported once
    u1, v1 = f.velocity(x, y, g)
    f.sync()
    assert torch.equal(u0, u1) and torch.equal(v0, v1)
    # on a fresh handle that has not evaluated anything yet
    f2 = lib.FMM(w.depth, w.p, w.sigma, precision="mixed", domain=w.domain)
    f2.selftest_timeout(64)
    with pytest.raises(_lib.FMMError) as err:
        f2.sync()
    assert err.value.status == _lib.FMM_ETIMEOUT
    with pytest.raises(_lib.FMMError):
        f2.selftest_timeout(0)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 1e-6)])
def test_autotune_p_meets_the_target_against_the_oracle(lib, oracle, precision, tol):
    """fmm_autotune_p keeps the smallest p whose evaluation is within the target of the FP64 form at p = 32; the
    chosen p's GPU result checked on a sample against the oracle's split sum (what the FMM converges to, §2) stays
    within the target (the estimate is global, the check sampled: a factor 3 of slack), and p - 1 misses it."""
    w = fi.uniform(60000, seed_index=50, depth=5, p=17)
    f = lib.FMM(w.depth, w.p, w.sigma, precision=precision, domain=w.domain)
    x, y, g = dev(w.x), dev(w.y), dev(w.gamma)
    p, est = f.autotune_p(x, y, g, tol, 2, 30)
    assert 2 < p <= 30 and est <= tol
    u, v = f.velocity(x, y, g)
    f.sync()
    t = fi.sample_targets(w.n, 400)
    us, vs = oracle.split_direct(w.x, w.y, w.gamma, w.sigma, w.depth, domain=w.domain, targets=t)
    assert rel_l2((u.cpu().numpy()[t], v.cpu().numpy()[t]), (us, vs)) < 3 * tol
    f2 = lib.FMM(w.depth, w.p, w.sigma, precision=precision, domain=w.domain)
    p2, est2 = f2.autotune_p(x, y, g, tol, p - 1, p - 1)
    assert p2 == p - 1 and est2 > tol


def test_autotune_batched_picks_depths_and_tile(lib, oracle):
    """fmm_autotune_batched times leaf occupancies and tiles; the chosen depths follow round(log4(N_k / B)) for one
    of its occupancies B, and the batch evaluated with them matches the oracle per system."""
    b = fi.batched(nsys=5, nmin=2000, nmax=30000, p=10, seed_index=44)
    off = b.offsets
    x = np.concatenate([s.x for s in b.systems])
    y = np.concatenate([s.y for s in b.systems])
    g = np.concatenate([s.gamma for s in b.systems])
    sig = [s.sigma for s in b.systems]
    doms = [s.domain for s in b.systems]
    f = lib.FMM(3, b.p, 0.01, precision="mixed", graph=True)
    xd, yd, gd = dev(x), dev(y), dev(g)
    prm = f.autotune_batched(off, xd, yd, gd, sigmas=sig, domains=doms)
    deps = prm["depths"]
    assert len(deps) == len(b.systems)
    assert any(all(d == max(0, min(12, round(math.log(s.n / occ, 4)))) for d, s in zip(deps, b.systems))
               for occ in (16, 32, 48, 64, 96, 128))
    assert prm["p2p_threads"] in (32, 64, 128, 192, 256) and prm["p2p_targets_per_thread"] in (2, 4)
    u, v = f.velocity_batched(off, xd, yd, gd, depths=deps, sigmas=sig, domains=doms)
    f.sync()
    u, v = u.cpu().numpy(), v.cpu().numpy()
    for k, s in enumerate(b.systems):
        uo, vo, _ = oracle.fmm(s.x, s.y, s.gamma, s.sigma, deps[k], b.p, domain=s.domain)
        assert rel_l2((u[off[k]:off[k + 1]], v[off[k]:off[k + 1]]), (uo, vo)) < TOL32, k


def test_probe_peaks_reports_every_unit(lib):
    """The throughput probe returns finite, positive rates for the FP32, FP64 and SFU pipes, the SM count, and the
    cycles per TF32 tensor-core MMA at N = 48 and N = 256 (the figures the M2L engine choice rests on)."""
    from paper_1008_2410_gb300 import _lib

    pk = _lib.probe_peaks()
    for k in ("fp32_tflops", "fp64_tflops", "sfu_tops", "tf32_mma_cycles_n48", "tf32_mma_cycles_n256"):
        assert np.isfinite(pk[k]) and pk[k] > 0, k
    assert pk["sms"] > 0
