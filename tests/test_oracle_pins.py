"""Pins of the FP64 CPU oracle against facts fixed by the paper and by the mathematics (no GPU).

Each test checks the oracle against something other than its own formulas: a quadrature of the
Biot-Savart integral (Eqs. 2 and 5), the Lamb-Oseen closed form, impulse invariants that follow from the
kernel's antisymmetry, the analytic point-vortex field, the §3 near-field pair-count formula, and the
geometric convergence of the truncated expansions.
"""
import math

import numpy as np
import pytest

import fmm_inputs as fi


def rel_l2(a, b):
    a = np.concatenate([np.ravel(t) for t in a]) if isinstance(a, tuple) else np.ravel(a)
    b = np.concatenate([np.ravel(t) for t in b]) if isinstance(b, tuple) else np.ravel(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# ---------------------------------------------------------------------------------------- Eq. 6


def _biot_savart_quadrature(px, py, sigma, nr=400, nt=256):
    """Velocity of one Gaussian blob (Eq. 2, centred at 0) at (px, py) by quadrature of Eq. 5 in polar
    coordinates about the evaluation point: u = 1/(2 pi) int int omega(x + rho e_theta) (sin t, -cos t) drho dt."""
    rmax = math.hypot(px, py) + 12.0 * sigma
    xg, wg = np.polynomial.legendre.leggauss(nr)
    rho = 0.5 * rmax * (xg + 1.0)
    wr = 0.5 * rmax * wg
    th = 2.0 * math.pi * np.arange(nt) / nt
    R, T = np.meshgrid(rho, th, indexing="ij")
    qx, qy = px + R * np.cos(T), py + R * np.sin(T)
    om = np.exp(-(qx * qx + qy * qy) / (2 * sigma * sigma)) / (2 * math.pi * sigma * sigma)
    wt = (wr[:, None] * (2 * math.pi / nt)) / (2 * math.pi)
    u = np.sum(wt * om * np.sin(T))
    v = np.sum(wt * om * -np.cos(T))
    return u, v


@pytest.mark.parametrize("pt", [(0.3, 0.1), (-0.05, 0.02), (0.01, -0.4), (1e-3, 2e-3)])
def test_kernel_is_biot_savart_of_gaussian_blob(oracle, pt):
    """Eq. 6 is the analytic Biot-Savart integral (Eq. 5) of the Gaussian basis (Eq. 2), sign included."""
    sigma = 0.07
    ku, kv = oracle.kernel(pt[0], pt[1], sigma)
    qu, qv = _biot_savart_quadrature(pt[0], pt[1], sigma)
    scale = math.hypot(qu, qv)
    assert abs(ku - qu) <= 1e-9 * scale + 1e-14
    assert abs(kv - qv) <= 1e-9 * scale + 1e-14


def test_kernel_limits_and_symmetry(oracle):
    sigma = 0.01
    assert oracle.kernel(0.0, 0.0, sigma) == (0.0, 0.0)  # K_sigma(0) := 0
    rs = np.random.default_rng(0)
    for _ in range(50):
        a, b = rs.normal(size=2) * 0.03
        ku, kv = oracle.kernel(a, b, sigma)
        mu, mv = oracle.kernel(-a, -b, sigma)
        assert ku == -mu and kv == -mv  # odd kernel
        assert abs(ku * a + kv * b) <= 1e-15 * math.hypot(ku, kv) * math.hypot(a, b)  # K(z) is perpendicular to z
    # far away: point vortex 1/(2 pi r); near the centre: solid rotation (-b, a)/(4 pi sigma^2)
    ku, kv = oracle.kernel(0.0, 1.0, sigma)
    assert abs(ku + 1.0 / (2 * math.pi)) < 1e-15 and kv == 0.0
    a, b = 1e-7, 2e-7
    ku, kv = oracle.kernel(a, b, sigma)
    assert abs(ku - (-b) / (4 * math.pi * sigma**2)) < 1e-8 * abs(ku)
    assert abs(kv - a / (4 * math.pi * sigma**2)) < 1e-8 * abs(kv)


# ---------------------------------------------------------------------------------------- Eq. 7


def lamb_oseen_velocity(x, y, circulation, core2):
    """u_theta(r) = Gamma / (2 pi r) (1 - exp(-r^2 / r_c^2)) of the Lamb-Oseen vortex, as (u, v)."""
    r2 = x * x + y * y
    f = circulation * (-np.expm1(-r2 / core2)) / (2 * math.pi * r2)
    return -y * f, x * f


def test_direct_sum_matches_lamb_oseen(oracle):
    """Blob sum on the 128^2 lattice = Lamb-Oseen with r_c'^2 = r_c^2 + 2 sigma^2 (Gaussian * Gaussian);
    quadrature and domain-truncation errors are far below 1e-8."""
    w = fi.lattice_lamb_oseen()
    u, v = oracle.direct(w.x, w.y, w.gamma, w.sigma)
    core2 = w.extra["core"] ** 2 + 2 * w.sigma**2
    ue, ve = lamb_oseen_velocity(w.x, w.y, 1.0, core2)
    assert rel_l2((u, v), (ue, ve)) < 1e-8
    # the field is a solid body rotation about the centre: it is NOT close to the unsmoothed core value
    ue2, ve2 = lamb_oseen_velocity(w.x, w.y, 1.0, w.extra["core"] ** 2)
    assert rel_l2((u, v), (ue2, ve2)) > 1e-3


def test_direct_sum_impulse_invariants(oracle):
    """sum gamma_i u_i = sum gamma_i v_i = 0 (odd kernel) and sum gamma_i (x_i u_i + y_i v_i) = 0 (K(z) _|_ z)."""
    w = fi.uniform(3000, seed_index=21)
    u, v = oracle.direct(w.x, w.y, w.gamma, w.sigma)
    scale = np.sum(np.abs(w.gamma) * np.hypot(u, v))
    assert abs(np.sum(w.gamma * u)) < 1e-13 * scale
    assert abs(np.sum(w.gamma * v)) < 1e-13 * scale
    assert abs(np.sum(w.gamma * (w.x * u + w.y * v))) < 1e-13 * scale


def test_direct_sum_two_particles(oracle):
    """Two blobs: each moves with the other's K_sigma; a far pair moves as point vortices."""
    x = np.array([0.0, 0.5])
    y = np.array([0.0, 0.0])
    g = np.array([1.0, 2.0])
    u, v = oracle.direct(x, y, g, sigma=1e-3)
    # target 0, source 1 at distance 0.5 on the +x axis: z = -0.5 -> velocity (0, -g1/(2 pi 0.5))
    assert abs(u[0]) < 1e-18 and abs(v[0] + 2.0 / (2 * math.pi * 0.5)) < 1e-15
    assert abs(u[1]) < 1e-18 and abs(v[1] - 1.0 / (2 * math.pi * 0.5)) < 1e-15


def test_direct_sum_subset_targets(oracle):
    w = fi.uniform(500, seed_index=22)
    u, v = oracle.direct(w.x, w.y, w.gamma, w.sigma)
    t = fi.sample_targets(w.n, 37)
    us, vs = oracle.direct(w.x, w.y, w.gamma, w.sigma, targets=t)
    assert np.array_equal(us, u[t]) and np.array_equal(vs, v[t])


# ---------------------------------------------------------------------------------------- tree / lists


def test_leaf_binning_rule(oracle):
    dom = (0.0, 0.0, 1.0)
    x = np.array([0.0, 0.25, 0.2499999999, 0.999, 1.0, 0.5])
    y = np.array([0.0, 0.75, 0.1, 0.999, 1.0, 0.5])
    ix, iy = oracle.leaf_coords(x, y, 2, dom)
    assert ix.tolist() == [0, 1, 0, 3, 3, 2]  # ties go to the upper box, x = x0 + S to the last box
    assert iy.tolist() == [0, 3, 0, 3, 3, 2]
    with pytest.raises(ValueError):
        oracle.leaf_coords(np.array([1.0000001]), np.array([0.5]), 2, dom)
    d = oracle.default_domain(np.array([0.0, 2.0]), np.array([1.0, 1.5]))
    side = 2.0 * (1 + 2.0**-20)
    assert d[2] == side and d[0] == 1.0 - 0.5 * side and d[1] == 1.25 - 0.5 * side


def test_lattice_leaf_occupancy(oracle):
    """The 128^2 lattice at depth 4 puts exactly 8 x 8 = 64 particles in every leaf."""
    w = fi.lattice_lamb_oseen()
    ix, iy = oracle.leaf_coords(w.x, w.y, w.depth, w.domain)
    counts = np.bincount(iy.astype(np.int64) * 16 + ix, minlength=256)
    assert np.all(counts == 64)


def _brute_force_list_sizes(level):
    """Boxes at the same level that are not adjacent but whose parents are adjacent (set definition)."""
    ns = 1 << level
    out = np.zeros((ns, ns), np.int32)
    for by in range(ns):
        for bx in range(ns):
            c = 0
            for sy in range(ns):
                for sx in range(ns):
                    adj = abs(sx - bx) <= 1 and abs(sy - by) <= 1
                    padj = abs((sx >> 1) - (bx >> 1)) <= 1 and abs((sy >> 1) - (by >> 1)) <= 1
                    c += (not adj) and padj
            out[by, bx] = c
    return out


@pytest.mark.parametrize("level", [2, 3, 4, 5])
def test_interaction_lists(oracle, level):
    s = oracle.interaction_list_sizes(level)
    assert np.array_equal(s, _brute_force_list_sizes(level))
    assert s.max() == (12 if level == 2 else 27)  # §3: 27 is the maximum list size
    totals = {2: 156, 3: 1116, 4: 5628, 5: 25020}
    assert int(s.sum()) == totals[level]


def _paper_near_pairs(B, L):
    """§3 W_direct / 22: corner, edge and interior leaves of a uniform tree with B particles per leaf."""
    return 4 * (4 * B * B - B) + (2 ** (L + 2) - 8) * (6 * B * B - B) + (4**L - 2 ** (L + 2) + 4) * (9 * B * B - B)


@pytest.mark.parametrize("side,depth", [(128, 4), (64, 3), (32, 2), (96, 4)])
def test_near_field_pair_count(oracle, side, depth):
    """The oracle's stage-9 ordered pair count equals the paper's W_direct/22 on uniform lattices
    (config side 128, depth 4: 8,650,752)."""
    w = fi.lattice_lamb_oseen(side=side, depth=depth, p=4)
    _, _, npairs = oracle.fmm(w.x, w.y, w.gamma, w.sigma, depth, 4, domain=w.domain)
    B = (side // (1 << depth)) ** 2
    assert npairs == _paper_near_pairs(B, depth)
    if side == 128:
        assert npairs == 8650752


# ---------------------------------------------------------------------------------------- expansions


def test_p2m_far_field_is_point_vortex_sum(oracle):
    """sum_m a_m / dz^(m+1) of the §3 coefficients converges to sum_j q_j / (z - z_j), q = -i gamma / 2 pi."""
    rs = np.random.default_rng(1)
    xs, ys = rs.uniform(-0.5, 0.5, 20), rs.uniform(-0.5, 0.5, 20)
    g = rs.normal(size=20)
    q = -1j * g / (2 * math.pi)
    z = 2.2 + 1.3j
    exact = np.sum(q / (z - (xs + 1j * ys)))
    errs = []
    for p in (4, 8, 16, 32):
        a = oracle.p2m(xs, ys, q, 0j, p)
        errs.append(abs(oracle.multipole_eval(a, z) - exact) / abs(exact))
    assert errs[-1] < 1e-13
    assert errs[0] > errs[1] > errs[2]
    # velocity sign: u - i v of the far field equals the direct Eq. 6 sum at large distance
    su = sum(g[j] * oracle.kernel(z.real - xs[j], z.imag - ys[j], 1e-3)[0] for j in range(20))
    sv = sum(g[j] * oracle.kernel(z.real - xs[j], z.imag - ys[j], 1e-3)[1] for j in range(20))
    w = oracle.multipole_eval(oracle.p2m(xs, ys, q, 0j, 32), z)
    assert abs(w.real - su) < 1e-12 and abs(-w.imag - sv) < 1e-12


def test_m2m_is_exact(oracle):
    """M2M of a child expansion equals P2M about the parent centre, to rounding."""
    rs = np.random.default_rng(2)
    xs, ys = rs.uniform(0, 0.25, 30), rs.uniform(0.25, 0.5, 30)
    q = rs.normal(size=30) + 1j * rs.normal(size=30)
    p = 20
    cc, cp = 0.125 + 0.375j, 0.25 + 0.25j
    a_child = oracle.p2m(xs, ys, q, cc, p)
    a_parent = oracle.p2m(xs, ys, q, cp, p)
    moved = oracle.m2m(a_child, cc - cp)
    assert np.max(np.abs(moved - a_parent) / (np.abs(a_parent) + 1e-300)) < 1e-12


def test_l2l_is_exact(oracle):
    """A local expansion re-centred by L2L evaluates to the same polynomial."""
    rs = np.random.default_rng(3)
    p = 18
    b = rs.normal(size=p) + 1j * rs.normal(size=p)
    cp, cc = 0.5 + 0.5j, 0.25 + 0.75j
    bc = oracle.l2l(b, cc - cp)
    for _ in range(5):
        z = cc + complex(*rs.uniform(-0.25, 0.25, 2))
        assert abs(oracle.l2p(bc, z - cc) - oracle.l2p(b, z - cp)) < 1e-13 * max(1.0, abs(oracle.l2p(b, z - cp)))


def test_m2l_converges_geometrically(oracle):
    """The local expansion of a well-separated multipole converges to the multipole's value; the error of the
    truncated M2L decays at least like (sqrt(2)/(4 - sqrt(2)))^p for boxes one box apart."""
    rs = np.random.default_rng(4)
    w = 1.0
    xs, ys = rs.uniform(-w / 2, w / 2, 25), rs.uniform(-w / 2, w / 2, 25)
    q = rs.normal(size=25) + 1j * rs.normal(size=25)
    cS, cT = 0j, 2.0 + 0j  # adjacent-but-one boxes of side 1
    targets = cT + rs.uniform(-w / 2, w / 2, 10) + 1j * rs.uniform(-w / 2, w / 2, 10)
    exact = np.array([np.sum(q / (z - (xs + 1j * ys))) for z in targets])
    prev = None
    for p in (5, 10, 15, 20, 25, 30):
        a = oracle.p2m(xs, ys, q, cS, p)
        b = oracle.m2l(a, cS - cT)
        approx = np.array([oracle.l2p(b, z - cT) for z in targets])
        err = np.max(np.abs(approx - exact)) / np.max(np.abs(exact))
        bound = 40 * (math.sqrt(2) / (4 - math.sqrt(2))) ** p
        assert err < bound
        if prev is not None:
            assert err < prev
        prev = err
    assert prev < 1e-8


# ---------------------------------------------------------------------------------------- the FMM


def test_fmm_converges_to_split_direct_sum(oracle):
    """As p grows the FMM converges geometrically to the near-K_sigma / far-point-vortex sum (§2 end)."""
    w = fi.uniform(2500, seed_index=23, depth=3)
    ue, ve = oracle.split_direct(w.x, w.y, w.gamma, w.sigma, w.depth, domain=w.domain)
    errs = []
    for p in (4, 8, 12, 16, 24, 30):
        u, v, _ = oracle.fmm(w.x, w.y, w.gamma, w.sigma, w.depth, p, domain=w.domain)
        errs.append(rel_l2((u, v), (ue, ve)))
    for k in range(1, len(errs)):
        assert errs[k] < errs[k - 1]
    assert errs[-1] < 1e-12
    for e, p in zip(errs, (4, 8, 12, 16, 24, 30)):
        assert e < 5 * (math.sqrt(2) / (4 - math.sqrt(2))) ** p


def test_fmm_shallow_tree_is_direct_sum(oracle):
    """With depth 0 or 1 every leaf pair is adjacent: the FMM is the Eq. 7 direct sum."""
    w = fi.uniform(700, seed_index=24)
    ue, ve = oracle.direct(w.x, w.y, w.gamma, w.sigma)
    for depth in (0, 1):
        u, v, npairs = oracle.fmm(w.x, w.y, w.gamma, w.sigma, depth, 8, domain=w.domain)
        assert npairs == w.n * (w.n - 1)
        assert rel_l2((u, v), (ue, ve)) < 1e-14


def test_fmm_near_far_split(oracle):
    """Stage 9 alone at depth <= 1 is the direct sum; the far part is then zero; near + far is the FMM."""
    w = fi.uniform(600, seed_index=28)
    ud, vd = oracle.direct(w.x, w.y, w.gamma, w.sigma)
    un, vn, _ = oracle.fmm(w.x, w.y, w.gamma, w.sigma, 1, 6, domain=w.domain, parts="near")
    uf, vf, _ = oracle.fmm(w.x, w.y, w.gamma, w.sigma, 1, 6, domain=w.domain, parts="far")
    assert rel_l2((un, vn), (ud, vd)) < 1e-14 and not np.any(uf) and not np.any(vf)
    un, vn, _ = oracle.fmm(w.x, w.y, w.gamma, w.sigma, 3, 9, domain=w.domain, parts="near")
    uf, vf, _ = oracle.fmm(w.x, w.y, w.gamma, w.sigma, 3, 9, domain=w.domain, parts="far")
    u, v, _ = oracle.fmm(w.x, w.y, w.gamma, w.sigma, 3, 9, domain=w.domain)
    assert np.allclose(un + uf, u, rtol=0, atol=1e-15 * np.abs(u).max())
    assert np.allclose(vn + vf, v, rtol=0, atol=1e-15 * np.abs(v).max())


def test_fmm_single_source_point_vortex(oracle):
    """One source and one distant target: the far field is the point vortex -i gamma / (2 pi (z_t - z_s))."""
    x = np.array([0.1, 0.83])
    y = np.array([0.12, 0.71])
    g = np.array([0.7, 0.0])
    u, v, _ = oracle.fmm(x, y, g, 1e-3, 3, 24, domain=(0, 0, 1))
    w = -1j * 0.7 / (2 * math.pi * ((0.83 - 0.1) + 1j * (0.71 - 0.12)))
    assert abs(u[1] - w.real) < 1e-12 * abs(w) and abs(v[1] + w.imag) < 1e-12 * abs(w)


def test_fmm_linear_impulse_is_conserved(oracle):
    """The truncated far-field operator is antisymmetric (the M2L matrix for -d is minus the transpose of the
    one for d), so sum gamma_i u_i = sum gamma_i v_i = 0 holds for the FMM at any p, to rounding."""
    w = fi.uniform(4000, seed_index=25, depth=3)
    for p in (3, 9):
        u, v, _ = oracle.fmm(w.x, w.y, w.gamma, w.sigma, w.depth, p, domain=w.domain)
        scale = np.sum(np.abs(w.gamma) * np.hypot(u, v))
        assert abs(np.sum(w.gamma * u)) < 1e-13 * scale
        assert abs(np.sum(w.gamma * v)) < 1e-13 * scale


def test_fmm_subset_targets_equal_full(oracle):
    w = fi.clustered(3000)
    u, v, _ = oracle.fmm(w.x, w.y, w.gamma, w.sigma, w.depth, w.p, domain=w.domain)
    t = fi.sample_targets(w.n, 100)
    us, vs, _ = oracle.fmm(w.x, w.y, w.gamma, w.sigma, w.depth, w.p, domain=w.domain, targets=t)
    assert np.allclose(us, u[t], rtol=0, atol=1e-15 * np.max(np.abs(u)))
    assert np.allclose(vs, v[t], rtol=0, atol=1e-15 * np.max(np.abs(v)))


def test_fmm_lattice_against_direct_sum(oracle):
    """Lattice workload (depth 4, p = 12): the FMM differs from Eq. 7 by truncation plus the Gaussian tail of
    the far pairs (closest far pair r = w + h = 4.5 sigma, tail factor exp(-10.1))."""
    w = fi.lattice_lamb_oseen()
    u, v, _ = oracle.fmm(w.x, w.y, w.gamma, w.sigma, w.depth, w.p, domain=w.domain)
    ud, vd = oracle.direct(w.x, w.y, w.gamma, w.sigma)
    us, vs = oracle.split_direct(w.x, w.y, w.gamma, w.sigma, w.depth, domain=w.domain)
    e_fmm_split = rel_l2((u, v), (us, vs))
    e_split_direct = rel_l2((us, vs), (ud, vd))
    assert e_fmm_split < 1e-6
    assert 1e-8 < e_split_direct < 1e-4
    assert rel_l2((u, v), (ud, vd)) < 1e-4


def test_far_tail_closes_the_gap_to_eq7(oracle):
    """The regularised far-field correction (§2, last paragraph): the split sum plus (K_sigma - K_point) over the
    pairs whose leaves are two leaves apart is Eq. 7 up to the tail of the pairs at least two leaf widths apart,
    exp(-(2 w)^2 / 2 sigma^2) = exp(-32) on the lattice (w = 4 sigma); without it the gap is the exp(-10) tail of
    the nearest far pairs. With no rings the correction is zero, and a wrong sign, a missing or doubled ring would
    leave a gap of the size of the uncorrected one."""
    w = fi.lattice_lamb_oseen()
    ud, vd = oracle.direct(w.x, w.y, w.gamma, w.sigma)
    us, vs = oracle.split_direct(w.x, w.y, w.gamma, w.sigma, w.depth, domain=w.domain)
    ut, vt = oracle.far_tail(w.x, w.y, w.gamma, w.sigma, w.depth, 1, domain=w.domain)
    gap = rel_l2((us, vs), (ud, vd))
    assert gap > 1e-8
    assert rel_l2((us + ut, vs + vt), (ud, vd)) < 1e-12
    u0, v0 = oracle.far_tail(w.x, w.y, w.gamma, w.sigma, w.depth, 0, domain=w.domain)
    assert not np.any(u0) and not np.any(v0)
    # two rings add only the exp(-32) pairs: the same sum to 1e-12
    u2, v2 = oracle.far_tail(w.x, w.y, w.gamma, w.sigma, w.depth, 2, domain=w.domain)
    assert rel_l2((us + u2, vs + v2), (ud, vd)) < 1e-12
    assert rel_l2((u2, v2), (ut, vt)) < 1e-6


def test_fmm_empty_and_outside(oracle):
    u, v, npairs = oracle.fmm(np.zeros(0), np.zeros(0), np.zeros(0), 0.1, 3, 5, domain=(0, 0, 1))
    assert u.size == 0 and npairs == 0
    with pytest.raises(ValueError):
        oracle.fmm(np.array([0.5, 1.5]), np.array([0.5, 0.5]), np.ones(2), 0.1, 3, 5, domain=(0, 0, 1))


# ---------------------------------------------------------------------------------------- the adjoint


def test_adjoint_matches_finite_differences(oracle):
    """Gradient of L = sum(gu u + gv v) against central differences of the oracle FMM (explicit domain so
    the tree does not move; small steps keep every particle in its leaf)."""
    w = fi.uniform(300, seed_index=26, depth=3, p=10)
    rs = np.random.default_rng(5)
    gu, gv = rs.normal(size=w.n), rs.normal(size=w.n)

    def loss(x, y, g):
        u, v, _ = oracle.fmm(x, y, g, w.sigma, w.depth, w.p, domain=w.domain)
        return float(np.sum(gu * u + gv * v))

    dg, dx, dy = oracle.fmm_adjoint(w.x, w.y, w.gamma, w.sigma, w.depth, w.p, gu, gv, domain=w.domain)
    for j in rs.choice(w.n, 8, replace=False):
        h = 1e-6 / w.n
        gp, gm = w.gamma.copy(), w.gamma.copy()
        gp[j] += h
        gm[j] -= h
        fd = (loss(w.x, w.y, gp) - loss(w.x, w.y, gm)) / (2 * h)
        assert abs(fd - dg[j]) < 1e-6 * max(1.0, abs(dg[j]))
        h = 1e-7
        xp, xm = w.x.copy(), w.x.copy()
        xp[j] += h
        xm[j] -= h
        fd = (loss(xp, w.y, w.gamma) - loss(xm, w.y, w.gamma)) / (2 * h)
        assert abs(fd - dx[j]) < 1e-5 * max(1e-3, abs(dx[j]))
        yp, ym = w.y.copy(), w.y.copy()
        yp[j] += h
        ym[j] -= h
        fd = (loss(w.x, yp, w.gamma) - loss(w.x, ym, w.gamma)) / (2 * h)
        assert abs(fd - dy[j]) < 1e-5 * max(1e-3, abs(dy[j]))


def test_adjoint_direct_limit_matches_autograd(oracle):
    """Depth 1 (all near field): the adjoint equals autograd through a torch FP64 Eq. 7 sum."""
    torch = pytest.importorskip("torch")
    w = fi.uniform(200, seed_index=27)
    rs = np.random.default_rng(6)
    gu, gv = rs.normal(size=w.n), rs.normal(size=w.n)
    x = torch.tensor(w.x, requires_grad=True)
    y = torch.tensor(w.y, requires_grad=True)
    g = torch.tensor(w.gamma, requires_grad=True)
    a = x[:, None] - x[None, :]
    b = y[:, None] - y[None, :]
    eye = torch.eye(w.n, dtype=torch.bool)
    r2 = torch.where(eye, torch.ones_like(a), a * a + b * b)
    f = torch.where(eye, torch.zeros_like(a), -torch.expm1(-r2 / (2 * w.sigma**2)) / (2 * math.pi * r2))
    u = torch.sum(g[None, :] * (-b) * f, dim=1)
    v = torch.sum(g[None, :] * a * f, dim=1)
    L = torch.sum(torch.tensor(gu) * u + torch.tensor(gv) * v)
    L.backward()
    dg, dx, dy = oracle.fmm_adjoint(w.x, w.y, w.gamma, w.sigma, 1, 8, gu, gv, domain=w.domain)
    for got, ref in ((dg, g.grad), (dx, x.grad), (dy, y.grad)):
        ref = ref.numpy()
        assert np.max(np.abs(got - ref)) < 1e-10 * np.max(np.abs(ref))


# ---------------------------------------------------------------------------------------- Eq. 3 (advection)


def _exact_pair_rotation(x, y, g, T):
    """Two point vortices rotate rigidly about their centre of vorticity at Omega = (g1 + g2) / (2 pi d^2)."""
    d2 = (x[1] - x[0]) ** 2 + (y[1] - y[0]) ** 2
    om = (g[0] + g[1]) / (2 * math.pi * d2)
    cx, cy = np.dot(g, x) / g.sum(), np.dot(g, y) / g.sum()
    c, s = math.cos(om * T), math.sin(om * T)
    return cx + c * (x - cx) - s * (y - cy), cy + s * (x - cx) + c * (y - cy)


def test_advect_two_vortices_closed_form_and_order(oracle):
    """Blobs far apart (d = 100 sigma: Gaussian factor e^-5000) move as point vortices; RK errors fall by 4
    (order 2) and 16 (order 4) when dt halves, and RK4 reaches the closed form."""
    x, y, g = np.array([0.0, 1.0]), np.array([0.0, 0.0]), np.array([1.0, 0.5])
    T = 0.5 * 2 * math.pi / (g.sum())  # half a radian
    ex, ey = _exact_pair_rotation(x, y, g, T)
    for order, ratio in ((2, 4.0), (4, 16.0)):
        errs = []
        for nst in (10, 20, 40):
            xs, ys = oracle.advect(x, y, g, 0.01, 0, 1, T / nst, nst, order=order, velocity="direct")
            errs.append(np.hypot(xs - ex, ys - ey).max())
        assert errs[0] / errs[1] == pytest.approx(ratio, rel=0.1) and errs[1] / errs[2] == pytest.approx(ratio, rel=0.1)
        if order == 4:
            assert errs[2] < 1e-9


def test_advect_lamb_oseen_lattice_rotates_rigidly(oracle):
    """The blob lattice of a Lamb-Oseen vortex (R12) keeps its axisymmetric field while it moves: every particle
    turns on its circle at u_theta(r)/r of the Lamb-Oseen closed form with r_c'^2 = r_c^2 + 2 sigma^2."""
    n1, rc = 64, 0.2
    h = 2.0 / n1
    sigma = 2 * h
    g1 = -1 + (np.arange(n1) + 0.5) * h
    X, Y = np.meshgrid(g1, g1)
    x, y = X.ravel(), Y.ravel()
    r2 = x * x + y * y
    gam = h * h * np.exp(-r2 / (rc * rc)) / (math.pi * rc * rc)
    r = np.sqrt(r2)
    om = (1 - np.exp(-r2 / (rc * rc + 2 * sigma * sigma))) / (2 * math.pi * r2)
    T = 0.02
    ex, ey = np.cos(om * T) * x - np.sin(om * T) * y, np.sin(om * T) * x + np.cos(om * T) * y
    xs, ys = oracle.advect(x, y, gam, sigma, 0, 1, T / 8, 8, order=4, velocity="direct")
    assert np.hypot(xs - ex, ys - ey).max() < 1e-11  # displacements up to 0.009
    e2 = []
    for nst in (8, 16):
        xs, ys = oracle.advect(x, y, gam, sigma, 0, 1, T / nst, nst, order=2, velocity="direct")
        e2.append(np.hypot(xs - ex, ys - ey).max())
    assert e2[0] / e2[1] == pytest.approx(4.0, rel=0.1)


def test_advect_fmm_conserves_linear_impulse(oracle):
    """The truncated FMM operator is antisymmetric, so sum gamma_i u_i = 0 at every stage and every Runge-Kutta
    step keeps sum gamma_i z_i to rounding."""
    w = fi.uniform(3000, seed_index=81, depth=3, p=12)
    g = w.gamma
    for order in (2, 4):
        xs, ys = oracle.advect(w.x, w.y, g, w.sigma, w.depth, w.p, 2e-3, 3, order=order, domain=None)
        scale = np.abs(g).sum()
        assert abs(np.dot(g, xs) - np.dot(g, w.x)) < 1e-15 * scale
        assert abs(np.dot(g, ys) - np.dot(g, w.y)) < 1e-15 * scale
        assert np.hypot(xs - w.x, ys - w.y).max() > 1e-9  # the particles did move
