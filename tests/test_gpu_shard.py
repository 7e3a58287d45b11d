"""The sharded evaluation (paper §3-§4: parts own level-k subtrees, the root tree comes from the summed level-k
multipoles, one layer of neighbouring boxes is exchanged) through the CUDA library: P = 2 and 4 parts run as
threads of one process on one GPU, each with its own handle (they meet only on the host, after synchronising
their work). The assembled velocities must equal the single-handle evaluation and the oracle FMM: FP64 form to
1e-12 relative L2, precision form to 1e-6."""
import threading

import numpy as np
import pytest

import fmm_inputs as fi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def run_parts(lib, w, parts, level, precision):
    from paper_1008_2410_gb300 import shard

    hub = shard.ThreadComm(parts)
    n = w.n
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    x, y, g = dev(w.x), dev(w.y), dev(w.gamma)
    idx = torch.arange(n, dtype=torch.int64, device="cuda")
    out, err = [None] * parts, []

    def part(r):
        try:
            f = lib.FMM(w.depth, w.p, w.sigma, precision=precision, domain=w.domain)
            sl = slice(r * n // parts, (r + 1) * n // parts)
            out[r] = shard.velocity_sharded(f, hub.for_rank(r), x[sl], y[sl], g[sl], idx[sl], w.domain, level)
            f.sync()
        except Exception as e:  # noqa: BLE001 - re-raised below
            err.append(e)
            hub._bar.abort()

    th = [threading.Thread(target=part, args=(r,)) for r in range(parts)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    if err:
        raise err[0]
    u = np.full(n, np.nan)
    v = np.full(n, np.nan)
    for o in out:
        i = o["index"].cpu().numpy()
        u[i] = o["u"].cpu().numpy()
        v[i] = o["v"].cpu().numpy()
    return u, v, [(o["own"], o["halo"]) for o in out]


CASES = [
    ("uniform40k_d5_p14_k2", lambda: fi.uniform(40000, seed_index=120, depth=5, p=14), 2),
    ("uniform40k_d5_p14_k3", lambda: fi.uniform(40000, seed_index=120, depth=5, p=14), 3),
    ("clustered30k_d5_p12_k3", lambda: fi.clustered(30000, seed_index=121, depth=5, p=12), 3),
]


@pytest.mark.parametrize("parts", [2, 4])
@pytest.mark.parametrize("name,make,level", CASES, ids=[c[0] for c in CASES])
def test_sharded_matches_single_handle_and_oracle(lib, oracle, parts, name, make, level):
    w = make()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    uo, vo, _ = oracle.fmm(w.x, w.y, w.gamma, w.sigma, w.depth, w.p, domain=w.domain)
    for precision, tol in (("fp64", 1e-12), ("mixed", 1e-6)):
        u, v, split = run_parts(lib, w, parts, level, precision)
        assert not np.isnan(u).any() and not np.isnan(v).any()
        assert sum(s[0] for s in split) == w.n
        f = lib.FMM(w.depth, w.p, w.sigma, precision=precision, domain=w.domain)
        us, vs = f.velocity(dev(w.x), dev(w.y), dev(w.gamma))
        f.sync()
        assert rel_l2((u, v), (us.cpu().numpy(), vs.cpu().numpy())) < tol, (precision, "vs single handle")
        assert rel_l2((u, v), (uo, vo)) < tol, (precision, "vs oracle")


def test_level_calls_reject_what_they_cannot_serve(lib):
    from paper_1008_2410_gb300 import _lib

    w = fi.uniform(2000, seed_index=122, depth=4, p=8)
    x = torch.from_numpy(w.x).cuda()
    f = lib.FMM(w.depth, w.p, w.sigma)  # no explicit root square
    with pytest.raises(_lib.FMMError):
        f.level_multipoles(x, x, x, 2)
    f.set_domain(*w.domain)
    for bad in (1, 5):
        with pytest.raises(_lib.FMMError):
            f.level_multipoles(x, x, x, bad)
    M, cnt = f.level_multipoles(x, x, x, 2)
    f.sync()
    assert int(cnt.sum()) == w.n and M.shape == (16, w.p, 2)
