"""The allocation-free entry point fmm_velocity_noalloc, called through the C ABI, against fmm_velocity.

Callers that cannot let a library allocate device memory (code under another framework's allocator, inside
an allocation-free region, on a fixed budget) use this entry point; its scratch is a fixed device array.
Two calls in a row must both agree with the handle-based entry point (they share the array, so the second
call also checks that the first left nothing behind that changes the result). This file is named so that
pytest collects it last.
"""
import ctypes

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
    from paper_1008_2410_gb300 import _lib, build

    build.build()
    return _lib.load()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
@pytest.mark.parametrize("explicit_domain", [True, False])
def test_noalloc_matches_velocity_twice(lib, precision, tol, explicit_domain):
    from paper_1008_2410_gb300 import api

    w = fi.uniform(20000, seed_index=71, depth=5, p=14)
    x, y, g = dev(w.x), dev(w.y), dev(w.gamma)
    f = api.FMM(w.depth, w.p, w.sigma, precision=precision, domain=w.domain if explicit_domain else None)
    ur, vr = f.velocity(x, y, g)
    f.sync()
    ref = (ur.cpu().numpy(), vr.cpu().numpy())
    mode = 0 if precision == "fp64" else 1
    dom = (ctypes.c_double * 3)(*w.domain) if explicit_domain else None
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        u = torch.full_like(x, float("nan"))
        v = torch.full_like(x, float("nan"))
        st = lib.fmm_velocity_noalloc(w.depth, w.p, w.sigma, mode, dom, w.n, x.data_ptr(), y.data_ptr(),
                                      g.data_ptr(), u.data_ptr(), v.data_ptr(), stream)
        assert st == 0, lib.fmm_status_string(st)
        assert rel_l2((u.cpu().numpy(), v.cpu().numpy()), ref) < tol


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    x = torch.zeros(10, dtype=torch.float64, device="cuda")
    # depth 9 needs far more than the fixed scratch: refused before any device work
    st = lib.fmm_velocity_noalloc(9, 20, 0.01, 1, None, 10, x.data_ptr(), x.data_ptr(), x.data_ptr(),
                                  x.data_ptr(), x.data_ptr(), None)
    assert st == 1
