"""Host-only checks: the paper's model numbers (Table 1, §4) and the C ABI library's exports."""
import ctypes
import json
import math
import os

import numpy as np
import pytest

import fmm_inputs as fi

from paper_1008_2410_gb300 import model

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


def test_table1_b_opt_and_overlap_numbers():
    t = GOLD["table1_t"]["value"]
    assert round(model.b_opt(t)) == GOLD["B_opt_this_paper"]["value"]        # §4: approx 18
    assert abs(model.overlap_ratio(t) - GOLD["b_over_d"]["value"]) < 0.005   # §4: 215.22
    ex = GOLD["worked_example"]
    assert abs(model.min_leaf_occupancy_for_overlap(t, ex["N"], ex["P"]) - ex["B_min"]) < 0.005  # 14.30
    ms = GOLD["memory_scalable"]
    assert round(model.overlap_ratio(t) / ms["B"]) == ms["M_coeff"]          # M >= 12 log4 P
    mc = GOLD["million_cores"]
    assert abs(ms["M_coeff"] * math.log(mc["P_min"], 4) - mc["M_max_approx"]) < 1.0  # ~120 per core
    # §4 prints B_opt ~ 30 for Greengard-Gropp's c = 25 s^2, d = 9, s = 15, but sqrt(c/d) of those inputs is 25:
    # the printed value does not follow from the printed inputs (a discrepancy in the paper, kept as is).
    gg = GOLD["B_opt_greengard_gropp"]
    s = gg["inputs"]["s"]
    assert math.sqrt(gg["inputs"]["c_over_s2"] * s * s / gg["inputs"]["d"]) == 25.0
    assert gg["value"] == 30


def test_table1_coefficients_match_section3_sums():
    """d = 198 = 9 * 22 (§3); a = a1 + a2 + a3 + a4 = (8t+3) + (8t+2) + 2 - 22 (§3)."""
    for t in (5, 12, 15, 20):
        k = model.coefficients(t)
        assert k["d"] == GOLD["d_coefficient_times_r"]["value"] == 9 * GOLD["p2p_flops_per_pair"]["value"]
        assert k["a"] == (8 * t + 3) + (8 * t + 2) + 2 - 22


def test_near_pair_formula_lattice_value():
    assert model.near_pairs_uniform(64, 4) == 8650752


def test_library_exports_every_declared_symbol():
    from paper_1008_2410_gb300 import _lib, build

    path = build.build()
    lib = ctypes.CDLL(path)
    names = _lib.header_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(names) == set(_lib.SIGNATURES), set(names) ^ set(_lib.SIGNATURES)


def test_product_path_has_no_fallback():
    """The package never imports the oracle, and loading fails loudly without the built library."""
    import paper_1008_2410_gb300 as pkg

    root = os.path.dirname(pkg.__file__)
    for dirpath, _, files in os.walk(root):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text and "fmm_oracle" not in text


def test_suggest_depth_rule():
    """Occupancy depth round(log4(n / 64)), reduced until exp(-w^2 / 2 sigma^2) <= tail_tol for leaf width w."""
    from paper_1008_2410_gb300 import api

    n = 1 << 20
    assert api.suggest_depth(n, 0.5 / 1024, 1.0) == 7  # uniform_1m: w / sigma = 16, tail e^-128
    # the Lamb-Oseen lattice (sigma = 2h, square side 2): depth 4 leaves are 4 sigma wide (tail e^-8 = 3.4e-4)
    assert api.suggest_depth(128 * 128, 2 * 2 / 128, 2.0, tail_tol=1e-12) == 3
    assert api.suggest_depth(128 * 128, 2 * 2 / 128, 2.0, tail_tol=1e-3) == 4
    assert api.suggest_depth(100, 1.0, 1.0) == 0
    assert api.suggest_depth(1 << 30, 1e-9, 1.0) == 12
    for bad in ((0, 1.0, 1.0), (10, 0.0, 1.0), (10, 1.0, -1.0)):
        with pytest.raises(ValueError):
            api.suggest_depth(*bad)
    with pytest.raises(ValueError):
        api.suggest_depth(10, 1.0, 1.0, tail_tol=1.5)


def test_suggested_depth_removes_the_far_field_tail(oracle):
    """§2: the expansions carry the point-vortex kernel, so the FMM converges (in p) to the split sum, which
    misses the Gaussian tail of pairs beyond adjacent leaves. On the Lamb-Oseen lattice at depth 4 (leaves
    4 sigma wide) that tail caps the agreement with Eq. 7 near 1e-7; at the suggested depth 3 (8 sigma) the FMM at
    p = 30 reaches 1e-14."""
    from paper_1008_2410_gb300 import api

    w = fi.lattice_lamb_oseen()
    d = api.suggest_depth(w.n, w.sigma, w.domain[2], tail_tol=1e-12)
    assert d == 3
    t = fi.sample_targets(w.n, 256)
    ud, vd = oracle.direct(w.x, w.y, w.gamma, w.sigma, targets=t)
    errs = {}
    for depth in (4, d):
        u, v, _ = oracle.fmm(w.x, w.y, w.gamma, w.sigma, depth, 30, domain=w.domain, targets=t)
        errs[depth] = float(np.linalg.norm(np.concatenate([u - ud, v - vd])) / np.linalg.norm(np.concatenate([ud, vd])))
    assert errs[4] > 1e-7  # tail-limited: 1.34e-7 whatever p (measured at p = 20 and 30)
    assert errs[d] < 1e-12


def test_default_m2l_engine_is_the_cuda_core_kernel():
    """Until the tensor-core M2L wins at the measured configurations, a handle that is not autotuned runs the FP32
    M2L levels on the CUDA cores: the header documents it and the handle's initialiser sets it."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    hdr = open(os.path.join(root, "include", "fmm2d.h")).read()
    assert "FMM_M2L_CUDA_CORES (default)" in hdr and "FMM_M2L_TENSOR (default)" not in hdr
    src = open(os.path.join(root, "paper_1008_2410_gb300", "csrc", "capi.cu")).read()
    assert "int m2l_engine = FMM_M2L_CUDA_CORES;" in src
    na = open(os.path.join(root, "paper_1008_2410_gb300", "csrc", "noalloc.cu")).read()
    assert "w.m2l_tc = 0;" in na
