"""FP64 CPU oracle for the 2D vortex-blob FMM velocity evaluation -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its ``cpu_baseline`` leg and the
``--impl reference`` arm) may import this package. It shares no code with the CUDA library in
``paper_1008_2410_gb300`` and never imports it.

The arithmetic lives in ``fmm_oracle.c`` (plain C99, ``double complex``, no FMA contraction); this module
compiles it with gcc and exposes thin numpy wrappers. Every function follows the paper (M. G. Knepley,
"Removing the Barrier to Scalability in Parallel FMM"):

* ``kernel``          -- Eq. 6, the Gaussian-regularised Biot-Savart kernel K_sigma
* ``direct``          -- Eq. 7, the O(N^2) velocity sum (optionally at a subset of targets)
* ``split_direct``    -- the sum the FMM converges to (§2, last paragraph): K_sigma for particles in equal or
                         adjacent leaves, the point-vortex kernel for all other pairs
* ``far_tail``        -- the regularised far-field correction: (K_sigma - K_point) over the pairs whose leaves are
                         2 .. 1 + rings leaves apart
* ``fmm``             -- the serial FMM of Fig. 1, stages 1-10, with the §3 multipole coefficients
* ``fmm_adjoint``     -- gradient of sum(gu*u + gv*v) by the transposed stages in reverse order
* ``advect``          -- Eq. 3: particles moved with the FMM or direct-sum velocity, Runge-Kutta order 2 or 4
* ``p2m, m2m, m2l, l2l, l2p, multipole_eval`` -- the single-box expansion operations used by ``fmm``

Pins (tests marked ``not gpu``): brute force on tiny inputs, the Lamb-Oseen closed form, impulse invariants,
geometric decay of the FMM error in p towards ``split_direct``, exactness of M2M/L2L, the §3 near-field pair
count and interaction-list sizes, and finite differences for the adjoint.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fmm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)
_I32 = ctypes.POINTER(ctypes.c_int32)


def build(force: bool = False) -> str:
    """Compile ``fmm_oracle.c`` into ``oracle/_build/liboracle.so`` (gcc, -O2, OpenMP, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.oracle_kernel.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, _D, _D]
        lib.oracle_direct.argtypes = [ctypes.c_int64, _D, _D, _D, ctypes.c_double, ctypes.c_int64, _I64, _D, _D]
        lib.oracle_default_domain.argtypes = [ctypes.c_int64, _D, _D, _D]
        lib.oracle_leaf_coords.argtypes = [ctypes.c_int64, _D, _D, ctypes.c_int, _D, ctypes.c_int, _I32, _I32]
        lib.oracle_p2m.argtypes = [ctypes.c_int64, _D, _D, _D, _D, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_int, _D]
        lib.oracle_multipole_eval.argtypes = [ctypes.c_int, _D, ctypes.c_double, ctypes.c_double, _D]
        for name in ("oracle_m2m", "oracle_m2l", "oracle_l2l"):
            getattr(lib, name).argtypes = [ctypes.c_int, _D, ctypes.c_double, ctypes.c_double, _D]
        lib.oracle_l2p.argtypes = [ctypes.c_int, _D, ctypes.c_double, ctypes.c_double, _D]
        lib.oracle_interaction_list_sizes.argtypes = [ctypes.c_int, _I32]
        lib.oracle_fmm.argtypes = [ctypes.c_int64, _D, _D, _D, ctypes.c_double, ctypes.c_int, ctypes.c_int, _D,
                                   ctypes.c_int64, _I64, _D, _D, _I64]
        lib.oracle_fmm.restype = ctypes.c_int
        lib.oracle_fmm_parts.argtypes = lib.oracle_fmm.argtypes + [ctypes.c_int]
        lib.oracle_fmm_parts.restype = ctypes.c_int
        lib.oracle_split_direct.argtypes = [ctypes.c_int64, _D, _D, _D, ctypes.c_double, ctypes.c_int, _D,
                                            ctypes.c_int64, _I64, _D, _D]
        lib.oracle_split_direct.restype = ctypes.c_int
        lib.oracle_far_tail.argtypes = [ctypes.c_int64, _D, _D, _D, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                        _D, ctypes.c_int64, _I64, _D, _D]
        lib.oracle_far_tail.restype = ctypes.c_int
        lib.oracle_fmm_adjoint.argtypes = [ctypes.c_int64, _D, _D, _D, ctypes.c_double, ctypes.c_int,
                                           ctypes.c_int, _D, _D, _D, _D, _D, _D]
        lib.oracle_fmm_adjoint.restype = ctypes.c_int
        lib.oracle_advect.argtypes = [ctypes.c_int64, _D, _D, _D, ctypes.c_double, ctypes.c_int, ctypes.c_int, _D,
                                      ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.oracle_advect.restype = ctypes.c_int
        lib.oracle_p2l.argtypes = [ctypes.c_int64, _D, _D, _D, _D, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_int, _D]
        lib.oracle_adaptive_lists_check.argtypes = [ctypes.c_int64, _D, _D, ctypes.c_int, ctypes.c_int, _D, _I64]
        lib.oracle_adaptive_lists_check.restype = ctypes.c_int
        lib.oracle_adaptive_fmm.argtypes = [ctypes.c_int64, _D, _D, _D, ctypes.c_double, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_int, _D, _D, _D, ctypes.c_int]
        lib.oracle_adaptive_fmm.restype = ctypes.c_int
        lib.oracle_adaptive_split_direct.argtypes = [ctypes.c_int64, _D, _D, _D, ctypes.c_double, ctypes.c_int,
                                                     ctypes.c_int, _D, _D, _D]
        lib.oracle_adaptive_split_direct.restype = ctypes.c_int
        _lib = lib
        return lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray | None, t=_D):
    return None if a is None else a.ctypes.data_as(t)


def _targets(n: int, targets):
    if targets is None:
        return n, None
    t = np.ascontiguousarray(np.asarray(targets, dtype=np.int64))
    if t.size and (t.min() < 0 or t.max() >= n):
        raise ValueError("target index out of range")
    return int(t.size), t


def _dom(domain):
    return None if domain is None else _f64(domain).reshape(3)


def kernel(a: float, b: float, sigma: float) -> tuple[float, float]:
    """Eq. 6 at displacement (a, b): returns (K_u, K_v); zero displacement gives (0, 0)."""
    ku, kv = ctypes.c_double(), ctypes.c_double()
    _load().oracle_kernel(float(a), float(b), float(sigma), ctypes.byref(ku), ctypes.byref(kv))
    return ku.value, kv.value


def direct(x, y, gamma, sigma: float, targets=None):
    """Eq. 7 direct sum (self excluded). Returns (u, v) at ``targets`` (all particles if None)."""
    x, y, g = _f64(x), _f64(y), _f64(gamma)
    n = x.size
    nt, t = _targets(n, targets)
    u, v = np.zeros(nt), np.zeros(nt)
    _load().oracle_direct(n, _ptr(x), _ptr(y), _ptr(g), float(sigma), nt, _ptr(t, _I64), _ptr(u), _ptr(v))
    return u, v


def default_domain(x, y) -> np.ndarray:
    """Root square {x0, y0, S} of the bounding-box rule (centre of the box, side = extent*(1+2^-20))."""
    x, y = _f64(x), _f64(y)
    out = np.zeros(3)
    _load().oracle_default_domain(x.size, _ptr(x), _ptr(y), _ptr(out))
    return out


def leaf_coords(x, y, depth: int, domain=None, check: bool = True):
    """Leaf column/row of each particle at ``depth`` (floor rule, clamped). Raises on points outside an
    explicit square when ``check``."""
    x, y = _f64(x), _f64(y)
    d = default_domain(x, y) if domain is None else _dom(domain)
    ix, iy = np.zeros(x.size, np.int32), np.zeros(x.size, np.int32)
    rc = _load().oracle_leaf_coords(x.size, _ptr(x), _ptr(y), int(depth), _ptr(d), int(bool(check)),
                                    _ptr(ix, _I32), _ptr(iy, _I32))
    if rc != 0:
        raise ValueError("point outside the root square")
    return ix, iy


def p2m(x, y, q, centre, p: int) -> np.ndarray:
    """§3 multipole coefficients sum_j q_j (z_j - c)^m, m < p, for complex charges q."""
    x, y = _f64(x), _f64(y)
    q = np.asarray(q, dtype=np.complex128)
    qre, qim = _f64(q.real), _f64(q.imag)
    a = np.zeros(2 * p)
    _load().oracle_p2m(x.size, _ptr(x), _ptr(y), _ptr(qre), _ptr(qim), float(centre.real), float(centre.imag),
                       int(p), _ptr(a))
    return a.view(np.complex128)


def _cvec(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128)).view(np.float64)


def multipole_eval(a, dz: complex) -> complex:
    """sum_m a_m / dz^(m+1)."""
    a = _cvec(a)
    w = np.zeros(2)
    _load().oracle_multipole_eval(a.size // 2, _ptr(a), float(dz.real), float(dz.imag), _ptr(w))
    return complex(w[0], w[1])


def _translate(name: str, a, d: complex) -> np.ndarray:
    a = _cvec(a)
    out = np.zeros_like(a)
    getattr(_load(), name)(a.size // 2, _ptr(a), float(d.real), float(d.imag), _ptr(out))
    return out.view(np.complex128)


def m2m(a, d: complex) -> np.ndarray:
    """Stage 5: multipole about the parent from one about the child, d = c_child - c_parent."""
    return _translate("oracle_m2m", a, d)


def m2l(a, d: complex) -> np.ndarray:
    """Stage 6: local expansion about c_T from a multipole about c_S, d = c_S - c_T."""
    return _translate("oracle_m2l", a, d)


def l2l(b, d: complex) -> np.ndarray:
    """Stage 7: local expansion about the child from one about the parent, d = c_child - c_parent."""
    return _translate("oracle_l2l", b, d)


def l2p(b, dz: complex) -> complex:
    """Stage 8: sum_l b_l dz^l."""
    b = _cvec(b)
    w = np.zeros(2)
    _load().oracle_l2p(b.size // 2, _ptr(b), float(dz.real), float(dz.imag), _ptr(w))
    return complex(w[0], w[1])


def interaction_list_sizes(level: int) -> np.ndarray:
    """Stage 3: interaction-list size of each box at ``level`` (row-major 2^l x 2^l)."""
    out = np.zeros(1 << (2 * level), np.int32)
    _load().oracle_interaction_list_sizes(int(level), _ptr(out, _I32))
    return out.reshape(1 << level, 1 << level)


def fmm(x, y, gamma, sigma: float, depth: int, p: int, domain=None, targets=None, parts: str = "both"):
    """Serial FMM (Fig. 1). Returns (u, v, near_pairs) at ``targets`` (all particles if None).
    parts = "near" (stage 9 only), "far" (stages 4-8 only) or "both"."""
    x, y, g = _f64(x), _f64(y), _f64(gamma)
    n = x.size
    nt, t = _targets(n, targets)
    u, v = np.zeros(nt), np.zeros(nt)
    npairs = ctypes.c_int64(0)
    code = {"near": 1, "far": 2, "both": 3}[parts]
    rc = _load().oracle_fmm_parts(n, _ptr(x), _ptr(y), _ptr(g), float(sigma), int(depth), int(p),
                                  _ptr(_dom(domain)), nt, _ptr(t, _I64), _ptr(u), _ptr(v), ctypes.byref(npairs), code)
    if rc == -1:
        raise ValueError("point outside the root square")
    if rc != 0:
        raise MemoryError("oracle_fmm failed")
    return u, v, npairs.value


def far_tail(x, y, gamma, sigma: float, depth: int, rings: int, domain=None, targets=None):
    """Regularised far-field correction: (K_sigma - K_point) summed over the pairs whose leaves are 2 .. 1 + rings
    leaves apart (Chebyshev distance). Returns (u, v) at ``targets`` (all particles if None)."""
    x, y, g = _f64(x), _f64(y), _f64(gamma)
    n = x.size
    nt, t = _targets(n, targets)
    u, v = np.zeros(nt), np.zeros(nt)
    rc = _load().oracle_far_tail(n, _ptr(x), _ptr(y), _ptr(g), float(sigma), int(depth), int(rings),
                                 _ptr(_dom(domain)), nt, _ptr(t, _I64), _ptr(u), _ptr(v))
    if rc != 0:
        raise ValueError("oracle_far_tail failed")
    return u, v


def split_direct(x, y, gamma, sigma: float, depth: int, domain=None, targets=None):
    """Exact sum the FMM converges to as p grows (near pairs K_sigma, far pairs point vortex)."""
    x, y, g = _f64(x), _f64(y), _f64(gamma)
    n = x.size
    nt, t = _targets(n, targets)
    u, v = np.zeros(nt), np.zeros(nt)
    rc = _load().oracle_split_direct(n, _ptr(x), _ptr(y), _ptr(g), float(sigma), int(depth), _ptr(_dom(domain)),
                                     nt, _ptr(t, _I64), _ptr(u), _ptr(v))
    if rc != 0:
        raise ValueError("oracle_split_direct failed")
    return u, v


def fmm_adjoint(x, y, gamma, sigma: float, depth: int, p: int, gu, gv, domain=None):
    """Gradient of sum(gu*u + gv*v) for u, v = fmm(...): returns (dgamma, dx, dy)."""
    x, y, g, gu, gv = _f64(x), _f64(y), _f64(gamma), _f64(gu), _f64(gv)
    n = x.size
    dg, dx, dy = np.zeros(n), np.zeros(n), np.zeros(n)
    rc = _load().oracle_fmm_adjoint(n, _ptr(x), _ptr(y), _ptr(g), float(sigma), int(depth), int(p),
                                    _ptr(_dom(domain)), _ptr(gu), _ptr(gv), _ptr(dg), _ptr(dx), _ptr(dy))
    if rc != 0:
        raise ValueError("oracle_fmm_adjoint failed")
    return dg, dx, dy


def advect(x, y, gamma, sigma: float, depth: int, p: int, dt: float, nsteps: int, order: int = 2,
           domain=None, velocity: str = "fmm"):
    """Eq. 3: nsteps explicit Runge-Kutta steps (order 2: midpoint rule; order 4: classical) of the particles,
    each stage's velocity from the FMM (``velocity="fmm"``) or the direct sum (``"direct"``). Returns new
    (x, y); circulations are unchanged."""
    xs, ys, g = _f64(x).copy(), _f64(y).copy(), _f64(gamma)
    mode = {"fmm": 0, "direct": 1}[velocity]
    rc = _load().oracle_advect(xs.size, _ptr(xs), _ptr(ys), _ptr(g), float(sigma), int(depth), int(p),
                               _ptr(_dom(domain)), float(dt), int(nsteps), int(order), mode)
    if rc == -1:
        raise ValueError("point outside the root square")
    if rc != 0:
        raise RuntimeError(f"oracle_advect failed ({rc})")
    return xs, ys


# ---------------------------------------------------------------- adaptive quadtree (§5, uneven densities)

def p2l(x, y, q, centre, p: int) -> np.ndarray:
    """X-list operator: local expansion about ``centre`` of point charges q_j at (x_j, y_j)."""
    x, y = _f64(x), _f64(y)
    q = np.asarray(q, np.complex128)
    qre, qim = np.ascontiguousarray(q.real), np.ascontiguousarray(q.imag)
    out = np.zeros(2 * p)
    _load().oracle_p2l(x.size, _ptr(x), _ptr(y), _ptr(qre), _ptr(qim), float(np.real(centre)),
                       float(np.imag(centre)), int(p), _ptr(out))
    return out[0::2] + 1j * out[1::2]


def adaptive_lists_check(x, y, max_depth: int, leaf_capacity: int, domain=None):
    """Builds the adaptive tree and its U, V, W, X lists from their definitions. Returns (bad, sizes): bad =
    the number of ordered leaf pairs whose interaction the lists deliver other than exactly once; sizes =
    dict of boxes, leaves, total |U|, |V|, |W|, |X|, max |V|, the deepest leaf level and the ordered near
    pairs (i, j != i) of the U lists."""
    x, y = _f64(x), _f64(y)
    sizes = np.zeros(9, np.int64)
    bad = _load().oracle_adaptive_lists_check(x.size, _ptr(x), _ptr(y), int(max_depth), int(leaf_capacity),
                                              _ptr(_dom(domain)), _ptr(sizes, _I64))
    if bad < 0:
        raise ValueError("oracle_adaptive_lists_check failed")
    keys = ("boxes", "leaves", "U", "V", "W", "X", "maxV", "deepest", "near_pairs")
    return bad, dict(zip(keys, (int(s) for s in sizes)))


def adaptive_fmm(x, y, gamma, sigma: float, max_depth: int, leaf_capacity: int, p: int, domain=None,
                 parts: str = "both"):
    """Serial adaptive FMM (U, V, W, X lists). Returns (u, v) in input order."""
    x, y, g = _f64(x), _f64(y), _f64(gamma)
    u, v = np.zeros(x.size), np.zeros(x.size)
    code = {"near": 1, "far": 2, "both": 3}[parts]
    rc = _load().oracle_adaptive_fmm(x.size, _ptr(x), _ptr(y), _ptr(g), float(sigma), int(max_depth),
                                     int(leaf_capacity), int(p), _ptr(_dom(domain)), _ptr(u), _ptr(v), code)
    if rc == -1:
        raise ValueError("point outside the root square")
    if rc != 0:
        raise MemoryError("oracle_adaptive_fmm failed")
    return u, v


def adaptive_split_direct(x, y, gamma, sigma: float, max_depth: int, leaf_capacity: int, domain=None):
    """Exact sum the adaptive FMM converges to: K_sigma between particles in adjacent (or equal) leaves of the
    adaptive tree, the point-vortex kernel between all other pairs."""
    x, y, g = _f64(x), _f64(y), _f64(gamma)
    u, v = np.zeros(x.size), np.zeros(x.size)
    rc = _load().oracle_adaptive_split_direct(x.size, _ptr(x), _ptr(y), _ptr(g), float(sigma), int(max_depth),
                                              int(leaf_capacity), _ptr(_dom(domain)), _ptr(u), _ptr(v))
    if rc != 0:
        raise ValueError("oracle_adaptive_split_direct failed")
    return u, v
