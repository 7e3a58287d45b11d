"""Python face of the C ABI: an ``FMM`` handle class over torch tensors and ``FMMVelocity``, an
``autograd.Function`` whose backward is the library's hand-written adjoint.

PyTorch supplies device memory and the current stream only; each method passes raw pointers to the CUDA
library and every stage of the evaluation runs there. Device tensors must be contiguous float64 on the
handle's GPU; ``velocity_host`` takes CPU tensors (pinned or pageable) and copies inside the library.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import FMM_FP64, FMM_MIXED, check


def _dev(t: torch.Tensor, name: str) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    return t.data_ptr()


def _host(t: torch.Tensor, name: str) -> int:
    if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float64 CPU tensor")
    return t.data_ptr()


def suggest_depth(n: int, sigma: float, side: float, tail_tol: float = 1e-12, leaf_target: float = 64.0) -> int:
    """Tree depth for n particles (occupancy about leaf_target per leaf) whose leaves are wide enough that the
    Gaussian tail left out of the far field stays below tail_tol (see fmm_suggest_depth)."""
    d = _lib.load().fmm_suggest_depth(int(n), float(sigma), float(side), float(tail_tol), float(leaf_target))
    if d < 0:
        raise ValueError("n, sigma and side must be positive and 0 < tail_tol < 1")
    return d


class FMM:
    """One FMM configuration: tree depth L (4^L leaves), p expansion terms, blob core sigma.

    precision: "fp64" (plain form) or "mixed" (precision form). domain: (x0, y0, side) or None for the
    bounding-box rule. graph: capture and replay the evaluation as a CUDA graph. m2l_engine: "cuda_cores"
    (default) or "tensor" (tcgen05) for the FP32 M2L levels of the precision form. leaf_capacity: 0 for the
    uniform tree; B > 0 for the adaptive tree (depth is then its maximum depth; boxes holding more than B
    particles are split; both precision forms, FP32 expansions and near field in the precision form).
    """

    def __init__(self, depth: int, p: int, sigma: float, precision: str = "fp64", domain=None,
                 graph: bool = False, coarse_level: int | None = None, m2l_engine: str | None = None,
                 leaf_capacity: int = 0):
        self._lib = _lib.load()
        h = ctypes.c_void_p()
        st = self._lib.fmm_create(int(depth), int(p), float(sigma), ctypes.byref(h))
        if st != _lib.FMM_OK:
            raise _lib.FMMError(st, self._lib.fmm_status_string(st).decode())
        self.h = h
        self.set_precision(precision)
        if domain is not None:
            self.set_domain(*domain)
        if graph:
            self.set_graph(True)
        if coarse_level is not None:
            check(self._lib.fmm_set_coarse_level(self.h, int(coarse_level)), self.h)
        if m2l_engine is not None:
            self.set_m2l_engine(m2l_engine)
        if leaf_capacity:
            self.set_adaptive(leaf_capacity)

    # -- configuration
    def close(self) -> None:
        if getattr(self, "h", None):
            self._lib.fmm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_precision(self, precision: str) -> None:
        mode = {"fp64": FMM_FP64, "mixed": FMM_MIXED}[precision]
        check(self._lib.fmm_set_precision(self.h, mode), self.h)
        self.precision = precision

    def set_m2l_engine(self, engine: str) -> None:
        code = {"cuda_cores": 0, "tensor": 1}[engine]
        check(self._lib.fmm_set_m2l_engine(self.h, code), self.h)

    def set_adjoint_precision(self, precision: str) -> None:
        """Near-field part of the adjoint: "fp64" (default, exact to rounding) or "mixed" (FP32, ~1e-6)."""
        mode = {"fp64": FMM_FP64, "mixed": FMM_MIXED}[precision]
        check(self._lib.fmm_set_adjoint_precision(self.h, mode), self.h)
        self.adjoint_precision = precision

    def set_adaptive(self, leaf_capacity: int) -> None:
        """0: uniform tree; B > 0: adaptive tree splitting boxes with more than B particles."""
        check(self._lib.fmm_set_adaptive(self.h, int(leaf_capacity)), self.h)

    def set_domain(self, x0: float, y0: float, side: float) -> None:
        check(self._lib.fmm_set_domain(self.h, float(x0), float(y0), float(side)), self.h)

    def clear_domain(self) -> None:
        check(self._lib.fmm_clear_domain(self.h), self.h)

    def set_params(self, depth: int, p: int, sigma: float) -> None:
        check(self._lib.fmm_set_params(self.h, int(depth), int(p), float(sigma)), self.h)

    def set_graph(self, enable: bool) -> None:
        check(self._lib.fmm_set_graph(self.h, int(bool(enable))), self.h)

    def set_p2p_tile(self, threads: int, targets_per_thread: int) -> None:
        check(self._lib.fmm_set_p2p_tile(self.h, int(threads), int(targets_per_thread)), self.h)

    def set_far_tail(self, rings: int) -> None:
        """Regularised far-field correction over the leaves 2 .. 1 + rings leaves away (0: off; uniform tree)."""
        check(self._lib.fmm_set_far_tail(self.h, int(rings)), self.h)

    def set_timing(self, enable) -> None:
        """True: every stage event; "near": only the near field's two events (uniform tree; fewer graph nodes)."""
        check(self._lib.fmm_set_timing(self.h, 2 if enable == "near" else int(bool(enable))), self.h)

    def set_count_pairs(self, enable: bool) -> None:
        check(self._lib.fmm_set_count_pairs(self.h, int(bool(enable))), self.h)

    def params(self) -> dict:
        d, p, th, kt = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        s = ctypes.c_double()
        check(self._lib.fmm_get_params(self.h, ctypes.byref(d), ctypes.byref(p), ctypes.byref(s), ctypes.byref(th),
                                       ctypes.byref(kt)), self.h)
        eng = self._lib.fmm_get_m2l_engine(self.h)
        return {"depth": d.value, "p": p.value, "sigma": s.value, "p2p_threads": th.value,
                "p2p_targets_per_thread": kt.value, "m2l_engine": {0: "cuda_cores", 1: "tensor"}.get(eng, "?"),
                "leaf_capacity": self._lib.fmm_get_adaptive(self.h)}

    def _stream(self) -> None:
        s = torch.cuda.current_stream()
        check(self._lib.fmm_set_stream(self.h, ctypes.c_void_p(s.cuda_stream)), self.h)

    # -- evaluations
    def _call(self, fn, x, y, gamma, u, v):
        n = x.numel()
        if u is None:
            u = torch.empty_like(x)
        if v is None:
            v = torch.empty_like(x)
        for t, nm in ((y, "y"), (gamma, "gamma"), (u, "u"), (v, "v")):
            if t.numel() != n:
                raise ValueError(f"{nm} has {t.numel()} elements, expected {n}")
        self._stream()
        check(fn(self.h, n, _dev(x, "x"), _dev(y, "y"), _dev(gamma, "gamma"), _dev(u, "u"), _dev(v, "v")), self.h)
        return u, v

    def velocity(self, x, y, gamma, u=None, v=None):
        """(u, v) at every particle: the full FMM evaluation (Fig. 1, stages 1-10)."""
        return self._call(self._lib.fmm_velocity, x, y, gamma, u, v)

    def velocity_near(self, x, y, gamma, u=None, v=None):
        """Stage 9 alone: K_sigma over particles in the same or adjacent leaves."""
        return self._call(self._lib.fmm_velocity_near, x, y, gamma, u, v)

    def velocity_far(self, x, y, gamma, u=None, v=None):
        """Stages 4-8 alone: the expansions' point-vortex field of all non-adjacent leaves."""
        return self._call(self._lib.fmm_velocity_far, x, y, gamma, u, v)

    def advect(self, x, y, gamma, dt: float, nsteps: int, order: int = 2) -> None:
        """Eq. 3: nsteps Runge-Kutta steps (order 2 or 4) of the particles, x and y (CUDA float64) in place."""
        self._stream()
        check(self._lib.fmm_advect(self.h, x.numel(), _dev(x, "x"), _dev(y, "y"), _dev(gamma, "gamma"), float(dt),
                                   int(nsteps), int(order)), self.h)

    def velocity_host(self, x, y, gamma, u=None, v=None):
        """Same as velocity() for CPU tensors: copies in and out inside the library, synchronous."""
        n = x.numel()
        u = torch.empty_like(x) if u is None else u
        v = torch.empty_like(x) if v is None else v
        self._stream()
        check(self._lib.fmm_velocity_host(self.h, n, _host(x, "x"), _host(y, "y"), _host(gamma, "gamma"),
                                          _host(u, "u"), _host(v, "v")), self.h)
        return u, v

    def adjoint(self, x, y, gamma, gu, gv, need=(True, True, True)):
        """Gradient of sum(gu * u + gv * v) w.r.t. (gamma, x, y); entries of ``need`` that are False give None."""
        n = x.numel()
        outs = [torch.empty_like(x) if k else None for k in need]
        self._stream()
        ptr = [o.data_ptr() if o is not None else None for o in outs]
        check(self._lib.fmm_velocity_adjoint(self.h, n, _dev(x, "x"), _dev(y, "y"), _dev(gamma, "gamma"),
                                             _dev(gu, "gu"), _dev(gv, "gv"), ptr[0], ptr[1], ptr[2]), self.h)
        return tuple(outs)

    def velocity_batched(self, offsets, x, y, gamma, depths=None, sigmas=None, domains=None, u=None, v=None):
        """Independent systems in one evaluation; offsets (nsys + 1, host ints) delimit them in x, y, gamma."""
        import numpy as np

        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        nsys = off.size - 1
        dep = None if depths is None else np.ascontiguousarray(np.asarray(depths, dtype=np.int32))
        sig = None if sigmas is None else np.ascontiguousarray(np.asarray(sigmas, dtype=np.float64))
        dom = None if domains is None else np.ascontiguousarray(np.asarray(domains, dtype=np.float64).reshape(-1))
        u = torch.empty_like(x) if u is None else u
        v = torch.empty_like(x) if v is None else v
        self._stream()
        check(self._lib.fmm_velocity_batched(
            self.h, nsys, off.ctypes.data, None if dep is None else dep.ctypes.data,
            None if sig is None else sig.ctypes.data, None if dom is None else dom.ctypes.data,
            _dev(x, "x"), _dev(y, "y"), _dev(gamma, "gamma"), _dev(u, "u"), _dev(v, "v")), self.h)
        return u, v

    def autotune(self, x, y, gamma, depth_lo: int, depth_hi: int) -> dict:
        u = torch.empty_like(x)
        v = torch.empty_like(x)
        self._stream()
        check(self._lib.fmm_autotune(self.h, x.numel(), _dev(x, "x"), _dev(y, "y"), _dev(gamma, "gamma"),
                                     _dev(u, "u"), _dev(v, "v"), int(depth_lo), int(depth_hi)), self.h)
        return self.params()

    def level_multipoles(self, x, y, gamma, level: int):
        """(M, counts) of the given particles at tree level `level`: M a (4^level, p) complex128 CUDA tensor in the
        library's radius-scaled form, counts a (4^level,) int64 CUDA tensor (see fmm_level_multipoles)."""
        nb = 1 << (2 * int(level))
        p = self.params()["p"]
        M = torch.empty((nb, p, 2), dtype=torch.float64, device=x.device)
        cnt = torch.empty(nb, dtype=torch.int64, device=x.device)
        self._stream()
        check(self._lib.fmm_level_multipoles(self.h, x.numel(), _dev(x, "x"), _dev(y, "y"), _dev(gamma, "gamma"),
                                             int(level), M.data_ptr(), cnt.data_ptr()), self.h)
        return M, cnt

    def velocity_level(self, x, y, gamma, level: int, M, counts, u=None, v=None):
        """fmm_velocity with level `level`'s multipoles and counts taken from (M, counts) (fmm_velocity_level)."""
        n = x.numel()
        u = torch.empty_like(x) if u is None else u
        v = torch.empty_like(x) if v is None else v
        if not (M.is_cuda and M.dtype == torch.float64 and M.is_contiguous() and counts.is_cuda and
                counts.dtype == torch.int64 and counts.is_contiguous()):
            raise TypeError("M must be contiguous float64 and counts contiguous int64 CUDA tensors")
        self._stream()
        check(self._lib.fmm_velocity_level(self.h, n, _dev(x, "x"), _dev(y, "y"), _dev(gamma, "gamma"), int(level),
                                           M.data_ptr(), counts.data_ptr(), _dev(u, "u"), _dev(v, "v")), self.h)
        return u, v

    def autotune_batched(self, offsets, x, y, gamma, sigmas=None, domains=None) -> dict:
        """Leaf occupancy (per-system depths) and near-field tile of the fastest batched evaluation; returns the
        handle's parameters plus the chosen "depths"."""
        import numpy as np

        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        nsys = off.size - 1
        sig = None if sigmas is None else np.ascontiguousarray(np.asarray(sigmas, dtype=np.float64))
        dom = None if domains is None else np.ascontiguousarray(np.asarray(domains, dtype=np.float64).reshape(-1))
        dep = np.zeros(nsys, dtype=np.int32)
        u, v = torch.empty_like(x), torch.empty_like(x)
        self._stream()
        check(self._lib.fmm_autotune_batched(
            self.h, nsys, off.ctypes.data, None if sig is None else sig.ctypes.data,
            None if dom is None else dom.ctypes.data, _dev(x, "x"), _dev(y, "y"), _dev(gamma, "gamma"),
            _dev(u, "u"), _dev(v, "v"), dep.ctypes.data), self.h)
        prm = self.params()
        prm["depths"] = [int(d) for d in dep]
        return prm

    def autotune_p(self, x, y, gamma, rel_tol: float, p_lo: int = 1, p_hi: int = 32) -> tuple[int, float]:
        """Smallest p in [p_lo, p_hi] within rel_tol (relative L2) of the FP64 form at p = 32; sets the handle's p
        and returns (p, estimated error)."""
        err = ctypes.c_double()
        self._stream()
        check(self._lib.fmm_autotune_p(self.h, x.numel(), _dev(x, "x"), _dev(y, "y"), _dev(gamma, "gamma"),
                                       float(rel_tol), int(p_lo), int(p_hi), ctypes.byref(err)), self.h)
        return self.params()["p"], err.value

    # -- diagnostics
    def sync(self) -> None:
        check(self._lib.fmm_sync(self.h), self.h)

    def selftest_timeout(self, polls: int = 4096) -> None:
        """Runs the library's bounded device wait on a barrier nothing completes (see fmm_selftest_timeout); the
        next sync() raises FMMError with status FMM_ETIMEOUT."""
        self._stream()
        check(self._lib.fmm_selftest_timeout(self.h, int(polls)), self.h)

    def stage_times(self) -> list[float]:
        buf = (ctypes.c_float * 8)()
        k = self._lib.fmm_stage_times(self.h, buf, 8)
        return [buf[i] for i in range(k)]

    def pair_count(self) -> int:
        return int(self._lib.fmm_last_pair_count(self.h))

    def kernel_launches(self) -> int:
        return int(self._lib.fmm_kernel_launches(self.h))


class FMMVelocity(torch.autograd.Function):
    """(u, v) = FMM(x, y, gamma) with the library's adjoint as backward (FP64 form for the gradient)."""

    @staticmethod
    def forward(ctx, x, y, gamma, fmm: FMM):
        u, v = fmm.velocity(x.contiguous(), y.contiguous(), gamma.contiguous())
        ctx.save_for_backward(x, y, gamma)
        ctx.fmm = fmm
        return u, v

    @staticmethod
    def backward(ctx, gu, gv):
        x, y, gamma = ctx.saved_tensors
        fmm = ctx.fmm
        gu = torch.zeros_like(x) if gu is None else gu.contiguous()
        gv = torch.zeros_like(x) if gv is None else gv.contiguous()
        need = (ctx.needs_input_grad[2], ctx.needs_input_grad[0], ctx.needs_input_grad[1])
        prec = fmm.precision
        if prec != "fp64":
            fmm.set_precision("fp64")
        try:
            dg, dx, dy = fmm.adjoint(x.contiguous(), y.contiguous(), gamma.contiguous(), gu, gv, need=need)
        finally:
            if prec != "fp64":
                fmm.set_precision(prec)
        return dx, dy, dg, None


def fmm_velocity(x, y, gamma, fmm: FMM):
    """Differentiable FMM velocity: returns (u, v)."""
    return FMMVelocity.apply(x, y, gamma, fmm)
