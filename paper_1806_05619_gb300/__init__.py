"""GB300 (sm_103a) library for the multigrid multilevel (quasi-)Monte Carlo
method with sample recycling (Robbe, Nuyens, Vandewalle, arXiv 1806.05619).

This module only marshals arguments to the C ABI declared in
``include/mlqmc.h`` (``libmlqmc.so``, built in-tree by :func:`build`). Every
step of the method runs in the library's CUDA kernels; PyTorch is used for
device memory and streams only. Importing works without a GPU; any call that
needs the library raises if ``libmlqmc.so`` is missing.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Iterable, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmlqmc.so")
_lock = threading.Lock()
_lib = None

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "POINTS_EXHAUSTED", 5: "NOT_CONVERGED",
          6: "TIMEOUT", 7: "DEVICE_STATUS", 8: "UNSUPPORTED", 9: "SCRATCH_LIMIT"}
PRECISION = {"fp64": 0, "mixed_tf32": 1, "mixed_bf16x3": 2}
QOI = {"center": 0, "mean": 1}
SAMPLER = {"mc": 0, "lattice": 1}


class MlqmcError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)} ({_status_text(code)})")


class Problem(C.Structure):
    _fields_ = [
        ("n_levels", C.c_int32), ("coarse_cells", C.c_int32), ("n_modes", C.c_int32), ("pad0", C.c_int32),
        ("sigma", C.c_double), ("corr_len", C.c_double),
        ("qoi", C.c_int32), ("mu0", C.c_int32), ("nu1", C.c_int32), ("nu2", C.c_int32),
        ("precision", C.c_int32), ("pad1", C.c_int32),
        ("refine_rtol", C.c_double), ("refine_max_iter", C.c_int32), ("sampler", C.c_int32),
        ("seed", C.c_uint64), ("n_shifts", C.c_int32), ("pad2", C.c_int32),
        ("genvec", C.POINTER(C.c_uint32)), ("log2_nmax", C.c_int32), ("reuse", C.c_int32),
        ("covariance", C.c_int32), ("nystrom_m", C.c_int32), ("matern_nu", C.c_double),
        ("nystrom_theta", C.POINTER(C.c_double)), ("nystrom_psi", C.POINTER(C.c_double)),
    ]


class Work(C.Structure):
    _fields_ = [("level", C.c_int32), ("pad", C.c_int32), ("n_begin", C.c_int64), ("n_end", C.c_int64),
                ("r_begin", C.c_int32), ("r_end", C.c_int32)]


class RunOpts(C.Structure):
    _fields_ = [("max_rounds", C.c_int32), ("cost_model", C.c_int32), ("batched", C.c_int32),
                ("pad", C.c_int32)]


class Result(C.Structure):
    _fields_ = [
        ("Q", C.c_double), ("varQ", C.c_double), ("bias", C.c_double), ("alpha", C.c_double),
        ("L", C.c_int32), ("rounds", C.c_int32), ("run_status", C.c_int32), ("alpha_clamped", C.c_int32),
        ("wall_seconds", C.c_double), ("gpu_seconds", C.c_double),
        ("N", C.c_int64 * 32), ("Ybar", C.c_double * 32), ("Vell", C.c_double * 32), ("C", C.c_double * 32),
    ]


MIMC_MAX_M = 8


class MimcResult(C.Structure):
    _fields_ = [
        ("Q", C.c_double), ("varQ", C.c_double), ("bias", C.c_double), ("alpha", C.c_double),
        ("bias_cycles", C.c_double),
        ("L", C.c_int32), ("K", C.c_int32), ("rounds", C.c_int32), ("run_status", C.c_int32),
        ("alpha_clamped", C.c_int32), ("pad", C.c_int32),
        ("wall_seconds", C.c_double), ("gpu_seconds", C.c_double),
        ("N", C.c_int64 * (MIMC_MAX_M * 32)), ("Ybar", C.c_double * (MIMC_MAX_M * 32)),
        ("Vell", C.c_double * (MIMC_MAX_M * 32)), ("C", C.c_double * (MIMC_MAX_M * 32)),
    ]


def build(verbose: bool = False) -> str:
    """Compile ``libmlqmc.so`` for sm_103a in-tree (nvcc)."""
    from . import buildlib as _b
    return _b.build(verbose=verbose)


def lib():
    """The loaded C library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libmlqmc.so is not built ({LIB_PATH}); call paper_1806_05619_gb300.build()")
            L = C.CDLL(LIB_PATH)
            vp, i32, i64, dp = C.c_void_p, C.c_int32, C.c_int64, C.POINTER(C.c_double)
            L.mlqmc_create.argtypes = [C.POINTER(Problem), i64, C.POINTER(vp)]
            L.mlqmc_destroy.argtypes = [vp]
            L.mlqmc_destroy.restype = None
            L.mlqmc_sample_levels.argtypes = [vp, C.POINTER(Work), i32, vp, vp, vp]
            L.mlqmc_estimate.argtypes = [vp, C.c_double, C.POINTER(RunOpts), C.POINTER(Result)]
            L.mlqmc_estimate_mlmc.argtypes = [vp, C.c_double, C.POINTER(RunOpts), C.POINTER(Result)]
            L.mlqmc_sample_mixed.argtypes = [vp, vp, C.POINTER(Work), i32, vp, vp, vp]
            L.mlqmc_estimate_mimc.argtypes = [C.POINTER(vp), i32, C.c_double, C.POINTER(RunOpts),
                                              C.POINTER(MimcResult)]
            L.mlqmc_nystrom_modes.argtypes = [C.c_double, C.c_double, C.c_double, i32, i32, dp, dp]
            L.mlqmc_get_device_status.argtypes = [vp, vp]
            L.mlqmc_status_string.argtypes = [C.c_int]
            L.mlqmc_status_string.restype = C.c_char_p
            L.mlqmc_cbc_genvec.argtypes = [i32, i32, dp, C.POINTER(C.c_uint32), dp]
            L.mlqmc_modes.argtypes = [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), dp]
            L.mlqmc_point_bits.argtypes = [vp, i32, i32, i64, i32, vp, vp]
            L.mlqmc_normals.argtypes = [vp, i32, i32, i64, i32, vp, vp]
            L.mlqmc_fields.argtypes = [vp, i32, vp, i32, vp, vp]
            L.mlqmc_sample_solution.argtypes = [vp, i32, i32, i64, vp, vp, vp]
            L.mlqmc_fmg_fields_noalloc.argtypes = [i32, i32, i32, i32, i32, i32, i32, vp, vp, vp]
            L.mlqmc_last_iterations.argtypes = [vp, C.POINTER(C.c_int32)]
            L.mlqmc_profile.argtypes = [vp, i32]
            L.mlqmc_profile_read.argtypes = [vp, dp, C.POINTER(C.c_int64)]
            L.mlqmc_profile_work.argtypes = [vp, dp, dp, dp, dp]
            L.mlqmc_profile_read_levels.argtypes = [vp, dp, C.POINTER(C.c_int64), dp, dp, dp, dp]
            L.mlqmc_smoother_info.argtypes = [vp, C.POINTER(C.c_int32), dp]
            L.mlqmc_set_smoother.argtypes = [vp, i32, i32]
            L.mlqmc_schedule_info.argtypes = [vp, C.POINTER(C.c_int32), dp, C.POINTER(C.c_int32), dp]
            L.mlqmc_set_graphs.argtypes = [vp, i32]
            L.mlqmc_estimator_from_sums.argtypes = [i32, i32, i32, C.POINTER(C.c_int64), dp, dp, dp, dp, dp]
            L.mlqmc_graph_stats.argtypes = [vp, C.POINTER(C.c_int64)]
            L.mlqmc_set_round_graphs.argtypes = [vp, i32]
            L.mlqmc_test_wait_timeout.argtypes = [vp, i64, vp]
            L.mlqmc_graph_replays.argtypes = [vp]
            L.mlqmc_graph_replays.restype = i64
            L.mlqmc_launch_count.argtypes = [vp]
            L.mlqmc_launch_count.restype = i64
            for name in ["mlqmc_create", "mlqmc_sample_levels", "mlqmc_estimate", "mlqmc_estimate_mlmc",
                         "mlqmc_sample_mixed", "mlqmc_estimate_mimc",
                         "mlqmc_nystrom_modes",
                         "mlqmc_get_device_status",
                         "mlqmc_cbc_genvec", "mlqmc_modes", "mlqmc_point_bits", "mlqmc_normals", "mlqmc_fields",
                         "mlqmc_sample_solution", "mlqmc_profile", "mlqmc_profile_read", "mlqmc_profile_work", "mlqmc_profile_read_levels", "mlqmc_smoother_info", "mlqmc_set_smoother", "mlqmc_schedule_info", "mlqmc_set_graphs",
                         "mlqmc_estimator_from_sums", "mlqmc_graph_stats", "mlqmc_set_round_graphs", "mlqmc_test_wait_timeout",
                         "mlqmc_fmg_fields_noalloc", "mlqmc_last_iterations"]:
                getattr(L, name).restype = C.c_int
            _lib = L
    return _lib


def _status_text(code: int) -> str:
    try:
        return lib().mlqmc_status_string(int(code)).decode()
    except Exception:
        return ""


def _check(code: int, where: str):
    if code != 0:
        raise MlqmcError(code, where)


def cbc_genvec(s: int, m: int, gamma: Optional[Sequence[float]] = None):
    """CBC generating vector for 2^m points with product weights (default j^-2)."""
    if gamma is None:
        gamma = [1.0 / (j + 1) ** 2 for j in range(s)]
    g = np.ascontiguousarray(gamma, dtype=np.float64)
    z = (C.c_uint32 * s)()
    e2 = np.zeros(s)
    _check(lib().mlqmc_cbc_genvec(int(s), int(m), g.ctypes.data_as(C.POINTER(C.c_double)), z,
                                  e2.ctypes.data_as(C.POINTER(C.c_double))), "mlqmc_cbc_genvec")
    return np.array(list(z), dtype=np.uint32), e2


def estimator_from_sums(N, sums, R: int, reuse: bool = True):
    """Q, varQ, Ybar, Vell from reuse sums [L+1][R][2] (host; eqs. MGMLQMC,
    var_of_mgmlqmc, Upsilon-reuse-bar, sample_variances)."""
    Nn = np.ascontiguousarray(N, dtype=np.int64)
    S = np.ascontiguousarray(sums, dtype=np.float64).reshape(-1)
    L = len(Nn) - 1
    if S.size != (L + 1) * R * 2:
        raise ValueError("sums must hold (L+1) x R x 2 values")
    Q, V = C.c_double(), C.c_double()
    Yb, Vl = np.zeros(L + 1), np.zeros(L + 1)
    dp = C.POINTER(C.c_double)
    _check(lib().mlqmc_estimator_from_sums(int(L), int(R), 1 if reuse else 0, Nn.ctypes.data_as(C.POINTER(C.c_int64)),
                                           S.ctypes.data_as(dp), C.byref(Q), C.byref(V), Yb.ctypes.data_as(dp),
                                           Vl.ctypes.data_as(dp)), "mlqmc_estimator_from_sums")
    return dict(Q=Q.value, varQ=V.value, Ybar=Yb, Vell=Vl)


COVARIANCE = {"sep_exp": 0, "matern": 1}


def nystrom_modes(nu, corr_len, sigma, m, s):
    """Nystrom eigenpairs of the Matern covariance on the m x m midpoint nodes
    (``mlqmc_nystrom_modes``): (theta (s,), psi (m*m, s)), descending."""
    th = np.zeros(s)
    ps = np.zeros(m * m * s)
    dp = C.POINTER(C.c_double)
    _check(lib().mlqmc_nystrom_modes(float(nu), float(corr_len), float(sigma), int(m), int(s), th.ctypes.data_as(dp),
                                     ps.ctypes.data_as(dp)), "mlqmc_nystrom_modes")
    return th, ps.reshape(m * m, s)


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    return C.c_void_p(int(t.data_ptr()))


def _stream(stream) -> C.c_void_p:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(int(stream.cuda_stream))


class Context:
    """One problem on the current CUDA device (wraps ``mlqmc_ctx``)."""

    def __init__(self, n_levels, coarse_cells, n_modes, sigma=1.0, corr_len=0.3, qoi="mean", mu0=2, nu1=2,
                 nu2=2, precision="fp64", refine_rtol=0.0, refine_max_iter=60, sampler="lattice", seed=0,
                 n_shifts=16, genvec=None, log2_nmax=20, reuse=True, max_samples=65536, covariance="sep_exp",
                 matern_nu=0.5, nystrom_m=0, nystrom_theta=None, nystrom_psi=None):
        """covariance "matern": Matern covariance (eq. matern) with the Nystrom
        eigenpairs nystrom_theta (n_modes) and nystrom_psi (nystrom_m^2 x n_modes,
        node-major) as `nystrom_modes` returns them."""
        self.n_levels, self.n0, self.s, self.R = n_levels, coarse_cells, n_modes, n_shifts
        self.precision = precision
        zp = None
        self._z = None
        if sampler == "lattice":
            if genvec is None:
                raise ValueError("lattice sampler needs a generating vector")
            self._z = (C.c_uint32 * n_modes)(*[int(v) for v in genvec[:n_modes]])
            zp = C.cast(self._z, C.POINTER(C.c_uint32))
        p = Problem(n_levels=n_levels, coarse_cells=coarse_cells, n_modes=n_modes, sigma=sigma, corr_len=corr_len,
                    qoi=QOI[qoi], mu0=mu0, nu1=nu1, nu2=nu2, precision=PRECISION[precision],
                    refine_rtol=refine_rtol, refine_max_iter=refine_max_iter, sampler=SAMPLER[sampler],
                    seed=seed, n_shifts=n_shifts, genvec=zp, log2_nmax=log2_nmax, reuse=1 if reuse else 0)
        if covariance == "matern":
            th = np.ascontiguousarray(nystrom_theta, dtype=np.float64)
            ps = np.ascontiguousarray(nystrom_psi, dtype=np.float64)
            if th.size != n_modes or ps.size != nystrom_m * nystrom_m * n_modes:
                raise ValueError("Nystrom modes: n_modes eigenvalues and nystrom_m^2 x n_modes nodal values")
            p.covariance, p.nystrom_m, p.matern_nu = COVARIANCE["matern"], int(nystrom_m), float(matern_nu)
            p.nystrom_theta = th.ctypes.data_as(C.POINTER(C.c_double))
            p.nystrom_psi = ps.ctypes.data_as(C.POINTER(C.c_double))
        elif covariance != "sep_exp":
            raise ValueError(f"unknown covariance {covariance!r}")
        h = C.c_void_p()
        _check(lib().mlqmc_create(C.byref(p), int(max_samples), C.byref(h)), "mlqmc_create")
        self.h = h

    @classmethod
    def from_config(cls, cfg: dict, genvec=None, **over):
        kw = dict(n_levels=cfg["n_levels"], coarse_cells=cfg["n0"], n_modes=cfg["s"], sigma=cfg["sigma"],
                  corr_len=cfg["corr_len"], qoi=cfg["qoi"], mu0=cfg["mu0"], nu1=cfg["nu1"], nu2=cfg["nu2"],
                  precision=cfg["precision"], refine_rtol=cfg["rtol"], refine_max_iter=cfg["max_cycles"],
                  sampler=cfg["sampler"], seed=cfg["seed"], n_shifts=cfg["R"], log2_nmax=cfg["log2_nmax"],
                  reuse=cfg["reuse"], genvec=genvec)
        kw.update(over)
        return cls(**kw)

    def close(self):
        if getattr(self, "h", None):
            lib().mlqmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def n(self, t):
        return self.n0 << t

    def modes(self):
        a = (C.c_int32 * self.s)(); b = (C.c_int32 * self.s)(); th = np.zeros(self.s)
        _check(lib().mlqmc_modes(self.h, a, b, th.ctypes.data_as(C.POINTER(C.c_double))), "mlqmc_modes")
        return np.array(list(a)), np.array(list(b)), th

    def sample_levels(self, work: Iterable, sums, F=None, stream=None):
        """Accumulate the reuse sums (device tensor n_levels x R x 2, float64) for a work list."""
        work = list(work)
        arr = (Work * max(1, len(work)))()
        for i, (lv, nb, ne, rb, re_) in enumerate(work):
            arr[i] = Work(level=lv, pad=0, n_begin=nb, n_end=ne, r_begin=rb, r_end=re_)
        _check(lib().mlqmc_sample_levels(self.h, arr, len(work), _ptr(sums), _ptr(F), _stream(stream)),
               "mlqmc_sample_levels")

    def sample_mixed(self, lo, work: Iterable, sums, D=None, stream=None):
        """Accumulate the sums of the mixed differences D_{t,m} (this context's
        cycle count against ``lo``'s; ``lo=None`` for the first direction) into
        ``sums`` (device n_levels x R x 2, float64); per-sample D into ``D``."""
        work = list(work)
        arr = (Work * max(1, len(work)))()
        for i, (lv, nb, ne, rb, re_) in enumerate(work):
            arr[i] = Work(level=lv, pad=0, n_begin=nb, n_end=ne, r_begin=rb, r_end=re_)
        _check(lib().mlqmc_sample_mixed(self.h, lo.h if lo is not None else None, arr, len(work), _ptr(sums),
                                        _ptr(D), _stream(stream)), "mlqmc_sample_mixed")

    def device_status(self, stream=None):
        return lib().mlqmc_get_device_status(self.h, _stream(stream))

    def check_device(self, stream=None):
        _check(self.device_status(stream), "device status")

    def estimate(self, eps, max_rounds=0, cost_model=0, batched=False):
        o = RunOpts(max_rounds=max_rounds, cost_model=cost_model, batched=1 if batched else 0)
        res = Result()
        _check(lib().mlqmc_estimate(self.h, float(eps), C.byref(o), C.byref(res)), "mlqmc_estimate")
        L = res.L
        return dict(Q=res.Q, varQ=res.varQ, bias=res.bias, alpha=res.alpha, L=L, rounds=res.rounds,
                    run_status=res.run_status, alpha_clamped=res.alpha_clamped, wall_seconds=res.wall_seconds,
                    gpu_seconds=res.gpu_seconds, N=[res.N[i] for i in range(self.n_levels)],
                    Ybar=[res.Ybar[i] for i in range(self.n_levels)],
                    Vell=[res.Vell[i] for i in range(self.n_levels)], C=[res.C[i] for i in range(self.n_levels)])

    def estimate_mlmc(self, eps, max_rounds=0, cost_model=0):
        """Plain MLMC (Monte Carlo sampler, no recycling): the comparison baseline
        of the paper's speed-ups, sample counts from eq. nopt."""
        o = RunOpts(max_rounds=max_rounds, cost_model=cost_model, batched=0)
        res = Result()
        _check(lib().mlqmc_estimate_mlmc(self.h, float(eps), C.byref(o), C.byref(res)), "mlqmc_estimate_mlmc")
        L = res.L
        return dict(Q=res.Q, varQ=res.varQ, bias=res.bias, alpha=res.alpha, L=L, rounds=res.rounds,
                    run_status=res.run_status, alpha_clamped=res.alpha_clamped, wall_seconds=res.wall_seconds,
                    gpu_seconds=res.gpu_seconds, N=[res.N[i] for i in range(self.n_levels)],
                    Ybar=[res.Ybar[i] for i in range(self.n_levels)],
                    Vell=[res.Vell[i] for i in range(self.n_levels)], C=[res.C[i] for i in range(self.n_levels)])

    def point_bits(self, level, r, n_begin, count, stream=None):
        import torch
        out = torch.empty(count * self.s, dtype=torch.int64, device="cuda")
        _check(lib().mlqmc_point_bits(self.h, level, r, n_begin, count, _ptr(out), _stream(stream)), "point_bits")
        return out.view(count, self.s)

    def normals(self, level, r, n_begin, count, stream=None):
        import torch
        out = torch.empty(count * self.s, dtype=torch.float64, device="cuda")
        _check(lib().mlqmc_normals(self.h, level, r, n_begin, count, _ptr(out), _stream(stream)), "normals")
        return out.view(count, self.s)

    def fields(self, t, y, stream=None):
        import torch
        y = y.to(device="cuda", dtype=torch.float64).contiguous()
        count = y.shape[0]
        out = torch.empty(count * self.n(t) ** 2, dtype=torch.float64, device="cuda")
        _check(lib().mlqmc_fields(self.h, t, _ptr(y), count, _ptr(out), _stream(stream)), "fields")
        return out.view(count, self.n(t) ** 2)

    def sample_solution(self, level, r, n, stream=None):
        import torch
        tot = sum(self.n(t) ** 2 for t in range(level + 1))
        u = torch.empty(tot, dtype=torch.float64, device="cuda")
        F = torch.empty(level + 1, dtype=torch.float64, device="cuda")
        _check(lib().mlqmc_sample_solution(self.h, level, r, n, _ptr(u), _ptr(F), _stream(stream)),
               "sample_solution")
        sols, off = [], 0
        for t in range(level + 1):
            m = self.n(t) ** 2
            sols.append(u[off:off + m])
            off += m
        return sols, F

    def profile(self, enable: bool = True):
        """Start (or stop) per-kernel CUDA-event timing of sample_levels; clears totals."""
        _check(lib().mlqmc_profile(self.h, 1 if enable else 0), "mlqmc_profile")

    PROFILE_KINDS = ["points", "level0", "synth", "smooth", "transfer", "coarse", "reduce", "kl_tc"]

    def profile_read(self):
        """{kind: (ms, launches)} per kernel kind since profile(); kinds as in mlqmc_profile_read."""
        ms = np.zeros(8)
        n = (C.c_int64 * 8)()
        _check(lib().mlqmc_profile_read(self.h, ms.ctypes.data_as(C.POINTER(C.c_double)), n), "mlqmc_profile_read")
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(self.PROFILE_KINDS)}

    def profile_work(self):
        """{kind: {"bytes", "f64", "f32", "ftc"}}: algorithmic work of the launches since profile()."""
        a = [np.zeros(8) for _ in range(4)]
        _check(lib().mlqmc_profile_work(self.h, *[x.ctypes.data_as(C.POINTER(C.c_double)) for x in a]),
               "mlqmc_profile_work")
        return {k: {"bytes": float(a[0][i]), "f64": float(a[1][i]), "f32": float(a[2][i]), "ftc": float(a[3][i])}
                for i, k in enumerate(self.PROFILE_KINDS)}

    PROFILE_LEVELS = 13  # MLQMC_PROFILE_LEVELS: levels 0..11, then launches of no single level

    def profile_read_levels(self):
        """{(kind, level): {"ms", "n", "bytes", "f64", "f32", "ftc"}} since profile(), for
        the buckets with launches; level None holds the launches of no single level."""
        nk, nl = len(self.PROFILE_KINDS), self.PROFILE_LEVELS
        ms, by, f64, f32, ftc = (np.zeros(nk * nl) for _ in range(5))
        n = np.zeros(nk * nl, dtype=np.int64)
        dpp = C.POINTER(C.c_double)
        _check(lib().mlqmc_profile_read_levels(self.h, ms.ctypes.data_as(dpp), n.ctypes.data_as(C.POINTER(C.c_int64)),
                                               by.ctypes.data_as(dpp), f64.ctypes.data_as(dpp),
                                               f32.ctypes.data_as(dpp), ftc.ctypes.data_as(dpp)),
               "mlqmc_profile_read_levels")
        out = {}
        for k, name in enumerate(self.PROFILE_KINDS):
            for t in range(nl):
                i = k * nl + t
                if n[i] == 0:
                    continue
                out[(name, t if t < nl - 1 else None)] = {"ms": float(ms[i]), "n": int(n[i]), "bytes": float(by[i]),
                                                          "f64": float(f64[i]), "f32": float(f32[i]),
                                                          "ftc": float(ftc[i])}
        return out

    def last_iterations(self):
        """Per level, the most extra cycles / refinement steps any sample needed since the last query."""
        out = (C.c_int32 * self.n_levels)()
        _check(lib().mlqmc_last_iterations(self.h, out), "mlqmc_last_iterations")
        return list(out)

    SMOOTHERS = ["gs", "tile", "stream", "tma", "whole"]

    def smoother_info(self):
        """Per level (smoother name, {name: tuned ms}); level 0 has no sweeps."""
        kind = (C.c_int32 * self.n_levels)()
        nk = len(self.SMOOTHERS)
        ms = np.zeros(self.n_levels * nk)
        _check(lib().mlqmc_smoother_info(self.h, kind, ms.ctypes.data_as(C.POINTER(C.c_double))), "mlqmc_smoother_info")
        ms = ms.reshape(self.n_levels, nk)
        return [(self.SMOOTHERS[kind[t]], {self.SMOOTHERS[k]: float(ms[t, k]) for k in range(nk) if ms[t, k] > 0})
                for t in range(self.n_levels)]

    def schedule_info(self):
        """The autotuner's batch-size schedule: per level the small-batch smoother
        (with its tuning times) and the KL tile width (samples per tile) for
        small and large batches (with the timings of widths 128 and 256)."""
        nl, nk = self.n_levels, len(self.SMOOTHERS)
        ss = (C.c_int32 * nl)()
        sms = np.zeros(nl * nk)
        nt = (C.c_int32 * (2 * nl))()
        kms = np.zeros(nl * 4)
        dpp = C.POINTER(C.c_double)
        _check(lib().mlqmc_schedule_info(self.h, ss, sms.ctypes.data_as(dpp), nt, kms.ctypes.data_as(dpp)),
               "mlqmc_schedule_info")
        sms, kms = sms.reshape(nl, nk), kms.reshape(nl, 2, 2)
        return [{"smoother_small": self.SMOOTHERS[ss[t]],
                 "small_ms": {self.SMOOTHERS[k]: float(sms[t, k]) for k in range(nk) if sms[t, k] > 0},
                 "kl_nt": [nt[2 * t], nt[2 * t + 1]],
                 "kl_ms": [[float(kms[t, c_, k]) for k in range(2)] for c_ in range(2)]} for t in range(nl)]

    def set_smoother(self, level: int, name: str):
        """Force smoother `name` ("tile", "stream", "tma" or "whole") on `level` for later calls."""
        _check(lib().mlqmc_set_smoother(self.h, int(level), self.SMOOTHERS.index(name)), "mlqmc_set_smoother")

    def set_graphs(self, enable: bool):
        """Graph replay of repeated identical fixed-cycle calls (on by default)."""
        _check(lib().mlqmc_set_graphs(self.h, 1 if enable else 0), "mlqmc_set_graphs")

    def graph_replays(self) -> int:
        return int(lib().mlqmc_graph_replays(self.h))

    ROUND_GRAPHS = {"off": 0, "on": 1, "converged": 2}

    def set_round_graphs(self, mode: str):
        """Which one-off calls run as one graph launch: "off", "on", or "converged"
        (the default: calls of the converged forms only)."""
        _check(lib().mlqmc_set_round_graphs(self.h, self.ROUND_GRAPHS[mode]), "mlqmc_set_round_graphs")

    def graph_stats(self):
        """{"replays", "round_launches", "round_updates", "round_instantiations"} since creation."""
        out = (C.c_int64 * 4)()
        _check(lib().mlqmc_graph_stats(self.h, out), "mlqmc_graph_stats")
        return dict(zip(["replays", "round_launches", "round_updates", "round_instantiations"], list(out)))

    def launch_count(self) -> int:
        return int(lib().mlqmc_launch_count(self.h))


def estimate_mimc(contexts, eps, max_rounds=0, cost_model=0, batched=False):
    """Multi-index MLQMC (grid level x V-cycle count): Algorithm 1 over the
    levels with every cycle count at each level; ``contexts`` differ only in
    mu0, strictly increasing. Entries of N, Ybar, Vell and C are indexed
    [m][t], t = 0..L."""
    K = len(contexts)
    hs = (C.c_void_p * max(1, K))(*[c.h for c in contexts])
    o = RunOpts(max_rounds=max_rounds, cost_model=cost_model, batched=1 if batched else 0)
    res = MimcResult()
    _check(lib().mlqmc_estimate_mimc(hs, K, float(eps), C.byref(o), C.byref(res)), "mlqmc_estimate_mimc")
    nl = res.L + 1

    def grid(a):
        return [[a[m * 32 + t] for t in range(nl)] for m in range(K)]

    return dict(Q=res.Q, varQ=res.varQ, bias=res.bias, alpha=res.alpha, bias_cycles=res.bias_cycles, L=res.L,
                K=res.K, rounds=res.rounds, run_status=res.run_status, alpha_clamped=res.alpha_clamped,
                wall_seconds=res.wall_seconds, gpu_seconds=res.gpu_seconds,
                N=grid(res.N), Ybar=grid(res.Ybar), Vell=grid(res.Vell), C=grid(res.C))
