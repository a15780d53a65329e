"""Oracle: plain, slow FP64 CPU restatement of the MG-ML(Q)MC method with sample
recycling (Robbe, Nuyens, Vandewalle, arXiv 1806.05619).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` may import this package. The GPU
library does not import it and shares no code with it.

The arithmetic lives in ``mlqmc_oracle.c`` (built here with gcc, FMA contraction
off); this module only marshals arguments through ctypes. Each wrapper names
the passage of the paper its C function follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mlqmc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK = 0
ERR_ARG = 1
ERR_OOM = 3
ERR_EXHAUSTED = 4
ERR_NOT_CONVERGED = 5


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, -ffp-contract=off)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
             "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Problem(C.Structure):
    _fields_ = [
        ("n_levels", C.c_int), ("n0", C.c_int), ("s", C.c_int),
        ("sigma", C.c_double), ("corr_len", C.c_double),
        ("qoi", C.c_int), ("mu0", C.c_int), ("nu1", C.c_int), ("nu2", C.c_int),
        ("rtol", C.c_double), ("max_cycles", C.c_int),
        ("sampler", C.c_int), ("seed", C.c_uint64), ("R", C.c_int),
        ("z", C.POINTER(C.c_uint32)), ("log2_nmax", C.c_int), ("reuse", C.c_int),
    ]


class Work(C.Structure):
    _fields_ = [("level", C.c_int32), ("pad", C.c_int32), ("n_begin", C.c_int64),
                ("n_end", C.c_int64), ("r_begin", C.c_int32), ("r_end", C.c_int32)]


class Result(C.Structure):
    _fields_ = [
        ("Q", C.c_double), ("varQ", C.c_double), ("bias", C.c_double), ("alpha", C.c_double),
        ("L", C.c_int), ("rounds", C.c_int), ("status", C.c_int), ("alpha_clamped", C.c_int),
        ("Ybar", C.c_double * 32), ("Vell", C.c_double * 32), ("C", C.c_double * 32),
        ("N", C.c_int64 * 32),
    ]


def mlmc_nopt(V, Cost, eps):
    """eq. nopt (Sec. 2): N_l = ceil(2/eps^2 sqrt(V_l/C_l) sum_t sqrt(V_t C_t))."""
    V = np.ascontiguousarray(V, dtype=np.float64)
    Cost = np.ascontiguousarray(Cost, dtype=np.float64)
    out = np.zeros(len(V))
    lib().or_mlmc_nopt(len(V) - 1, _dp(V), _dp(Cost), float(eps), _dp(out))
    return out


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int)
            L.or_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
            L.or_u64_to_unit.argtypes = [C.c_uint64]
            L.or_u64_to_unit.restype = C.c_double
            L.or_ppnd16.argtypes = [C.c_double]
            L.or_ppnd16.restype = C.c_double
            L.or_kl1d.argtypes = [C.c_double, C.c_int, dp, dp, dp]
            L.or_psi1d.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double]
            L.or_psi1d.restype = C.c_double
            L.or_modes.argtypes = [C.c_double, C.c_double, C.c_int, ip, ip, dp]
            L.or_bitrev32.argtypes = [C.c_uint32]
            L.or_bitrev32.restype = C.c_uint32
            L.or_shift_bits.argtypes = [C.c_uint64, C.c_int, C.c_int, C.c_int]
            L.or_shift_bits.restype = C.c_uint64
            L.or_lattice_bits.argtypes = [C.c_uint32, C.c_uint64, C.c_uint64]
            L.or_lattice_bits.restype = C.c_uint64
            L.or_mc_bits.argtypes = [C.c_uint64, C.c_int, C.c_int, C.c_uint64, C.c_int]
            L.or_mc_bits.restype = C.c_uint64
            L.or_ctx_new.argtypes = [C.POINTER(Problem)]
            L.or_ctx_new.restype = C.c_void_p
            L.or_ctx_free.argtypes = [C.c_void_p]
            L.or_ctx_modes.argtypes = [C.c_void_p, ip, ip, dp]
            L.or_normals.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_uint64, dp]
            L.or_field.argtypes = [C.c_void_p, C.c_int, dp, dp]
            L.or_field_z.argtypes = [C.c_void_p, C.c_int, dp, dp]
            L.or_apply_A.argtypes = [C.c_int, dp, dp, dp]
            L.or_prolong_add.argtypes = [C.c_int, dp, dp]
            L.or_prolong_add.restype = None
            L.or_sample.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_uint64, dp, dp, ip, C.c_int, ip, ip]
            L.or_fmg_fields.argtypes = [C.c_void_p, C.c_int, dp, dp, dp, dp, ip]
            L.or_vcycle_fields.argtypes = [C.c_void_p, C.c_int, dp, dp, dp]
            L.or_sample_levels.argtypes = [C.c_void_p, C.POINTER(Work), C.c_int, dp, dp]
            L.or_finalize.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int64), dp, dp, dp, dp, dp, dp]
            L.or_estimate.argtypes = [C.c_void_p, C.c_double, C.c_int, C.POINTER(Result)]
            L.or_estimate_mlmc.argtypes = [C.c_void_p, C.c_double, C.c_int, C.POINTER(Result)]
            L.or_mlmc_nopt.argtypes = [C.c_int, dp, dp, C.c_double, dp]
            L.or_mlmc_nopt.restype = None
            L.or_cbc.argtypes = [C.c_int, C.c_int, dp, C.POINTER(C.c_uint32), dp]
            L.or_cbc_criterion.argtypes = [C.c_int, C.c_int, dp, C.POINTER(C.c_uint32)]
            L.or_cbc_criterion.restype = C.c_double
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


# --------------------------------------------------------------------------- #
# Building blocks                                                             #
# --------------------------------------------------------------------------- #
def philox4x32_10(ctr, key):
    """Philox4x32-10 block (Salmon et al., SC'11)."""
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def ppnd16(p):
    """Inverse normal CDF, Wichura AS 241 (the Phi^{-1} of Sec. 3.2)."""
    f = lib().or_ppnd16
    return np.array([f(float(v)) for v in np.atleast_1d(p)])


def u64_to_unit(x):
    return lib().or_u64_to_unit(int(x))


def kl1d(corr_len, K):
    """Closed-form 1D eigenpairs of exp(-|x-x'|/lambda) on [0,1] (eq. inteq)."""
    w = np.zeros(K); th = np.zeros(K); nr = np.zeros(K)
    st = lib().or_kl1d(float(corr_len), int(K), _dp(w), _dp(th), _dp(nr))
    assert st == OK
    return w, th, nr


def psi1d(w, corr_len, nrm, x):
    f = lib().or_psi1d
    c = 1.0 / corr_len
    return np.array([f(float(w), c, float(nrm), float(v)) for v in np.atleast_1d(x)])


def modes(corr_len, sigma, s):
    """Top-s 2D modes (a, b, theta_ab) of the separable kernel (eq. truncatedKL)."""
    a = np.zeros(s, dtype=np.int32); b = np.zeros(s, dtype=np.int32); th = np.zeros(s)
    st = lib().or_modes(float(corr_len), float(sigma), int(s), _ip(a), _ip(b), _dp(th))
    assert st == OK
    return a, b, th


def bitrev32(v):
    return int(lib().or_bitrev32(int(v) & 0xFFFFFFFF))


def shift_bits(seed, level, r, j):
    return int(lib().or_shift_bits(int(seed), int(level), int(r), int(j)))


def lattice_bits(z, n, shift):
    return int(lib().or_lattice_bits(int(z) & 0xFFFFFFFF, int(n), int(shift)))


def mc_bits(seed, level, r, n, j):
    return int(lib().or_mc_bits(int(seed), int(level), int(r), int(n), int(j)))


def apply_A(n, k, u):
    """Cell-centred FV operator with harmonic-mean faces (eq. PDE)."""
    k = np.ascontiguousarray(k, dtype=np.float64).reshape(-1)
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
    out = np.zeros(n * n)
    lib().or_apply_A(int(n), _dp(k), _dp(u), _dp(out))
    return out


def prolong(nc, e):
    """Cell-centred bilinear prolongation of a coarse nc x nc grid function to
    2nc x 2nc with the odd reflection at the Dirichlet boundary (reading A4)."""
    e = np.ascontiguousarray(e, dtype=np.float64).reshape(-1)
    out = np.zeros(4 * nc * nc)
    lib().or_prolong_add(int(nc), _dp(e), _dp(out))
    return out


def cbc(s, m, gamma=None):
    """Naive CBC generating vector (Sec. 3.2; criterion of reading A13)."""
    if gamma is None:
        gamma = np.array([1.0 / (j + 1) ** 2 for j in range(s)])
    gamma = np.ascontiguousarray(gamma, dtype=np.float64)
    z = (C.c_uint32 * s)()
    e2 = np.zeros(s)
    st = lib().or_cbc(int(s), int(m), _dp(gamma), z, _dp(e2))
    assert st == OK, st
    return np.array(list(z), dtype=np.uint32), e2


def cbc_criterion(z, m, gamma=None):
    s = len(z)
    if gamma is None:
        gamma = np.array([1.0 / (j + 1) ** 2 for j in range(s)])
    gamma = np.ascontiguousarray(gamma, dtype=np.float64)
    zz = (C.c_uint32 * s)(*[int(v) for v in z])
    return lib().or_cbc_criterion(int(s), int(m), _dp(gamma), zz)


def finalize(L, R, reuse, N, sums):
    """Estimates from the sums (eqs. Upsilon-reuse, MGMLQMC, var_of_mgmlqmc,
    Upsilon-reuse-bar, sample_variances)."""
    Nn = np.ascontiguousarray(N, dtype=np.int64)
    sums = np.ascontiguousarray(sums, dtype=np.float64).reshape(-1)
    Ups = np.zeros((L + 1) * R); Yb = np.zeros(L + 1); Vl = np.zeros(L + 1)
    Q = C.c_double(); V = C.c_double()
    lib().or_finalize(int(L), int(R), int(reuse), Nn.ctypes.data_as(C.POINTER(C.c_int64)),
                      _dp(sums), _dp(Ups), _dp(Yb), _dp(Vl), C.byref(Q), C.byref(V))
    return dict(Q=Q.value, varQ=V.value, Ybar=Yb, Vell=Vl, Ups=Ups.reshape(L + 1, R))


# --------------------------------------------------------------------------- #
# Problem context                                                             #
# --------------------------------------------------------------------------- #
class Oracle:
    """One problem (PDE, covariance, sampler, estimator options) on the CPU."""

    def __init__(self, n_levels, n0, s, sigma=1.0, corr_len=0.3, qoi="mean", mu0=2, nu1=2, nu2=2,
                 rtol=0.0, max_cycles=60, sampler="lattice", seed=0, R=16, genvec=None,
                 log2_nmax=20, reuse=True):
        self.n_levels, self.n0, self.s, self.R = n_levels, n0, s, R
        self.reuse = bool(reuse)
        self._z = None
        zp = None
        if sampler == "lattice":
            assert genvec is not None and len(genvec) >= s
            self._z = (C.c_uint32 * s)(*[int(v) for v in genvec[:s]])
            zp = C.cast(self._z, C.POINTER(C.c_uint32))
        self.p = Problem(n_levels, n0, s, sigma, corr_len, 1 if qoi == "mean" else 0, mu0, nu1, nu2,
                         rtol, max_cycles, 1 if sampler == "lattice" else 0, seed, R, zp,
                         log2_nmax, 1 if reuse else 0)
        self.ctx = lib().or_ctx_new(C.byref(self.p))
        if not self.ctx:
            raise ValueError("oracle: invalid problem")

    def __del__(self):
        ctx = getattr(self, "ctx", None)
        if ctx:
            lib().or_ctx_free(ctx)
            self.ctx = None

    def n(self, t):
        return self.n0 << t

    def modes(self):
        a = np.zeros(self.s, dtype=np.int32); b = np.zeros(self.s, dtype=np.int32); th = np.zeros(self.s)
        K1 = lib().or_ctx_modes(self.ctx, _ip(a), _ip(b), _dp(th))
        return a, b, th, K1

    def normals(self, level, r, n):
        y = np.zeros(self.s)
        st = lib().or_normals(self.ctx, int(level), int(r), int(n), _dp(y))
        if st != OK:
            raise RuntimeError(f"oracle normals status {st}")
        return y

    def field(self, t, y):
        n = self.n(t)
        k = np.zeros(n * n)
        y = np.ascontiguousarray(y, dtype=np.float64)
        lib().or_field(self.ctx, int(n), _dp(y), _dp(k))
        return k

    def field_z(self, t, y):
        n = self.n(t)
        z = np.zeros(n * n)
        y = np.ascontiguousarray(y, dtype=np.float64)
        lib().or_field_z(self.ctx, int(n), _dp(y), _dp(z))
        return z

    def sample(self, level, r, n, want_u=False, log_cap=0):
        F = np.zeros(level + 1)
        tot = sum(self.n(t) ** 2 for t in range(level + 1))
        u = np.zeros(tot) if want_u else None
        log = np.zeros(max(log_cap, 1), dtype=np.int32)
        ll = C.c_int(0)
        cyc = np.zeros(level + 1, dtype=np.int32)
        st = lib().or_sample(self.ctx, int(level), int(r), int(n), _dp(F),
                             _dp(u) if want_u else None, _ip(log) if log_cap else None,
                             int(log_cap), C.byref(ll), _ip(cyc))
        out = dict(status=st, F=F, cycles=cyc)
        if want_u:
            sols, off = [], 0
            for t in range(level + 1):
                m = self.n(t) ** 2
                sols.append(u[off:off + m].copy())
                off += m
            out["u"] = sols
        if log_cap:
            out["log"] = log[:min(ll.value, log_cap)].tolist()
            out["log_len"] = ll.value
        return out

    def fmg_fields(self, level, k_levels, rhs=None):
        k_all = np.ascontiguousarray(np.concatenate([np.asarray(k, dtype=np.float64).reshape(-1)
                                                     for k in k_levels]))
        F = np.zeros(level + 1)
        tot = k_all.size
        u = np.zeros(tot)
        cyc = np.zeros(level + 1, dtype=np.int32)
        rp = None
        if rhs is not None:
            rhs = np.ascontiguousarray(rhs, dtype=np.float64).reshape(-1)
            rp = _dp(rhs)
        st = lib().or_fmg_fields(self.ctx, int(level), _dp(k_all), rp, _dp(F), _dp(u), _ip(cyc))
        sols, off = [], 0
        for t in range(level + 1):
            m = self.n(t) ** 2
            sols.append(u[off:off + m].copy())
            off += m
        return dict(status=st, F=F, u=sols, cycles=cyc)

    def vcycle_fields(self, t, k_levels, b, u):
        k_all = np.ascontiguousarray(np.concatenate([np.asarray(k, dtype=np.float64).reshape(-1)
                                                     for k in k_levels[:t + 1]]))
        b = np.ascontiguousarray(b, dtype=np.float64).reshape(-1).copy()
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1).copy()
        st = lib().or_vcycle_fields(self.ctx, int(t), _dp(k_all), _dp(b), _dp(u))
        assert st == OK
        return u

    def sample_levels(self, work, want_F=False):
        """work: list of (level, n_begin, n_end, r_begin, r_end). Returns sums[L+1][R][2]."""
        arr = (Work * len(work))()
        nsamp = 0
        for i, (lv, nb, ne, rb, re_) in enumerate(work):
            arr[i] = Work(lv, 0, nb, ne, rb, re_)
            nsamp += (ne - nb) * (re_ - rb)
        sums = np.zeros(self.n_levels * self.R * 2)
        F = np.zeros(nsamp * self.n_levels) if want_F else None
        st = lib().or_sample_levels(self.ctx, arr, len(work), _dp(sums), _dp(F) if want_F else None)
        if st != OK:
            raise RuntimeError(f"oracle sample_levels status {st}")
        out = dict(sums=sums.reshape(self.n_levels, self.R, 2))
        if want_F:
            out["F"] = F.reshape(nsamp, self.n_levels)
        return out

    def estimate_mlmc(self, eps, max_rounds=200):
        """Plain MLMC (Sec. 2: eqs. MSE, vardecomp, nopt; reading A28); Monte Carlo
        sampler and no recycling only."""
        res = Result()
        st = lib().or_estimate_mlmc(self.ctx, float(eps), int(max_rounds), C.byref(res))
        L = res.L
        return dict(status=st, run_status=res.status, Q=res.Q, varQ=res.varQ, bias=res.bias,
                    alpha=res.alpha, alpha_clamped=res.alpha_clamped, L=L, rounds=res.rounds,
                    N=[res.N[i] for i in range(self.n_levels)],
                    Ybar=[res.Ybar[i] for i in range(self.n_levels)],
                    Vell=[res.Vell[i] for i in range(self.n_levels)],
                    C=[res.C[i] for i in range(self.n_levels)])

    def estimate(self, eps, max_rounds=200):
        """Algorithm 1 with the deterministic cost model C_l = sum_{t<=l} n_t^2."""
        res = Result()
        st = lib().or_estimate(self.ctx, float(eps), int(max_rounds), C.byref(res))
        L = res.L
        return dict(status=st, run_status=res.status, Q=res.Q, varQ=res.varQ, bias=res.bias,
                    alpha=res.alpha, alpha_clamped=res.alpha_clamped, L=L, rounds=res.rounds,
                    N=[res.N[i] for i in range(self.n_levels)],
                    Ybar=[res.Ybar[i] for i in range(self.n_levels)],
                    Vell=[res.Vell[i] for i in range(self.n_levels)],
                    C=[res.C[i] for i in range(self.n_levels)])
