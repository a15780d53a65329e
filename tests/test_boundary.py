"""C-ABI boundary checks that need no GPU: the library builds and loads, it
exports every entry point that include/mlqmc.h declares, the ctypes layouts
match the C structs, host-side validation rejects bad problems, and the
host-only CBC construction agrees with the oracle's."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

import oracle as O
import paper_1806_05619_gb300 as M

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mlqmc.h")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(M.LIB_PATH):
        M.build()
    return M.lib()


def _declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mlqmc_[a-z_0-9]+)\s*\(", txt)))


def test_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert "mlqmc_sample_levels" in names and "mlqmc_estimate" in names
    nm = subprocess.run(["nm", "-D", "--defined-only", M.LIB_PATH], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s+(mlqmc_\w+)", nm))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(lib, n)


def test_struct_layouts_match_header():
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "mlqmc.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(mlqmc_problem), offsetof(mlqmc_problem, genvec),
         offsetof(mlqmc_problem, reuse), sizeof(mlqmc_work), sizeof(mlqmc_run_opts), sizeof(mlqmc_result),
         offsetof(mlqmc_result, C), sizeof(mlqmc_mimc_result), offsetof(mlqmc_mimc_result, N),
         offsetof(mlqmc_mimc_result, C));
  return 0;
}'''
    with tempfile.TemporaryDirectory() as d:
        cfile = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(cfile, "w").write(src)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), cfile, "-o", exe])
        vals = [int(v) for v in subprocess.check_output([exe]).split()]
    want = [C.sizeof(M.Problem), M.Problem.genvec.offset, M.Problem.reuse.offset, C.sizeof(M.Work),
            C.sizeof(M.RunOpts), C.sizeof(M.Result), M.Result.C.offset, C.sizeof(M.MimcResult),
            M.MimcResult.N.offset, M.MimcResult.C.offset]
    assert vals == want


def test_multi_index_entries_reject_bad_arguments_before_touching_the_device(lib):
    w = (M.Work * 1)(M.Work(level=0, pad=0, n_begin=0, n_end=1, r_begin=0, r_end=1))
    sums = C.c_void_p(256)  # never dereferenced: the calls return first
    assert lib.mlqmc_sample_mixed(None, None, w, 1, sums, None, None) == 1
    res = M.MimcResult()
    o = M.RunOpts()
    hs = (C.c_void_p * 2)()
    assert lib.mlqmc_estimate_mimc(None, 1, 1e-3, C.byref(o), C.byref(res)) == 1
    assert lib.mlqmc_estimate_mimc(hs, 0, 1e-3, C.byref(o), C.byref(res)) == 1   # K < 1
    assert lib.mlqmc_estimate_mimc(hs, 9, 1e-3, C.byref(o), C.byref(res)) == 1   # K > MLQMC_MIMC_MAX_M
    assert lib.mlqmc_estimate_mimc(hs, 2, 1e-3, C.byref(o), C.byref(res)) == 1   # NULL contexts
    assert lib.mlqmc_estimate_mimc(hs, 2, 0.0, C.byref(o), C.byref(res)) == 1    # eps <= 0


def test_status_strings(lib):
    for code in range(10):
        assert len(lib.mlqmc_status_string(code)) > 0


def _problem(**kw):
    base = dict(n_levels=3, coarse_cells=4, n_modes=4, sigma=1.0, corr_len=0.3, qoi=1, mu0=2, nu1=2, nu2=2,
                precision=0, refine_rtol=0.0, refine_max_iter=10, sampler=0, seed=1, n_shifts=2, genvec=None,
                log2_nmax=10, reuse=1)
    base.update(kw)
    return M.Problem(**base)


@pytest.mark.parametrize("bad", [dict(n_levels=0), dict(n_levels=13), dict(coarse_cells=3), dict(n_modes=0),
                                 dict(corr_len=0.0), dict(qoi=5), dict(mu0=0), dict(n_shifts=0),
                                 dict(precision=9), dict(sampler=1), dict(reuse=2), dict(refine_rtol=-1.0)])
def test_create_rejects_bad_problems_before_touching_the_device(lib, bad):
    p = _problem(**bad)
    h = C.c_void_p()
    assert lib.mlqmc_create(C.byref(p), 0, C.byref(h)) == 1
    assert not h.value


def _matern_problem(nu=1.5, m=4, theta=(0.5, 0.2, 0.1, 0.05), with_psi=True, **kw):
    p = _problem(**kw)
    th = (C.c_double * len(theta))(*theta)
    ps = (C.c_double * (m * m * 4))()
    p.covariance, p.nystrom_m, p.matern_nu = 1, m, nu
    p.nystrom_theta = C.cast(th, C.POINTER(C.c_double))
    p.nystrom_psi = C.cast(ps, C.POINTER(C.c_double)) if with_psi else None
    return p, (th, ps)


@pytest.mark.parametrize("bad", [dict(nu=0.75), dict(nu=3.0), dict(m=1), dict(m=129), dict(with_psi=False),
                                 dict(theta=(0.5, 0.0, 0.1, 0.05)), dict(theta=(0.5, -1.0, 0.1, 0.05)),
                                 dict(m=1, n_modes=4)])
def test_create_rejects_bad_matern_problems_before_touching_the_device(lib, bad):
    p, keep = _matern_problem(**bad)
    h = C.c_void_p()
    assert lib.mlqmc_create(C.byref(p), 0, C.byref(h)) == 1
    assert not h.value


def test_create_rejects_unknown_covariance_and_more_modes_than_nodes(lib):
    p = _problem()
    p.covariance = 2
    h = C.c_void_p()
    assert lib.mlqmc_create(C.byref(p), 0, C.byref(h)) == 1
    p, keep = _matern_problem(m=2, n_modes=5, theta=(0.5, 0.2, 0.1, 0.05, 0.01))  # 5 modes on 4 nodes
    assert lib.mlqmc_create(C.byref(p), 0, C.byref(h)) == 1


def test_nystrom_modes_rejects_bad_arguments(lib):
    th = np.zeros(4)
    ps = np.zeros(64)
    dp = C.POINTER(C.c_double)
    for args in [(0.75, 0.3, 1.0, 4, 4), (1.5, 0.0, 1.0, 4, 4), (1.5, 0.3, 0.0, 4, 4), (1.5, 0.3, 1.0, 1, 1),
                 (1.5, 0.3, 1.0, 4, 0), (1.5, 0.3, 1.0, 2, 5)]:
        assert lib.mlqmc_nystrom_modes(*args, th.ctypes.data_as(dp), ps.ctypes.data_as(dp)) == 1, args


def test_create_rejects_even_generating_vector(lib):
    z = (C.c_uint32 * 4)(1, 3, 4, 7)
    p = _problem(sampler=1, genvec=C.cast(z, C.POINTER(C.c_uint32)))
    h = C.c_void_p()
    assert lib.mlqmc_create(C.byref(p), 0, C.byref(h)) == 1


@pytest.mark.parametrize("s,m", [(1, 1), (5, 4), (20, 8), (100, 10), (8, 12)])
def test_cbc_matches_oracle(lib, s, m):
    z, e2 = M.cbc_genvec(s, m)
    zo, e2o = O.cbc(s, m)
    if not np.array_equal(z, zo):
        # only a rounding-level tie may differ: equal criteria
        g = np.array([1.0 / (j + 1) ** 2 for j in range(s)])
        assert abs(O.cbc_criterion(z, m, g) - O.cbc_criterion(zo, m, g)) < 1e-13
    assert np.allclose(e2, e2o, rtol=1e-12, atol=(2 ** m) * 2.0 ** -52)


def test_cbc_rejects_bad_sizes(lib):
    g = np.ones(4)
    z = (C.c_uint32 * 4)()
    gp = g.ctypes.data_as(C.POINTER(C.c_double))
    assert lib.mlqmc_cbc_genvec(0, 4, gp, z, None) == 1
    assert lib.mlqmc_cbc_genvec(4, 0, gp, z, None) == 1
    assert lib.mlqmc_cbc_genvec(4, 25, gp, z, None) == 1
