"""mlqmc_fmg_fields_noalloc against the regular path and the oracle.

Some callers cannot call cudaMalloc: plug-ins whose host application owns
all device memory and hands them only their inputs and outputs, and
real-time loops that must not wait on the allocator or risk an allocation
failing mid-run. For them the library has one entry point that allocates
nothing and keeps its scratch in a static device array. These tests give it
KL fields and check the F_t it returns (1e-12 relative, the tolerance of the
other FP64 parity tests), each on two calls in a row with different problem
shapes, so the second call runs over whatever the first left in the shared
scratch: against the regular mlqmc_sample_solution path on the fields a
regular context synthesises, and against the oracle's FMG on the oracle's
own fields.
"""
import ctypes as C
import os

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
M = pytest.importorskip("paper_1806_05619_gb300")


@pytest.fixture(scope="module")
def ctx():
    if not os.path.exists(M.LIB_PATH):
        M.build()
    assert torch.cuda.is_available()
    cfg = W.scaled(W.LATTICE_6LEVEL, n_levels=5, R=8)
    z, _ = O.cbc(cfg["s"], cfg["log2_nmax"])
    return cfg, M.Context.from_config(cfg, genvec=z)


def _fields(cfg, c, level, r, n_begin, count):
    """Per sample, the fields of levels 0..level from the regular context, concatenated."""
    y = c.normals(level, r, n_begin, count)
    per_level = [c.fields(t, y) for t in range(level + 1)]
    return torch.cat(per_level, dim=1).contiguous()


def _noalloc(cfg, n_levels, k, count):
    F = torch.full((count * n_levels,), float("nan"), dtype=torch.float64, device="cuda")
    st = M.lib().mlqmc_fmg_fields_noalloc(cfg["n0"], n_levels, M.QOI[cfg["qoi"]], cfg["mu0"], cfg["nu1"],
                                          cfg["nu2"], count, C.c_void_p(k.data_ptr()), C.c_void_p(F.data_ptr()),
                                          C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, st
    torch.cuda.synchronize()
    return F.view(count, n_levels).cpu().numpy()


def _regular(c, level, r, n_begin, count):
    return np.array([c.sample_solution(level, r, n_begin + i)[1].cpu().numpy() for i in range(count)])


def test_two_calls_match_regular_path(ctx):
    cfg, c = ctx
    # call 1: 20 samples on 5 levels (8x8..128x128), more samples than scratch slots
    k1 = _fields(cfg, c, 4, 3, 11, 20)
    F1 = _noalloc(cfg, 5, k1, 20)
    ref1 = _regular(c, 4, 3, 11, 20)
    assert np.max(np.abs(F1 - ref1) / np.abs(ref1)) < 1e-12
    # call 2: another shape (3 levels) over the scratch the first call left behind
    k2 = _fields(cfg, c, 2, 5, 0, 7)
    F2 = _noalloc(cfg, 3, k2, 7)
    ref2 = _regular(c, 2, 5, 0, 7)
    assert np.max(np.abs(F2 - ref2) / np.abs(ref2)) < 1e-12


def test_two_calls_match_oracle_on_its_fields(ctx):
    cfg, _ = ctx
    z, _ = O.cbc(cfg["s"], cfg["log2_nmax"])
    orc = O.Oracle(n_levels=cfg["n_levels"], n0=cfg["n0"], s=cfg["s"], sigma=cfg["sigma"], corr_len=cfg["corr_len"],
                   qoi=cfg["qoi"], mu0=cfg["mu0"], nu1=cfg["nu1"], nu2=cfg["nu2"], sampler="lattice",
                   seed=cfg["seed"], R=cfg["R"], genvec=z, log2_nmax=cfg["log2_nmax"], reuse=True)
    for level, r, count in [(4, 1, 3), (2, 6, 4)]:
        ks, refs = [], []
        for i in range(count):
            y = orc.normals(level, r, i)
            kl = [orc.field(t, y) for t in range(level + 1)]
            ks.append(np.concatenate(kl))
            ref = orc.fmg_fields(level, kl)
            assert ref["status"] == O.OK
            refs.append(ref["F"])
        k = torch.from_numpy(np.stack(ks)).cuda().contiguous()
        F = _noalloc(cfg, level + 1, k, count)
        ref = np.array(refs)
        assert np.max(np.abs(F - ref) / np.abs(ref)) < 1e-12


def test_rejects_problems_beyond_the_scratch(ctx):
    cfg, c = ctx
    k = torch.zeros(16, dtype=torch.float64, device="cuda")
    F = torch.zeros(16, dtype=torch.float64, device="cuda")
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    # 8 x 2^5 = 256 cells per side is above the 128 limit
    assert M.lib().mlqmc_fmg_fields_noalloc(8, 6, 1, 2, 2, 2, 1, C.c_void_p(k.data_ptr()),
                                            C.c_void_p(F.data_ptr()), s) == 9
    assert M.lib().mlqmc_fmg_fields_noalloc(32, 1, 1, 2, 2, 2, 1, C.c_void_p(k.data_ptr()),
                                            C.c_void_p(F.data_ptr()), s) == 9
    assert M.lib().mlqmc_fmg_fields_noalloc(3, 2, 1, 2, 2, 2, 1, C.c_void_p(k.data_ptr()),
                                            C.c_void_p(F.data_ptr()), s) == 1
