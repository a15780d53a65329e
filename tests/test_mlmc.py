"""Plain MLMC, the baseline of the paper's speed-up comparison (Sec. 2: eqs.
MSE, vardecomp, nopt; reading A28). Oracle pins on the CPU, then (GPU) the
library's driver against the oracle's."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W


def _mc_oracle(**over):
    cfg = W.scaled(W.MC_4LEVEL, **over)
    return cfg, O.Oracle(n_levels=cfg["n_levels"], n0=cfg["n0"], s=cfg["s"], sigma=cfg["sigma"],
                         corr_len=cfg["corr_len"], qoi=cfg["qoi"], mu0=cfg["mu0"], nu1=cfg["nu1"],
                         nu2=cfg["nu2"], rtol=0.0, max_cycles=100, sampler="mc", seed=cfg["seed"], R=1,
                         reuse=False)


def test_nopt_closed_forms():
    # one level: plain MC, N = ceil(2 V / eps^2) (values exact in binary)
    assert O.mlmc_nopt([0.25], [4.0], 0.125).tolist() == [32.0]
    assert O.mlmc_nopt([0.25], [9.0], 0.0625).tolist() == [128.0]
    # V = (4, 1), C = (1, 4): sum sqrt(V C) = 4; N_0 = 200 * 2 * 4, N_1 = 200 * 0.5 * 4
    assert O.mlmc_nopt([4.0, 1.0], [1.0, 4.0], 0.1).tolist() == [1600.0, 400.0]
    # before rounding the counts meet the variance budget exactly (eq. vardecomp)
    V, Cc, eps = np.array([2e-3, 3e-4, 5e-5]), np.array([64.0, 320.0, 1344.0]), 1e-3
    lam = np.sum(np.sqrt(V * Cc))
    n_real = 2.0 / eps ** 2 * np.sqrt(V / Cc) * lam
    assert np.sum(V / n_real) == pytest.approx(eps ** 2 / 2, rel=1e-12)
    assert np.array_equal(O.mlmc_nopt(V, Cc, eps), np.ceil(n_real))


def test_single_level_is_plain_monte_carlo():
    cfg, orc = _mc_oracle(n_levels=1)
    eps = 2e-3
    r = orc.estimate_mlmc(eps)
    assert r["status"] == O.OK and r["run_status"] == 7 and r["L"] == 0  # no finer level to test the bias on
    N0 = r["N"][0]
    ref = orc.sample_levels([(0, 0, N0, 0, 1)], want_F=True)
    F0 = ref["F"][:, 0]
    assert r["Q"] == pytest.approx(F0.mean(), rel=1e-13)
    assert r["Vell"][0] == pytest.approx(F0.var(ddof=1), rel=1e-10)
    assert N0 >= max(32, math.ceil(2 * F0.var(ddof=1) / eps ** 2))
    assert r["varQ"] <= eps ** 2 / 2 * (1 + 1e-12)


def test_multilevel_run_invariants_and_bookkeeping():
    cfg, orc = _mc_oracle()
    eps = 3e-3
    r = orc.estimate_mlmc(eps)
    assert r["status"] == O.OK and r["run_status"] == 0
    L = r["L"]
    assert L >= 2 and r["varQ"] <= eps ** 2 / 2 * (1 + 1e-12) and r["bias"] <= eps / math.sqrt(2)
    N = r["N"][:L + 1]
    assert all(n >= 32 for n in N)
    V, Cc = np.array(r["Vell"][:L + 1]), np.array(r["C"][:L + 1])
    assert np.all(np.array(N) >= O.mlmc_nopt(V, Cc, eps))  # every level holds at least its eq. nopt count
    # the estimate is the sum of the level means of independent samples (no recycling)
    Q = 0.0
    for lv in range(L + 1):
        F = orc.sample_levels([(lv, 0, N[lv], 0, 1)], want_F=True)["F"]
        d = F[:, lv] - (F[:, lv - 1] if lv else 0.0)
        assert r["Ybar"][lv] == pytest.approx(d.mean(), rel=1e-10, abs=1e-15)
        Q += d.mean()
    assert r["Q"] == pytest.approx(Q, rel=1e-12)


def test_rejects_lattice_or_recycling():
    cfg = W.scaled(W.LATTICE_6LEVEL, n_levels=3, s=4, R=2, log2_nmax=6)
    z, _ = O.cbc(cfg["s"], cfg["log2_nmax"])
    orc = O.Oracle(n_levels=3, n0=8, s=4, sampler="lattice", seed=1, R=2, genvec=z, log2_nmax=6)
    assert orc.estimate_mlmc(1e-2)["status"] == O.ERR_ARG
    _, orc2 = _mc_oracle(reuse=True)
    orc2 = O.Oracle(n_levels=3, n0=4, s=4, sampler="mc", seed=1, R=1, reuse=True)
    assert orc2.estimate_mlmc(1e-2)["status"] == O.ERR_ARG


@pytest.mark.gpu
@pytest.mark.parametrize("eps", [5e-3, 2e-3])
def test_gpu_mlmc_matches_oracle(eps):
    pytest.importorskip("torch")
    import paper_1806_05619_gb300 as M

    cfg, orc = _mc_oracle()
    cfg = dict(cfg, R=1, reuse=False)
    ctx = M.Context.from_config(cfg)
    g = ctx.estimate_mlmc(eps)
    o = orc.estimate_mlmc(eps)
    assert g["run_status"] == o["run_status"] and g["L"] == o["L"] and g["rounds"] == o["rounds"]
    assert g["N"] == o["N"]
    assert g["Q"] == pytest.approx(o["Q"], rel=1e-10)
    assert g["varQ"] == pytest.approx(o["varQ"], rel=1e-8)
    with pytest.raises(M.MlqmcError):
        M.Context.from_config(dict(cfg, reuse=True)).estimate_mlmc(eps)
