"""Rates of (A1)-(A4) and Proposition 1's cost-reduction factor: the host-side
fitting (no GPU) pinned on closed forms, and (GPU) the measured per-level
statistics against the oracle's samples."""
import math

import numpy as np
import pytest

from paper_1806_05619_gb300 import rates


def test_slopes_recover_exact_rates():
    lv = np.arange(1, 7)
    assert rates.decay_rate(lv, 3.0 * 2.0 ** (-1.7 * lv)) == pytest.approx(1.7, abs=1e-12)
    assert rates.decay_rate(lv, -0.5 * 2.0 ** (-2.0 * lv)) == pytest.approx(2.0, abs=1e-12)  # sign ignored
    assert rates.slope([0, 1, 2], [1.0, 3.0, 5.0]) == pytest.approx(2.0, abs=1e-15)


def test_prop1_closed_forms():
    # beta = gamma = 2, Monte Carlo (lambda = 1): 1 - 2^-2
    assert rates.prop1_ratio(2.0, 2.0, 1.0) == 0.75
    # QMC rate 1/lambda = 2: exponent (beta + gamma) / 3
    assert rates.prop1_ratio(2.0, 2.0, 0.5) == pytest.approx(1.0 - 2.0 ** (-4.0 / 3.0), rel=1e-15)
    # lambda -> infinity: 1 - rho^-(beta + gamma); rho = 4
    assert rates.prop1_ratio(1.0, 1.0, 1e12, rho=4.0) == pytest.approx(1.0 - 4.0 ** -2.0, rel=1e-9)
    # faster variance decay -> less to gain from recycling
    assert rates.prop1_ratio(4.0, 2.0, 1.0) > rates.prop1_ratio(2.0, 2.0, 1.0)


def test_reuse_cost_ratio_matches_prop1_for_the_optimal_counts():
    beta, gamma, lam = 4.0, 2.0, 1.0
    q = 2.0 ** (-(beta + gamma) * lam / (lam + 1.0))
    L = 60
    N = [q ** l for l in range(L + 1)]          # eq. nopt2: N_{l+1} = q N_l
    C = [2.0 ** (gamma * l) for l in range(L + 1)]
    # every level below L needs (1 - q) N_l new samples; the top level's own term is 2^-60 of the total
    assert rates.reuse_cost_ratio(N, C) == pytest.approx(rates.prop1_ratio(beta, gamma, lam), rel=1e-12)
    assert rates.reuse_cost_ratio([5, 0, 0], [1, 4, 16]) == 1.0
    assert rates.reuse_cost_ratio([4, 2, 1], [1, 1, 1]) == pytest.approx(4.0 / 7.0)


def test_lattice_variance_curve_by_hand():
    d = np.array([[1.0, 3.0, 5.0, 7.0], [2.0, 2.0, 2.0, 2.0]])
    ms, v = rates.lattice_variance_curve(d, R=2)
    assert ms == [1, 2]
    # m = 1: shift means (2, 2) -> 0; m = 2: (4, 2) -> sample variance 2, over R = 2 -> 1
    assert v == [0.0, 1.0]


def test_differences_telescope():
    F = np.array([[1.0, 1.5, 0.0], [2.0, 0.0, 0.0], [1.0, 2.0, 2.5]])
    d = rates.differences(F, [1, 0, 2])
    assert d[1].tolist() == [0.5] and d[0].tolist() == [2.0] and d[2].tolist() == [0.5]


@pytest.mark.gpu
def test_measured_statistics_match_oracle_and_rates_are_plausible():
    torch = pytest.importorskip("torch")
    import oracle as O
    import workloads as W
    import paper_1806_05619_gb300 as M

    cfg = W.scaled(W.LATTICE_6LEVEL, n_levels=5, s=20, R=8, log2_nmax=10)
    z, _ = M.cbc_genvec(cfg["s"], cfg["log2_nmax"])
    ctx = M.Context.from_config(cfg, genvec=z)
    r = rates.measure(ctx, n_points=64, lambda_level=2, gamma_levels=3)
    orc = O.Oracle(n_levels=cfg["n_levels"], n0=cfg["n0"], s=cfg["s"], sigma=cfg["sigma"],
                   corr_len=cfg["corr_len"], qoi=cfg["qoi"], mu0=2, nu1=2, nu2=2, rtol=0.0, max_cycles=100,
                   sampler="lattice", seed=cfg["seed"], R=cfg["R"], genvec=z, log2_nmax=cfg["log2_nmax"])
    for lv in (1, 3):
        ref = orc.sample_levels([(lv, 0, 64, 0, cfg["R"])], want_F=True)
        d = rates.differences(ref["F"], [lv] * ref["F"].shape[0])[lv]
        # each F is within 1e-12 of the oracle's, the difference carries that of |F_l| + |F_{l-1}|
        mag = float(np.mean(np.abs(ref["F"][:, lv]) + np.abs(ref["F"][:, lv - 1])))
        assert abs(r["E_dF"][lv] - d.mean()) <= 1e-12 * mag
        assert abs(r["V_dF"][lv] - d.var(ddof=1)) <= 4e-12 * mag * math.sqrt(d.var(ddof=1)) + 1e-300
    assert r["beta"] > 1.0 and r["alpha"] > 0.5
    assert 0.5 < r["gamma"] < 3.0
    assert 0.2 < r["lambda"] < 1.5
    assert 0.0 < r["prop1_ratio"] < 1.0
    assert all(math.isfinite(v) for v in r["ms_per_sample"])
