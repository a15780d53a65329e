"""Multi-index variant (grid level x V-cycle count; the outlook of Sec. 7) on
the oracle: pins of the mixed differences and of the estimator against
identities of the construction and the V-cycle contraction.

D_{t,m} = [F_t^m - F_{t-1}^m] - [F_t^{m-1} - F_{t-1}^{m-1}] for one sample y,
F^m the FMG QoI with mu_m cycles per level."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle import mimc

CFG = W.MIMC_4LEVEL


def _oracles(mus=None, **over):
    cfg = W.scaled(CFG, **over)
    z, _ = O.cbc(cfg["s"], cfg["log2_nmax"])
    return [O.Oracle(n_levels=cfg["n_levels"], n0=cfg["n0"], s=cfg["s"], sigma=cfg["sigma"],
                     corr_len=cfg["corr_len"], qoi=cfg["qoi"], mu0=mu, nu1=cfg["nu1"], nu2=cfg["nu2"],
                     rtol=0.0, max_cycles=cfg["max_cycles"], sampler="lattice", seed=cfg["seed"], R=cfg["R"],
                     genvec=z, log2_nmax=cfg["log2_nmax"], reuse=cfg["reuse"])
            for mu in (mus or cfg["mus"])]


# ragged work: several items, a partial shift range, an empty item
WORK = [(3, 0, 5, 0, 4), (1, 2, 9, 1, 3), (2, 4, 4, 0, 4), (0, 0, 3, 0, 4)]


def test_first_direction_is_the_level_difference():
    # m = 0 (no coarser cycle count): the sums are those of MG-MLQMC (eq. Upsilon-reuse)
    os_ = _oracles()
    s0, _ = mimc.mixed_sums(os_[0], None, WORK)
    ref = os_[0].sample_levels(WORK)["sums"]
    assert np.allclose(s0, ref, rtol=1e-14, atol=1e-16)


def test_telescoping_to_the_largest_cycle_count():
    # per sample: sum over m and t <= level of D_{t,m} = F_level with the largest mu
    os_ = _oracles()
    K = len(os_)
    Ds = [mimc.mixed_differences(os_[m], os_[m - 1] if m else None, WORK)[0] for m in range(K)]
    F = os_[-1].sample_levels(WORK, want_F=True)["F"]
    for q, (lv, _r) in enumerate(mimc.expand(WORK)):
        tot = sum(Ds[m][q, :lv + 1].sum() for m in range(K))
        assert abs(tot - F[q, lv]) <= 1e-15 * max(1.0, abs(F[q, lv]))
        assert np.all(Ds[0][q, lv + 1:] == 0.0)


def test_equal_counts_reduce_to_mlqmc_of_the_largest_cycle_count():
    # with the same samples in every direction the sums over m are the MG-MLQMC
    # sums of the largest mu: the multi-index estimator is then that estimator
    os_ = _oracles()
    tot = sum(mimc.mixed_sums(os_[m], os_[m - 1] if m else None, WORK)[0] for m in range(len(os_)))
    ref = os_[-1].sample_levels(WORK)["sums"]
    assert np.allclose(tot[..., 0], ref[..., 0], rtol=0, atol=1e-15)


def test_cycle_direction_contracts_like_the_v_cycle():
    # near k = 1 (sigma 0.1) one more V(2,2) cycle shrinks the solver error by
    # the V-cycle contraction factor (< 0.2 at k = 1), so D_{t,m+1} <= 0.2 D_{t,m}
    # in RMS for m >= 1; a sign error in the second bracket of D would make
    # D_{t,1} about twice the level difference and fail this
    os_ = _oracles(sigma=0.1)
    work = [(3, 0, 8, 0, 4)]
    rms = []
    for m in range(len(os_)):
        D, _, _ = mimc.mixed_differences(os_[m], os_[m - 1] if m else None, work)
        rms.append(np.sqrt((D ** 2).mean(axis=0)))
    rms = np.array(rms)
    for t in range(1, 4):
        assert rms[1, t] > 0 and rms[2, t] <= 0.2 * rms[1, t]
    # the first cycle direction is far below the level difference itself
    assert np.all(rms[1, 1:] < 0.2 * rms[0, 1:])


def test_estimator_from_replicates():
    # Q is the sum of the per-index means; varQ the variance of the mean of the
    # R replicate estimators (brute force with numpy)
    rng = np.random.default_rng(5)
    L, K, R = 2, 2, 5
    N = [[3, 2, 1], [2, 1, 1]]
    sums = [rng.standard_normal((L + 1, R, 2)) for _ in range(K)]
    e = mimc.finalize(L, K, R, True, N, sums)
    Qr = np.zeros(R)
    for m in range(K):
        for t in range(L + 1):
            Qr += sums[m][t, :, 0] / sum(N[m][t:])
    assert e["Q"] == pytest.approx(Qr.mean(), rel=1e-14)
    assert e["varQ"] == pytest.approx(np.var(Qr, ddof=1) / R, rel=1e-12)
    assert e["Q"] == pytest.approx(e["Ybar"].sum(), rel=1e-13)


def test_single_cycle_count_is_algorithm_1():
    # K = 1: the index set is the levels and D_{t,0} the level differences, so
    # the driver is Algorithm 1 (the C oracle's): same levels, counts, rounds
    eps = CFG["eps"][0]
    for mu in (1, 2):
        (o,) = _oracles(mus=[mu])
        r = mimc.estimate_mimc([o], eps)
        ref = o.estimate(eps)
        assert ref["status"] == O.OK
        assert r["L"] == ref["L"] and r["rounds"] == ref["rounds"] and r["run_status"] == ref["run_status"]
        assert r["N"][0] == ref["N"]
        assert r["Q"] == pytest.approx(ref["Q"], rel=1e-13)
        assert r["varQ"] == pytest.approx(ref["varQ"], rel=1e-11)
        assert r["bias"] == pytest.approx(ref["bias"], rel=1e-11)
        assert r["alpha"] == pytest.approx(ref["alpha"], rel=1e-11)


def test_estimate_agrees_with_mlqmc_of_the_largest_cycle_count():
    eps = CFG["eps"][0]
    os_ = _oracles()
    r = mimc.estimate_mimc(os_, eps)
    assert r["run_status"] == 0 and r["varQ"] <= eps * eps / 2 and r["bias"] <= eps / np.sqrt(2)
    ref = os_[-1].estimate(eps)
    assert ref["status"] == O.OK
    assert abs(r["Q"] - ref["Q"]) <= 4.0 * np.sqrt(r["varQ"] + ref["varQ"])
    # the cheap direction carries the samples: every index up to L was sampled,
    # and the cycle directions need far fewer points than the level differences
    N = np.array(r["N"])[:, :r["L"] + 1]
    assert np.all(N > 0) and np.all(np.array(r["N"])[:, r["L"] + 1:] == 0)
    assert N[1:].sum() * 10 <= N[0].sum()
    assert r["bias_cycles"] < r["bias"]
