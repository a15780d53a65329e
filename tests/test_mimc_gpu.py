"""Multi-index variant (grid level x V-cycle count) on the GPU against the
oracle, through the C ABI (mlqmc_sample_mixed, mlqmc_estimate_mimc).

Tolerances (FP64 form): per-sample mixed differences within 1e-11 of
|F_t^m| + |F_{t-1}^m| + |F_t^{m-1}| + |F_{t-1}^{m-1}| (the four QoI agree to
1e-12 relative and D cancels them), the sums within 1e-11 of the sum of those
scales over the samples entering them; the estimator's sample counts exactly
(the index choice compares variances that agree to far better than the gaps
between them), Q to 1e-10 relative."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle import mimc

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
M = pytest.importorskip("paper_1806_05619_gb300")

CFG = W.MIMC_4LEVEL
WORK = [(3, 0, 5, 0, 4), (1, 2, 9, 1, 3), (2, 4, 4, 0, 4), (0, 0, 3, 0, 4)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import os
    if not os.path.exists(M.LIB_PATH):
        M.build()
    assert torch.cuda.is_available()


def _genvec(cfg):
    z, _ = M.cbc_genvec(cfg["s"], cfg["log2_nmax"])
    zo, _ = O.cbc(cfg["s"], cfg["log2_nmax"])
    assert np.array_equal(z, zo)
    return z


def _pairs(mus=None, **over):
    cfg = W.scaled(CFG, **over)
    z = _genvec(cfg)
    mus = mus or cfg["mus"]
    ctxs = [M.Context.from_config(cfg, genvec=z, mu0=mu) for mu in mus]
    ors = [O.Oracle(n_levels=cfg["n_levels"], n0=cfg["n0"], s=cfg["s"], sigma=cfg["sigma"],
                    corr_len=cfg["corr_len"], qoi=cfg["qoi"], mu0=mu, nu1=cfg["nu1"], nu2=cfg["nu2"], rtol=0.0,
                    max_cycles=cfg["max_cycles"], sampler="lattice", seed=cfg["seed"], R=cfg["R"], genvec=z,
                    log2_nmax=cfg["log2_nmax"], reuse=cfg["reuse"])
           for mu in mus]
    return cfg, ctxs, ors


def _nsamp(work):
    return sum((ne - nb) * (re_ - rb) for (_, nb, ne, rb, re_) in work)


@pytest.mark.parametrize("reuse", [True, False])
def test_mixed_differences_and_sums_match_the_oracle(reuse):
    cfg, ctxs, ors = _pairs(reuse=reuse)
    nl, R = cfg["n_levels"], cfg["R"]
    for m in range(len(ctxs)):
        lo = ctxs[m - 1] if m else None
        sums = torch.zeros(nl * R * 2, dtype=torch.float64, device="cuda")
        D = torch.full((_nsamp(WORK) * nl,), np.nan, dtype=torch.float64, device="cuda")
        ctxs[m].sample_mixed(lo, WORK, sums, D)
        torch.cuda.synchronize()
        ctxs[m].check_device()
        Do, Fh, Fl = mimc.mixed_differences(ors[m], ors[m - 1] if m else None, WORK)
        so, _ = mimc.mixed_sums(ors[m], ors[m - 1] if m else None, WORK, reuse=reuse)
        Dg = D.cpu().numpy().reshape(-1, nl)
        scale = np.abs(Fh) + np.abs(Fl)
        scale[:, 1:] += np.abs(Fh[:, :-1]) + np.abs(Fl[:, :-1])
        assert np.all(np.abs(Dg - Do) <= 1e-11 * scale + 1e-300), m
        sg = sums.cpu().numpy().reshape(nl, R, 2)
        sc = np.zeros((nl, R))
        for q, (lv, r) in enumerate(mimc.expand(WORK)):
            for t in range(nl):
                if (lv >= t) if reuse else (lv == t):
                    sc[t, r] += scale[q, t]
        assert np.all(np.abs(sg[..., 0] - so[..., 0]) <= 1e-11 * sc + 1e-300), m
        assert np.all(np.abs(sg[..., 1] - so[..., 1]) <= 1e-10 * sc * sc + 1e-300), m


def test_sample_mixed_accumulates_and_skips_empty_work():
    cfg, ctxs, _ = _pairs()
    nl, R = cfg["n_levels"], cfg["R"]
    a = torch.zeros(nl * R * 2, dtype=torch.float64, device="cuda")
    ctxs[1].sample_mixed(ctxs[0], [], a)
    ctxs[1].sample_mixed(ctxs[0], [(2, 0, 0, 0, R)], a)
    torch.cuda.synchronize()
    assert torch.count_nonzero(a).item() == 0
    # two halves accumulate to the whole (same samples, same per-sample values)
    ctxs[1].sample_mixed(ctxs[0], [(2, 0, 3, 0, R)], a)
    ctxs[1].sample_mixed(ctxs[0], [(2, 3, 6, 0, R)], a)
    b = torch.zeros_like(a)
    ctxs[1].sample_mixed(ctxs[0], [(2, 0, 6, 0, R)], b)
    torch.cuda.synchronize()
    assert torch.allclose(a, b, rtol=1e-12, atol=1e-18)


def test_sample_mixed_rejects_incompatible_contexts():
    cfg, ctxs, _ = _pairs()
    nl, R = cfg["n_levels"], cfg["R"]
    sums = torch.zeros(nl * R * 2, dtype=torch.float64, device="cuda")
    z = _genvec(cfg)
    other_seed = M.Context.from_config(cfg, genvec=z, mu0=1, seed=cfg["seed"] + 1)
    for hi, lo in [(ctxs[1], other_seed), (ctxs[0], ctxs[1]), (ctxs[1], ctxs[1])]:
        with pytest.raises(M.MlqmcError) as e:
            hi.sample_mixed(lo, [(1, 0, 2, 0, R)], sums)
        assert e.value.code == 1
    with pytest.raises(M.MlqmcError) as e:
        ctxs[1].sample_mixed(ctxs[0], [(nl, 0, 2, 0, R)], sums)  # level out of range
    assert e.value.code == 1
    with pytest.raises(M.MlqmcError) as e:
        M.estimate_mimc([ctxs[1], ctxs[0]], 1e-3)  # mu0 not increasing
    assert e.value.code == 1


@pytest.mark.parametrize("batched", [False, True])
def test_estimate_matches_the_oracle(batched):
    eps = CFG["eps"][0]
    cfg, ctxs, ors = _pairs()
    r = M.estimate_mimc(ctxs, eps, batched=batched)
    ro = mimc.estimate_mimc(ors, eps, batched=batched)
    assert r["run_status"] == ro["run_status"] == 0
    assert r["L"] == ro["L"] and r["rounds"] == ro["rounds"]
    assert r["N"] == [row[:r["L"] + 1] for row in ro["N"]]
    assert r["Q"] == pytest.approx(ro["Q"], rel=1e-10)
    assert r["varQ"] == pytest.approx(ro["varQ"], rel=1e-6)
    assert r["bias"] == pytest.approx(ro["bias"], rel=1e-6)
    assert r["alpha"] == pytest.approx(ro["alpha"], rel=1e-6)
    assert r["bias_cycles"] == pytest.approx(ro["bias_cycles"], rel=1e-6)
    assert r["varQ"] <= eps * eps / 2


def test_one_cycle_count_is_algorithm_1():
    # K = 1: the multi-index driver is Algorithm 1 of mlqmc_estimate
    eps = CFG["eps"][0]
    cfg, ctxs, _ = _pairs(mus=[2])
    r = M.estimate_mimc(ctxs, eps)
    a = ctxs[0].estimate(eps)
    assert r["L"] == a["L"] and r["rounds"] == a["rounds"] and r["run_status"] == a["run_status"]
    assert r["N"][0] == a["N"][:a["L"] + 1]
    assert r["Q"] == pytest.approx(a["Q"], rel=1e-13)
    assert r["varQ"] == pytest.approx(a["varQ"], rel=1e-11)
    assert r["bias"] == pytest.approx(a["bias"], rel=1e-11)
