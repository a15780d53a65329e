"""Matern covariance with Nystrom eigenpairs (Sec. 5, eq. matern) on the GPU
path against the numpy oracle: the device eigensolver's eigenvalues and
eigenspaces, the interpolated fields on every level (FP64 to 1e-12, the
tensor-core forms within their rounding bound) and FMG solutions on them."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle import matern as MT
from test_parity_gpu import EXP_SLACK, _rel, _tf32_u

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
M = pytest.importorskip("paper_1806_05619_gb300")


def _kern(nu, lam, sigma):
    return MT.isotropic(lambda r: MT.matern(r, nu, lam, sigma))


def _groups(ev, s, tol=1e-8):
    """Index ranges of eigenvalue clusters among the first s (a cluster cut at s is dropped)."""
    out, start = [], 0
    for i in range(1, len(ev) + 1):
        if i == len(ev) or ev[i - 1] - ev[i] > tol * ev[0]:
            if i <= s:
                out.append((start, i))
            start = i
    return out


@pytest.mark.parametrize("nu", [0.5, 1.0, 1.5, 2.0, 2.5])
def test_nystrom_modes_match_oracle(nu):
    m, s, lam, sigma = 16, 40, 0.3, 1.2
    th, ps = M.nystrom_modes(nu, lam, sigma, m, s)
    tho, pso, ev = MT.nystrom(m, s, _kern(nu, lam, sigma))
    assert np.max(np.abs(th - tho) / tho) < 1e-11
    w = 1.0 / m ** 2
    # eigenspaces are unique (bases within a repeated eigenvalue and signs are not): compare projectors
    for a, b in _groups(ev, s):
        Pg = w * ps[:, a:b] @ ps[:, a:b].T
        Po = w * pso[:, a:b] @ pso[:, a:b].T
        assert np.max(np.abs(Pg - Po)) < 1e-9, (a, b)
    # the returned vectors are eigenvectors of the discrete equation, orthonormal in the weighted sum
    x1, x2, _ = MT.nodes(m)
    B = w * _kern(nu, lam, sigma)(x1[:, None] - x1[None, :], x2[:, None] - x2[None, :])
    assert np.max(np.abs(B @ ps - ps * th[None, :])) < 1e-12 * sigma ** 2 * np.abs(ps).max()
    assert np.allclose(w * ps.T @ ps, np.eye(s), atol=1e-12)


def _ctx(precision, nu, m, s, theta, psi, **over):
    cfg = W.scaled(W.LATTICE_6LEVEL, n_levels=4, s=s, R=2, precision=precision, log2_nmax=8, corr_len=0.3)
    cfg.update(over)
    z, _ = M.cbc_genvec(cfg["s"], cfg["log2_nmax"])
    ctx = M.Context.from_config(cfg, genvec=z, covariance="matern", matern_nu=nu, nystrom_m=m, nystrom_theta=theta,
                                nystrom_psi=psi)
    return cfg, z, ctx


@pytest.mark.parametrize("nu", [0.5, 1.0, 2.0, 2.5])
def test_fields_fp64_match_oracle(nu):
    m, s = 16, 30
    k = _kern(nu, 0.3, 1.0)
    theta, psi, _ = MT.nystrom(m, s, k)
    cfg, _, ctx = _ctx("fp64", nu, m, s, theta, psi)
    Y = W.random_normals(s, 3, tag=60)
    for t in range(cfg["n_levels"]):
        n = cfg["n0"] << t
        kg = ctx.fields(t, torch.from_numpy(Y)).cpu().numpy()
        for i in range(3):
            assert _rel(kg[i], MT.field(n, m, theta, psi, k, Y[i])) < 1e-12, (t, i)


def test_fields_tensor_core_within_bound():
    nu, m, s = 1.5, 16, 30
    k = _kern(nu, 0.3, 1.0)
    theta, psi, _ = MT.nystrom(m, s, k)
    cfg, _, ctx = _ctx("mixed_tf32", nu, m, s, theta, psi)
    Y = W.random_normals(s, 3, tag=61)
    for t in range(cfg["n_levels"]):
        n = cfg["n0"] << t
        P = MT.interpolate(n, m, theta, psi, k)
        kg = ctx.fields(t, torch.from_numpy(Y)).cpu().numpy()
        for i in range(3):
            want = np.exp(P @ (np.sqrt(theta) * Y[i]))
            eta = _tf32_u(s) * np.sum(np.abs(np.sqrt(theta) * Y[i]) * np.abs(P).max(axis=0))
            assert np.max(np.abs(np.log(kg[i] / want))) <= eta + EXP_SLACK, (t, i)


def test_fmg_solutions_fp64_match_oracle():
    nu, m, s = 1.5, 16, 30
    k = _kern(nu, 0.3, 1.0)
    theta, psi, _ = MT.nystrom(m, s, k)
    cfg, z, ctx = _ctx("fp64", nu, m, s, theta, psi)
    work = [(3, 0, 2, 0, 2), (1, 3, 5, 1, 2)]
    nl = cfg["n_levels"]
    ns = sum((ne - nb) * (re_ - rb) for (_, nb, ne, rb, re_) in work)
    sums = torch.zeros(nl * cfg["R"] * 2, dtype=torch.float64, device="cuda")
    F = torch.zeros(ns * nl, dtype=torch.float64, device="cuda")
    ctx.sample_levels(work, sums, F)
    torch.cuda.synchronize()
    ctx.check_device()
    Fg = F.cpu().numpy().reshape(ns, nl)
    orc = O.Oracle(n_levels=nl, n0=cfg["n0"], s=s, qoi=cfg["qoi"], mu0=cfg["mu0"], nu1=cfg["nu1"], nu2=cfg["nu2"],
                   rtol=0.0, sampler="lattice", seed=cfg["seed"], R=cfg["R"], genvec=z, log2_nmax=cfg["log2_nmax"])
    q = 0
    for (lv, nb, ne, rb, re_) in work:
        for r in range(rb, re_):
            for n in range(nb, ne):
                y = orc.normals(lv, r, n)
                ks = [MT.field(cfg["n0"] << t, m, theta, psi, k, y) for t in range(lv + 1)]
                ref = orc.fmg_fields(lv, ks)
                assert ref["status"] == O.OK
                assert _rel(Fg[q, :lv + 1], ref["F"]) < 1e-12, (lv, r, n)
                q += 1
    assert np.all(np.isfinite(sums.cpu().numpy()))


def test_mixed_forms_run_and_reject_bad_input():
    nu, m, s = 0.5, 12, 20
    theta, psi = M.nystrom_modes(nu, 0.3, 1.0, m, s)
    for prec in ("mixed_tf32", "mixed_bf16x3"):
        cfg, _, ctx = _ctx(prec, nu, m, s, theta, psi)
        F = torch.zeros(4 * cfg["n_levels"], dtype=torch.float64, device="cuda")
        sums = torch.zeros(cfg["n_levels"] * cfg["R"] * 2, dtype=torch.float64, device="cuda")
        ctx.sample_levels([(3, 0, 2, 0, 2)], sums, F)
        torch.cuda.synchronize()
        ctx.check_device()
        Fh = F.cpu().numpy()
        assert np.all(np.isfinite(Fh)) and np.all(Fh > 0)
    with pytest.raises(M.MlqmcError):
        _ctx("fp64", 0.75, m, s, theta, psi)  # nu outside {1/2, 1, 3/2, 2, 5/2}
    with pytest.raises(M.MlqmcError):
        _ctx("fp64", nu, m, s, -theta, psi)
    with pytest.raises(M.MlqmcError):
        M.nystrom_modes(3.0, 0.3, 1.0, m, s)
