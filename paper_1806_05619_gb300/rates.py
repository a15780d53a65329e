"""Rates of assumptions (A1)-(A4) and the cost-reduction factor of Proposition 1
(Sec. 3.3 "Cost analysis"; Sec. 6 "Numerical rate determination"), measured on
the GPU path through the public API.

With the geometric hierarchy h_l = h_0 / 2^l (rho = 2):

* alpha (A1): |E[F_l - F_{l-1}]| decays like 2^(-alpha l);
* beta  (A2): V[F_l - F_{l-1}] decays like 2^(-beta l);
* gamma (A3): the cost of a sample whose FMG ends on level l grows like
  2^(gamma l) (here: device time per sample of a batch of such samples);
* lambda (A4): V[Ybar_l] over the first N = 2^m points of the shifted lattice
  sequence decays like N^(-1/lambda).

Each rate is a least-squares slope of log2 of the values. Proposition 1 then
predicts cost(reuse) / cost(no reuse) = 1 - rho^(-(beta + gamma) lambda / (lambda + 1)),
which comes from N_{l+1} = rho^(-(beta + gamma) lambda / (lambda + 1)) N_l (eq. nopt2):
with recycling only N_l - N_{l+1} new samples are needed on level l.

Host-side arithmetic only (numpy); the samples come from `Context.sample_levels`.
"""
from __future__ import annotations

import numpy as np


def slope(x, y):
    """Least-squares slope of y against x."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    xc = x - x.mean()
    return float(np.dot(xc, y - y.mean()) / np.dot(xc, xc))


def decay_rate(levels, values):
    """r such that |values| ~ 2^(-r * level) (least squares in log2)."""
    return -slope(levels, np.log2(np.abs(np.asarray(values, dtype=np.float64))))


def prop1_ratio(beta, gamma, lam, rho=2.0):
    """Proposition 1: cost(MG-MLQMC) / cost(MLQMC) = 1 - rho^(-(beta + gamma) lambda / (lambda + 1));
    lambda = 1 for Monte Carlo."""
    return 1.0 - rho ** (-(beta + gamma) * lam / (lam + 1.0))


def reuse_cost_ratio(N, C):
    """Cost of the recycling estimator relative to the plain one for the same
    per-level sample counts N_l (samples used on level l) and per-sample
    costs C_l: sum (N_l - N_{l+1}) C_l / sum N_l C_l, as in the proof of
    Proposition 1 (N_{L+1} = 0)."""
    N = np.asarray(N, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    new = N - np.append(N[1:], 0.0)
    return float(np.dot(new, C) / np.dot(N, C))


def differences(F, levels):
    """Per-sample differences F_l - F_{l-1} (F_{-1} = 0) of rows F whose FMG
    ended on `levels` (same order): {level: array}."""
    out = {}
    for row, lv in zip(F, levels):
        d = row[lv] - (row[lv - 1] if lv > 0 else 0.0)
        out.setdefault(int(lv), []).append(d)
    return {k: np.asarray(v) for k, v in out.items()}


def lattice_variance_curve(d, R, m_min=1):
    """V[Ybar] of the first 2^m points per shift, m = m_min..log2(N): d has
    shape (R, N) (shift-major); V[Ybar] = sample variance over shifts of the
    per-shift means, divided by R (eq. sample_variances)."""
    d = np.asarray(d, dtype=np.float64).reshape(R, -1)
    m_max = int(np.log2(d.shape[1]))
    ms = list(range(m_min, m_max + 1))
    v = [float(np.var(d[:, :2 ** m].mean(axis=1), ddof=1) / R) for m in ms]
    return ms, v


def measure(ctx, n_points=256, lambda_level=None, gamma_levels=3, stream=None):
    """Sample every level l with the first `n_points` lattice points of each of
    the context's R shifts (one call per level, the FMG of each sample ending
    on l), then fit the four rates. gamma is fitted over the `gamma_levels`
    finest levels, where the device is busy enough for time to follow work.
    Returns a dict of per-level E, V, cost and the fitted rates."""
    import torch

    L = ctx.n_levels - 1
    R = ctx.R
    E, V, C_ms = [], [], []
    curves = {}
    lam_lv = lambda_level if lambda_level is not None else min(2, L)
    for lv in range(L + 1):
        work = [(lv, 0, n_points, 0, R)]
        ns = n_points * R
        sums = torch.zeros(ctx.n_levels * R * 2, dtype=torch.float64, device="cuda")
        F = torch.zeros(ns * ctx.n_levels, dtype=torch.float64, device="cuda")
        ctx.sample_levels(work, sums, F, stream=stream)  # warm-up (pools, graph)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st = stream if stream is not None else torch.cuda.current_stream()
        e0.record(st)
        ctx.sample_levels(work, sums, F, stream=stream)
        e1.record(st)
        torch.cuda.synchronize()
        ctx.check_device()
        C_ms.append(e0.elapsed_time(e1) / ns)
        Fh = F.cpu().numpy().reshape(ns, ctx.n_levels)
        d = differences(Fh, [lv] * ns)[lv]  # rows r-major: shift r, points 0..n_points-1
        E.append(float(d.mean()))
        V.append(float(d.var(ddof=1)))
        if lv == lam_lv:
            curves[lv] = lattice_variance_curve(d, R)
    lv1 = list(range(1, L + 1))
    alpha = decay_rate(lv1, E[1:])
    beta = decay_rate(lv1, V[1:])
    gl = list(range(L + 1 - gamma_levels, L + 1))
    gamma = -decay_rate(gl, [C_ms[t] for t in gl])
    ms, vy = curves[lam_lv]
    inv_lam = -slope(ms, np.log2(vy))
    lam = 1.0 / inv_lam
    return {"levels": list(range(L + 1)), "E_dF": E, "V_dF": V, "ms_per_sample": C_ms,
            "alpha": alpha, "beta": beta, "gamma": gamma, "gamma_levels": gl,
            "lambda": lam, "lambda_level": lam_lv, "lambda_curve": {"log2_N": ms, "V_Ybar": vy},
            "n_points": n_points, "R": R, "prop1_ratio": prop1_ratio(beta, gamma, lam)}
