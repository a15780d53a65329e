"""Oracle for the multi-index variant: grid level x number of V-cycles (the
outlook of Sec. 7, multi-index Monte Carlo with the multigrid cycle count as a
second refinement direction), built on the oracle's FMG solves. Plain numpy in
FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): only ``tests/`` may
import it.

Index (t, m): grid level t; cycle count mu_m, the mu0 of the m-th ``Oracle``
(strictly increasing in m). For one sample y whose FMG ends at level k,
    D_{t,m}(y) = [F_t^m(y) - F_{t-1}^m(y)] - [F_t^{m-1}(y) - F_{t-1}^{m-1}(y)],
t = 0..k, with F_{-1} = 0 and F^{-1} = 0 (so D_{t,0} is the level difference
of MG-MLQMC). The differences of every t <= k are recycled as in eq.
Upsilon-reuse; per index the estimator is that of eqs. Upsilon-reuse-bar and
sample_variances, and the variance of the sum over the index set comes from
the R shift replicates of the whole estimator (eq. var_of_mgmlqmc).
"""
from __future__ import annotations

import numpy as np


def expand(work):
    """(level, r) of every sample of a work list, in work order: item by item,
    then r, then n."""
    out = []
    for (lv, nb, ne, rb, re_) in work:
        for r in range(rb, re_):
            for _ in range(nb, ne):
                out.append((lv, r))
    return out


def mixed_differences(o_hi, o_lo, work):
    """Per-sample D_{t,m} (rows in work order, zeros above the sample's level)
    from the FMG QoI of the same samples by ``o_hi`` and ``o_lo`` (``o_lo`` None:
    the first direction)."""
    Fh = o_hi.sample_levels(work, want_F=True)["F"]
    Fl = o_lo.sample_levels(work, want_F=True)["F"] if o_lo is not None else np.zeros_like(Fh)
    desc = expand(work)
    D = np.zeros_like(Fh)
    for q, (lv, _r) in enumerate(desc):
        for t in range(lv + 1):
            hi = Fh[q, t] - (Fh[q, t - 1] if t > 0 else 0.0)
            lo = Fl[q, t] - (Fl[q, t - 1] if t > 0 else 0.0)
            D[q, t] = hi - lo
    return D, Fh, Fl


def mixed_sums(o_hi, o_lo, work, reuse=True):
    """sums[t][r] = (sum of D_{t,m}, sum of D_{t,m}^2) over the samples of shift r
    whose FMG level is >= t (recycling) or == t."""
    D, _, _ = mixed_differences(o_hi, o_lo, work)
    L1, R = o_hi.n_levels, o_hi.R
    sums = np.zeros((L1, R, 2))
    for q, (lv, r) in enumerate(expand(work)):
        for t in range(L1):
            if (lv >= t) if reuse else (lv == t):
                sums[t, r, 0] += D[q, t]
                sums[t, r, 1] += D[q, t] ** 2
    return sums, D


def finalize(L, K, R, reuse, N, sums):
    """Estimates from the per-direction sums: N[m][t] samples whose FMG ended at
    level t in direction m, sums[m][t][r][0] the sum of D_{t,m} of shift r."""
    Ybar = np.zeros((K, L + 1))
    V = np.zeros((K, L + 1))
    Qr = np.zeros(R)
    for m in range(K):
        for t in range(L + 1):
            cnt = sum(N[m][t:L + 1]) if reuse else N[m][t]
            U = np.array([sums[m][t][r][0] / cnt if cnt > 0 else 0.0 for r in range(R)])
            Qr += U
            Ybar[m, t] = U.mean()
            V[m, t] = ((U - U.mean()) ** 2).sum() / (R * (R - 1)) if R > 1 else np.inf
    Q = Qr.mean()
    varQ = ((Qr - Q) ** 2).sum() / (R * (R - 1)) if R > 1 else np.inf
    return dict(Q=Q, varQ=varQ, Ybar=Ybar, V=V, Qr=Qr)


def _fit_alpha(yl):
    """Least-squares rate of |Ybar_l| over l = 1..L (non-finite logs skipped),
    0.5 and flagged when not positive (readings A14 and A15)."""
    pts = [(l, np.log2(abs(yl[l]))) for l in range(1, len(yl))]
    pts = [(x, y) for (x, y) in pts if np.isfinite(y)]
    a = np.nan
    if len(pts) >= 2:
        x = np.array([p[0] for p in pts], dtype=np.float64)
        y = np.array([p[1] for p in pts])
        n = len(pts)
        a = -(n * (x * y).sum() - x.sum() * y.sum()) / (n * (x * x).sum() - x.sum() ** 2)
    if not a > 0.0:
        return 0.5, True
    return a, False


def estimate_mimc(oracles, eps, max_rounds=1000, batched=False):
    """Algorithm 1 with the level direction adaptive and the cycle direction
    complete: levels are added one at a time from L = 0; for the index set
    {0..L} x {0..K-1} each round doubles N_{t,m} (0 -> 1) of the index with the
    largest V/C (unsampled first; ties -> smallest m, then t; ``batched``: every
    index with at least half the largest ratio) until varQ <= eps^2/2; then, for
    L >= 2, the bias |Ybar_L| / (2^alpha + 1) of the level differences
    Ybar_l = sum_m Ybar_{l,m} decides between stopping and adding a level.
    C_{t,m} = (sum_{t'<=t} n_t'^2) (mu_m + mu_{m-1}), mu_{-1} = 0. The cycle
    direction's indicator is sum_t |Ybar_{t,K-1}|."""
    K = len(oracles)
    Lmax = oracles[0].n_levels - 1
    R = oracles[0].R
    reuse = oracles[0].reuse
    n0 = oracles[0].n0
    mus = [o.p.mu0 for o in oracles]
    cells = [sum((n0 << s) ** 2 for s in range(t + 1)) for t in range(Lmax + 1)]
    Cst = [[cells[t] * (mus[m] + (mus[m - 1] if m > 0 else 0)) for t in range(Lmax + 1)] for m in range(K)]
    N = [[0] * (Lmax + 1) for _ in range(K)]
    V = [[np.inf] * (Lmax + 1) for _ in range(K)]
    Ybar = [[0.0] * (Lmax + 1) for _ in range(K)]
    sums = [np.zeros((Lmax + 1, R, 2)) for _ in range(K)]
    rounds, run_status, L = 0, 0, -1
    Q, varQ, bias, alpha, clamped = 0.0, np.inf, np.inf, np.nan, False

    def unsampled(Lc):
        return any(np.isinf(V[m][t]) for m in range(K) for t in range(Lc + 1))

    def level_mean(l):
        return sum(Ybar[m][l] for m in range(K))

    done = False
    while not done:
        if L >= 2:
            alpha, clamped = _fit_alpha([level_mean(l) for l in range(L + 1)])
            bias = abs(level_mean(L)) / (2.0 ** alpha + 1.0)
            if not bias > eps / np.sqrt(2.0):
                break
        if L + 1 > Lmax:
            run_status = 7
            break
        L += 1
        while True:
            varQ = np.inf
            if not unsampled(L):
                e = finalize(L, K, R, reuse, N, sums)
                Q, varQ = e["Q"], e["varQ"]
            if not varQ > eps * eps / 2.0:
                break
            if rounds >= max_rounds:
                run_status = 8
                done = True
                break
            ratio = [[np.inf if np.isinf(V[m][t]) else V[m][t] / Cst[m][t] for t in range(L + 1)] for m in range(K)]
            best = max(max(row) for row in ratio)
            pick = []
            for m in range(K):
                for t in range(L + 1):
                    if batched:
                        take = np.isinf(ratio[m][t]) if np.isinf(best) else ratio[m][t] >= 0.5 * best
                    else:
                        take = ratio[m][t] == best and not pick
                    if take:
                        pick.append((m, t))
            for m in range(K):
                work = []
                for (mm, t) in pick:
                    if mm != m:
                        continue
                    old = N[m][t]
                    N[m][t] = 2 * old if old > 0 else 1
                    work.append((t, old, N[m][t], 0, R))
                if work:
                    s, _ = mixed_sums(oracles[m], oracles[m - 1] if m > 0 else None, work, reuse)
                    sums[m] += s
            e = finalize(L, K, R, reuse, N, sums)
            for m in range(K):
                for t in range(L + 1):
                    cnt = sum(N[m][t:L + 1]) if reuse else N[m][t]
                    if cnt > 0:
                        V[m][t] = e["V"][m, t]
                        Ybar[m][t] = e["Ybar"][m, t]
            rounds += 1
    bias_cycles = np.inf
    if L >= 0 and not unsampled(L):
        e = finalize(L, K, R, reuse, N, sums)
        Q, varQ = e["Q"], e["varQ"]
        bias_cycles = float(sum(abs(e["Ybar"][K - 1, t]) for t in range(L + 1)))
    return dict(Q=Q, varQ=varQ, bias=bias, alpha=alpha, alpha_clamped=clamped, bias_cycles=bias_cycles, N=N,
                rounds=rounds, run_status=run_status, L=L, K=K)
