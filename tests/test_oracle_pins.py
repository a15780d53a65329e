"""Pins of the oracle against what the paper and the mathematics fix.

None of these checks retypes the oracle's formula: each uses another route
(library routine, closed form, Mercer/trace identities, series solutions,
dual-lattice sums, brute force) so that a dropped term, a wrong sign or index,
or a transposed operand in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sps
import scipy.special as spc

import oracle as O
import workloads as W

# --------------------------------------------------------------------------- #
# Philox (Salmon et al. SC'11): no printed vectors in the paper; pinned by     #
# statistics and by its structure as a permutation of counters.               #
# --------------------------------------------------------------------------- #


def test_philox_uniform_and_avalanche():
    outs = []
    for i in range(4096):
        outs += O.philox4x32_10([i, 0, 0, 0], [1234, 5678])
    v = np.array(outs, dtype=np.uint64)
    # chi-square on the top 6 bits of 16384 words, 64 bins
    counts = np.bincount((v >> np.uint64(26)).astype(np.int64), minlength=64)
    exp = v.size / 64
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 120.0  # 63 dof, p ~ 1e-5
    # bit balance
    bits = np.unpackbits(v.astype(">u4").view(np.uint8))
    assert abs(bits.mean() - 0.5) < 0.01
    # flipping one counter bit changes about half the output bits
    base = O.philox4x32_10([7, 8, 9, 10], [1, 2])
    flips = []
    for b in range(32):
        o = O.philox4x32_10([7 ^ (1 << b), 8, 9, 10], [1, 2])
        flips.append(sum(bin(x ^ y).count("1") for x, y in zip(base, o)))
    assert 48 < np.mean(flips) < 80
    # distinct counters give distinct blocks (a permutation for a fixed key)
    seen = {tuple(O.philox4x32_10([i, 3, 0, 0], [9, 9])) for i in range(2000)}
    assert len(seen) == 2000


def test_philox_known_answer_vectors():
    # the generator's published known-answer vectors (tests/golden, cited there):
    # a wrong multiplier, a swapped word or a missed key bump changes every block
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for row in rows:
        w = [int(x, 16) for x in row]
        assert list(O.philox4x32_10(w[0:4], w[4:6])) == w[6:10]


def test_unit_map_open_interval():
    assert O.u64_to_unit(0) == 0.5 * 2.0 ** -53
    assert O.u64_to_unit(2 ** 64 - 1) == 1.0 - 0.5 * 2.0 ** -53
    assert 0.0 < O.u64_to_unit(2 ** 63) < 1.0
    assert O.u64_to_unit(2 ** 63) == 0.5 + 0.5 * 2.0 ** -53


# --------------------------------------------------------------------------- #
# Phi^{-1} (Sec. 3.2) against scipy's ndtri (a library routine)               #
# --------------------------------------------------------------------------- #


def test_ppnd16_against_ndtri():
    p = np.concatenate([np.linspace(1e-6, 1 - 1e-6, 4001), np.logspace(-300, -1, 300),
                        1 - np.logspace(-16, -1, 100), [0.075, 0.925, 0.5]])
    y = O.ppnd16(p)
    ref = spc.ndtri(p)
    rel = np.abs(y - ref) / np.maximum(np.abs(ref), 1e-300)
    assert rel.max() < 2e-15
    # Phi(Phi^{-1}(p)) = p and symmetry
    q = np.linspace(0.001, 0.999, 999)
    assert np.max(np.abs(spc.ndtr(O.ppnd16(q)) - q)) < 1e-15
    assert np.max(np.abs(O.ppnd16(q) + O.ppnd16(1 - q))) < 1e-13


# --------------------------------------------------------------------------- #
# Lattice sequence (Sec. 3.2 rank-1 rule, Sec. 6 lattice sequence)            #
# --------------------------------------------------------------------------- #


def test_bitrev32_bruteforce():
    r = W.rng(1)
    for v in list(r.integers(0, 2 ** 32, 200)) + [0, 1, 2 ** 31, 2 ** 32 - 1]:
        s = format(int(v), "032b")
        assert O.bitrev32(int(v)) == int(s[::-1], 2)


@pytest.mark.parametrize("m", [1, 4, 7])
def test_first_2m_points_are_the_rule(m):
    N = 2 ** m
    z = [1, 3, 5, 7, 11, 13, N - 1 if N > 1 else 1]
    for zj in z:
        pts = sorted((O.lattice_bits(zj, n, 0) >> 32) for n in range(N))
        rule = sorted(((k * zj) % N) << (32 - m) for k in range(N))
        assert pts == rule
        if zj % 2 == 1:  # odd z: a permutation of {0..N-1}/N
            assert sorted(p >> (32 - m) for p in pts) == list(range(N))


def test_shifted_point_is_fractional_part():
    r = W.rng(2)
    for _ in range(200):
        zj = int(r.integers(1, 2 ** 20)) | 1
        n = int(r.integers(0, 2 ** 20))
        S = int(r.integers(0, 2 ** 63)) * 2 + int(r.integers(0, 2))
        u = O.u64_to_unit(O.lattice_bits(zj, n, S))
        phi = O.bitrev32(n) / 2 ** 32
        want = (phi * zj + S / 2 ** 64) % 1.0
        d = abs(u - want)
        assert min(d, 1 - d) < 1e-9


def test_shifts_distinct_per_level_and_shift():
    seen = set()
    for lv in range(3):
        for r in range(4):
            seen.add(tuple(O.shift_bits(5, lv, r, j) for j in range(6)))
    assert len(seen) == 12


# --------------------------------------------------------------------------- #
# KL eigenpairs (eq. inteq, closed form for the exponential kernel)           #
# --------------------------------------------------------------------------- #


@pytest.mark.parametrize("lam", [0.05, 0.1, 0.3, 1.0])
def test_kl1d_trace_identity(lam):
    K = 20000
    w, th, nr = O.kl1d(lam, K)
    c = 1.0 / lam
    # sum of eigenvalues = integral of C(x,x) over [0,1] = 1; tail ~ 2c/(pi^2 K)
    tail = 2 * c / (math.pi ** 2 * K)
    assert abs(th.sum() + tail - 1.0) < 5e-6 * max(1.0, c)
    assert np.all(np.diff(th) < 0)
    # roots lie one per interval (k pi, (k+1) pi)
    k = np.arange(K)
    assert np.all(w > k * math.pi) and np.all(w < (k + 1) * math.pi)


def test_kl1d_mercer_expansion():
    lam = 0.3
    K = 40000
    w, th, nr = O.kl1d(lam, K)
    c = 1.0 / lam
    for x, xp in [(0.1, 0.7), (0.5, 0.5), (0.03, 0.04), (0.9, 0.2)]:
        px = (w * np.cos(w * x) + c * np.sin(w * x)) / np.sqrt(nr)
        pxp = (w * np.cos(w * xp) + c * np.sin(w * xp)) / np.sqrt(nr)
        # Mercer: sum theta_k psi_k(x) psi_k(x') = exp(-|x-x'|/lambda)
        got = np.sum(th * px * pxp)
        assert abs(got - math.exp(-abs(x - xp) / lam)) < 2e-4
        # the oracle's psi evaluation gives the same eigenfunction values
        assert abs(O.psi1d(w[3], lam, nr[3], x)[0] - px[3]) < 1e-14


def test_kl1d_orthonormal_and_integral_equation():
    lam = 0.3
    K = 12
    w, th, nr = O.kl1d(lam, K)
    xg, wg = np.polynomial.legendre.leggauss(200)
    x = 0.5 * (xg + 1)
    wq = 0.5 * wg
    psi = np.array([O.psi1d(w[k], lam, nr[k], x) for k in range(K)])
    G = (psi * wq) @ psi.T
    assert np.max(np.abs(G - np.eye(K))) < 1e-12
    # integral equation int C(x,x') psi(x') dx' = theta psi(x), split at the kink
    for x0 in [0.13, 0.5, 0.77]:
        for kk in [0, 3, 9]:
            tot = 0.0
            for a, b in [(0.0, x0), (x0, 1.0)]:
                xx = a + (b - a) * 0.5 * (xg + 1)
                ww = (b - a) * 0.5 * wg
                tot += np.sum(ww * np.exp(-np.abs(x0 - xx) / lam) * O.psi1d(w[kk], lam, nr[kk], xx))
            assert abs(tot - th[kk] * O.psi1d(w[kk], lam, nr[kk], x0)[0]) < 1e-12


def test_modes_sorted_and_products():
    a, b, th = O.modes(0.3, 1.0, 60)
    _, th1, _ = O.kl1d(0.3, 60)
    assert np.all(np.diff(th) <= 1e-15)
    assert np.allclose(th, th1[a] * th1[b], rtol=1e-15)
    # the smallest kept product is not below any excluded product
    kept = set(zip(a.tolist(), b.tolist()))
    excl = max(th1[i] * th1[j] for i in range(60) for j in range(60) if (i, j) not in kept)
    assert excl <= th[-1] * (1 + 1e-12)
    # sigma scales theta by sigma^2
    _, _, th2 = O.modes(0.3, 2.0, 60)
    assert np.allclose(th2, 4 * th, rtol=1e-15)


def test_field_orthonormal_modes_and_trace():
    # the Gaussian field of a unit vector y = e_m is sqrt(theta_m) psi_m(x);
    # its L2(D) norm^2 is theta_m and different modes are orthogonal. The grid
    # mean of sum_m z_m(x)^2 is the 2D trace identity sum_m theta_m (Sec. 6).
    o = O.Oracle(n_levels=1, n0=256, s=12, sampler="mc", R=1, corr_len=0.3)
    _, _, th, _ = o.modes()
    Z = np.array([o.field_z(0, np.eye(12)[m]) for m in range(12)])
    G = Z @ Z.T / Z.shape[1]  # midpoint rule on 256^2 cells
    assert np.max(np.abs(np.diag(G) - th)) < 2e-4 * th.max()
    off = G - np.diag(np.diag(G))
    assert np.max(np.abs(off)) < 2e-4 * th.max()
    y = W.random_normals(12, 1, tag=3)[0]
    assert np.allclose(o.field(0, y), np.exp(o.field_z(0, y)), rtol=1e-15)
    # linearity in y
    y2 = W.random_normals(12, 1, tag=4)[0]
    assert np.allclose(o.field_z(0, y + y2), o.field_z(0, y) + o.field_z(0, y2), atol=1e-12)


# --------------------------------------------------------------------------- #
# Operator (eq. PDE on the cell-centred FV grid)                             #
# --------------------------------------------------------------------------- #


def _textbook_laplacian(n):
    h = 1.0 / n
    T = sps.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tolil()
    T[0, 0] = 3.0
    T[n - 1, n - 1] = 3.0
    I = sps.identity(n)
    return ((sps.kron(I, T) + sps.kron(T, I)) / h ** 2).toarray()


def _dense_A(n, k):
    cols = []
    for q in range(n * n):
        e = np.zeros(n * n)
        e[q] = 1.0
        cols.append(O.apply_A(n, k, e))
    return np.array(cols).T


@pytest.mark.parametrize("n", [4, 8])
def test_operator_unit_coefficient_is_textbook(n):
    A = _dense_A(n, np.ones(n * n))
    assert np.allclose(A, _textbook_laplacian(n), rtol=0, atol=1e-9)


def test_operator_symmetric_positive_and_energy():
    n = 8
    k = W.random_log_field(n, tag=5)
    A = _dense_A(n, k)
    assert np.allclose(A, A.T, rtol=1e-14, atol=0)
    assert np.linalg.eigvalsh(A).min() > 0
    u = W.rng(6).standard_normal(n * n)
    # energy as a sum of squares over faces (summation by parts)
    K = k.reshape(n, n)
    U = u.reshape(n, n)
    e = 0.0
    for i2 in range(n):
        for i1 in range(n):
            for d1, d2 in [(1, 0), (0, 1)]:
                j1, j2 = i1 + d1, i2 + d2
                if j1 < n and j2 < n:
                    kf = 1.0 / (0.5 / K[i2, i1] + 0.5 / K[j2, j1])  # series conductances
                    e += kf * (U[i2, i1] - U[j2, j1]) ** 2
            nb = (i1 == 0) + (i1 == n - 1) + (i2 == 0) + (i2 == n - 1)
            e += nb * 2 * K[i2, i1] * U[i2, i1] ** 2
    assert abs(u @ O.apply_A(n, k, u) / n ** 2 - e) < 1e-11 * e


# --------------------------------------------------------------------------- #
# FMG (Sec. 4, Fig. FMG)                                                       #
# --------------------------------------------------------------------------- #


def _oracle(n0=4, levels=4, **kw):
    base = dict(n_levels=levels, n0=n0, s=4, sampler="mc", R=1, qoi="mean")
    base.update(kw)
    return O.Oracle(**base)


def test_fmg_visit_sequence_matches_figure():
    o = _oracle(mu0=1)
    out = o.sample(3, 0, 0, log_cap=64)
    assert out["log"] == [3, 2, 1, 0, 1, 0, 1, 2, 1, 0, 1, 2, 3, 2, 1, 0, 1, 2, 3]
    assert out["log_len"] == 19


def test_fmg_converges_to_direct_solution():
    for n0, L in [(4, 2), (8, 2)]:
        o = _oracle(n0=n0, levels=L + 1, rtol=1e-13, max_cycles=100)
        ks = [W.random_log_field(n0 << t, tag=10 + t, scale=0.8) for t in range(L + 1)]
        res = o.fmg_fields(L, ks)
        assert res["status"] == O.OK
        for t in range(L + 1):
            n = n0 << t
            x = np.linalg.solve(_dense_A(n, ks[t]), np.ones(n * n))
            assert np.max(np.abs(res["u"][t] - x)) < 1e-11 * np.max(np.abs(x))


def test_vcycle_contraction_unit_coefficient():
    o = _oracle(n0=4, levels=6)
    t = 5
    ks = [np.ones((4 << q) ** 2) for q in range(t + 1)]
    n = 4 << t
    u = W.rng(7).standard_normal(n * n)
    b = np.zeros(n * n)
    rates = []
    for _ in range(4):
        u2 = o.vcycle_fields(t, ks, b, u)
        rates.append(np.linalg.norm(O.apply_A(n, ks[t], u2)) / np.linalg.norm(O.apply_A(n, ks[t], u)))
        u = u2
    assert max(rates[1:]) < 0.2


def _poisson_series(x, y, terms=401):
    m = np.arange(1, terms, 2)
    M, N = np.meshgrid(m, m, indexing="ij")
    return np.sum(16 / (np.pi ** 4 * M * N * (M ** 2 + N ** 2)) * np.sin(M * np.pi * x) * np.sin(N * np.pi * y))


def _poisson_mean(terms=2001):
    m = np.arange(1, terms, 2, dtype=np.float64)
    M, N = np.meshgrid(m, m, indexing="ij")
    return np.sum(64 / (np.pi ** 6 * M ** 2 * N ** 2 * (M ** 2 + N ** 2)))


def test_fmg_qoi_converges_to_poisson_series():
    # f = 1, k = 1: mean of u and the centre value converge at O(h^2)
    mean_exact = _poisson_mean()
    ctr_exact = _poisson_series(0.5, 0.5)
    errs_m, errs_c = [], []
    for L in [3, 4, 5]:
        ks = [np.ones((4 << t) ** 2) for t in range(L + 1)]
        om = _oracle(n0=4, levels=L + 1, rtol=1e-12, qoi="mean")
        oc = _oracle(n0=4, levels=L + 1, rtol=1e-12, qoi="center")
        errs_m.append(abs(om.fmg_fields(L, ks)["F"][-1] - mean_exact))
        errs_c.append(abs(oc.fmg_fields(L, ks)["F"][-1] - ctr_exact))
    for e in (errs_m, errs_c):
        r1, r2 = e[0] / e[1], e[1] / e[2]
        assert 3.5 < r1 < 4.5 and 3.5 < r2 < 4.5, e


def _cell_grid(f, n):
    c = (np.arange(n) + 0.5) / n
    X1, X2 = np.meshgrid(c, c, indexing="xy")  # row = x2 (i2), column = x1 (i1)
    return f(X1, X2)


def test_prolongation_reproduces_bilinear_functions():
    # reading A4: P is bilinear interpolation between coarse cell centres, with an
    # odd reflection across the Dirichlet boundary for the missing neighbour
    nc = 8
    nf = 2 * nc

    def prol(f):
        return O.prolong(nc, _cell_grid(f, nc)).reshape(nf, nf)

    # interior fine cells (their four coarse neighbours exist): exact for any bilinear function
    g = lambda x1, x2: 0.3 - 1.7 * x1 + 2.9 * x2 + 4.1 * x1 * x2  # noqa: E731
    assert np.max(np.abs(prol(g) - _cell_grid(g, nf))[1:-1, 1:-1]) < 1e-14
    # boundary cells: the odd ghost equals the value of a function that is odd
    # about that boundary, so such bilinear functions are reproduced there too
    for f, sl in [(lambda x1, x2: x1 * x2, np.s_[:-1, :-1]),
                  (lambda x1, x2: (1 - x1) * (1 - x2), np.s_[1:, 1:]),
                  (lambda x1, x2: x1 * (1 - x2), np.s_[1:, :-1]),
                  (lambda x1, x2: (1 - x1) * x2, np.s_[:-1, 1:])]:
        assert np.max(np.abs(prol(f) - _cell_grid(f, nf))[sl]) < 1e-14
    # one interior coarse cell (I2, I1) = (3, 4) with value 16: its four children
    # take 9, the eight fine cells beside them 3, the four diagonal ones 1
    e = np.zeros(nc * nc)
    e[3 * nc + 4] = 16.0
    v = O.prolong(nc, e).reshape(nf, nf)
    w = np.outer([1, 3, 3, 1], [1, 3, 3, 1])
    assert np.array_equal(v[5:9, 7:11], w) and np.sum(v) == 64.0


@pytest.mark.parametrize("mu0,frac", [(1, 0.6), (2, 0.05)])
def test_fixed_cycle_fmg_reaches_discretisation_accuracy(mu0, frac):
    # FMG (Sec. 4, Fig. FMG) with a fixed number of V-cycles per level and no
    # tolerance: on every level its F is within a fixed fraction of the
    # discretisation error from the exact discrete solution's, so F converges to
    # the continuous value (Poisson series, f = 1, k = 1) at O(h^2)
    exact = {"mean": _poisson_mean(), "center": _poisson_series(0.5, 0.5)}
    L = 5
    ks = [np.ones((4 << t) ** 2) for t in range(L + 1)]
    for qoi, ex in exact.items():
        f = _oracle(n0=4, levels=L + 1, mu0=mu0, qoi=qoi).fmg_fields(L, ks)
        d = _oracle(n0=4, levels=L + 1, mu0=mu0, qoi=qoi, rtol=1e-12, max_cycles=100).fmg_fields(L, ks)
        assert f["status"] == O.OK and d["status"] == O.OK
        assert list(f["cycles"][1:]) == [mu0] * L
        F, Fh = f["F"], d["F"]
        for t in range(1, L + 1):
            assert abs(F[t] - Fh[t]) <= frac * abs(Fh[t] - ex), (qoi, t, F[t], Fh[t], ex)
        err = np.abs(F - ex)
        for t in range(2, L + 1):
            assert 3.5 < err[t - 1] / err[t] < 4.5, (qoi, err)


@pytest.mark.parametrize("variable_k", [False, True])
def test_manufactured_solution_second_order(variable_k):
    errs = []
    for L in [3, 4, 5]:
        n = 4 << L
        ks, rhs = [], None
        for t in range(L + 1):
            m = 4 << t
            c = (np.arange(m) + 0.5) / m
            X1, X2 = np.meshgrid(c, c, indexing="xy")  # row = x2, column = x1
            ks.append((np.exp(0.5 * (X1 + X2)) if variable_k else np.ones_like(X1)).reshape(-1))
        c = (np.arange(n) + 0.5) / n
        X1, X2 = np.meshgrid(c, c, indexing="xy")
        s1, s2 = np.sin(np.pi * X1), np.sin(np.pi * X2)
        c1, c2 = np.cos(np.pi * X1), np.cos(np.pi * X2)
        if variable_k:
            kk = np.exp(0.5 * (X1 + X2))
            f = kk * (2 * np.pi ** 2 * s1 * s2 - 0.5 * np.pi * (c1 * s2 + s1 * c2))
        else:
            f = 2 * np.pi ** 2 * s1 * s2
        o = _oracle(n0=4, levels=L + 1, rtol=1e-12)
        res = o.fmg_fields(L, ks, rhs=f.reshape(-1))
        errs.append(np.max(np.abs(res["u"][-1] - (s1 * s2).reshape(-1))))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.5 and 3.5 < r2 < 4.5, errs


def test_recycled_coarse_solutions_are_bitwise_identical():
    # F_t inside a level-k FMG equals F_t of a level-t FMG of the same y (reading A3)
    o = O.Oracle(n_levels=5, n0=4, s=10, sampler="mc", R=1, qoi="center")
    y = W.random_normals(10, 1, tag=8)[0]
    ks = [o.field(t, y) for t in range(5)]
    full = o.fmg_fields(4, ks)["F"]
    for t in range(4):
        part = o.fmg_fields(t, ks[:t + 1])["F"]
        assert np.array_equal(part, full[:t + 1])


# --------------------------------------------------------------------------- #
# Estimators (eqs. MLMC, MGMLMC and its L=2 expansion, Upsilon-reuse,         #
# var_of_mgmlqmc)                                                            #
# --------------------------------------------------------------------------- #


def test_l2_expansion_of_reuse_estimator():
    rg = W.rng(9)
    N = [7, 4, 3]
    R = 1
    # F tables: F[k][n] = (F_0, F_1, F_2 up to level k) for samples of level k
    F = [rg.standard_normal((N[k], k + 1)) for k in range(3)]
    sums = np.zeros((3, R, 2))
    for k in range(3):
        for n in range(N[k]):
            for t in range(k + 1):
                d = F[k][n, t] - (F[k][n, t - 1] if t else 0.0)
                sums[t, 0, 0] += d
    got = O.finalize(2, R, 1, N, sums)["Q"]
    N0, N1, N2 = N
    want = (F[0][:, 0].sum() + F[1][:, 0].sum() + F[2][:, 0].sum()) / (N0 + N1 + N2) \
        + ((F[1][:, 1] - F[1][:, 0]).sum() + (F[2][:, 1] - F[2][:, 0]).sum()) / (N1 + N2) \
        + (F[2][:, 2] - F[2][:, 1]).sum() / N2
    assert abs(got - want) < 1e-13


def test_variance_over_shifts_bruteforce():
    rg = W.rng(10)
    R, L = 8, 2
    sums = rg.standard_normal((L + 1, R, 2))
    N = [10, 5, 2]
    out = O.finalize(L, R, 1, N, sums)
    cnt = [17, 7, 2]
    Ups = sums[:, :, 0] / np.array(cnt)[:, None]
    Qr = Ups.sum(axis=0)
    assert abs(out["Q"] - Qr.mean()) < 1e-14
    assert abs(out["varQ"] - Qr.var(ddof=1) / R) < 1e-14
    assert np.allclose(out["Vell"], Ups.var(axis=1, ddof=1) / R, rtol=1e-13)
    assert np.allclose(out["Ybar"], Ups.mean(axis=1), rtol=1e-13)
    # no reuse: counts are N_t
    out2 = O.finalize(L, R, 0, N, sums)
    Ups2 = sums[:, :, 0] / np.array(N)[:, None]
    assert abs(out2["Q"] - Ups2.sum(axis=0).mean()) < 1e-14


def test_sample_level_sums_telescoping_and_reuse_rule():
    o = O.Oracle(n_levels=3, n0=4, s=6, sampler="mc", R=2, qoi="center")
    work = [(0, 0, 5, 0, 2), (1, 0, 3, 0, 2), (2, 0, 2, 0, 2)]
    out = o.sample_levels(work, want_F=True)
    F = out["F"]
    levels = [lv for (lv, nb, ne, rb, re_) in work for r in range(rb, re_) for n in range(nb, ne)]
    rs = [r for (lv, nb, ne, rb, re_) in work for r in range(rb, re_) for n in range(nb, ne)]
    want = np.zeros((3, 2))
    for i, (lv, r) in enumerate(zip(levels, rs)):
        for t in range(lv + 1):
            want[t, r] += F[i, t] - (F[i, t - 1] if t else 0.0)
        # telescoping per sample
        assert abs(sum(F[i, t] - (F[i, t - 1] if t else 0.0) for t in range(lv + 1)) - F[i, lv]) < 1e-15
    assert np.allclose(out["sums"][:, :, 0], want, rtol=1e-13, atol=1e-16)
    # only the finest level sampled: the reuse estimator is the plain mean of F_L
    only = o.sample_levels([(2, 0, 4, 0, 2)], want_F=True)
    est = O.finalize(2, 2, 1, [0, 0, 4], only["sums"])
    assert abs(est["Q"] - only["F"][:, 2].mean()) < 1e-14
    # reuse off keeps only the difference of each sample's own level
    o2 = O.Oracle(n_levels=3, n0=4, s=6, sampler="mc", R=2, qoi="center", reuse=False)
    out2 = o2.sample_levels(work, want_F=True)
    want2 = np.zeros((3, 2))
    for i, (lv, r) in enumerate(zip(levels, rs)):
        want2[lv, r] += F[i, lv] - (F[i, lv - 1] if lv else 0.0)
    assert np.allclose(out2["sums"][:, :, 0], want2, rtol=1e-13, atol=1e-16)


def test_algorithm1_stopping_rules_and_consistency():
    genvec, _ = O.cbc(6, 10)
    o = O.Oracle(n_levels=5, n0=4, s=6, sampler="lattice", genvec=genvec, R=4, qoi="mean",
                 log2_nmax=10, seed=11)
    eps = 4e-4
    res = o.estimate(eps)
    assert res["status"] == O.OK
    assert res["L"] >= 2
    assert res["varQ"] <= eps ** 2 / 2
    assert res["bias"] <= eps / math.sqrt(2) or res["run_status"] == 7
    for l in range(res["L"] + 1):
        Nl = res["N"][l]
        assert Nl >= 1 and (Nl & (Nl - 1)) == 0
    # the same samples drawn in one go give the same estimate
    work = [(l, 0, res["N"][l], 0, 4) for l in range(res["L"] + 1) if res["N"][l] > 0]
    s = o.sample_levels(work)["sums"]
    est = O.finalize(res["L"], 4, 1, res["N"][:res["L"] + 1], s[:res["L"] + 1])
    assert abs(est["Q"] - res["Q"]) < 1e-13 * abs(res["Q"])
    # close to the converged f=1, k=e^z mean (sanity: within a few eps of a long run)
    assert 0.0 < res["Q"] < 0.2


# --------------------------------------------------------------------------- #
# CBC generating vector (Sec. 3.2; criterion of reading A13)                  #
# --------------------------------------------------------------------------- #


def _dual_criterion(z, m, gamma):
    """e^2 through the dual lattice: sum over h != 0 with h.z = 0 mod N of
    prod_j r_j(h_j), r_j(0) = 1, r_j(h) = gamma_j/(2 pi^2 h^2), summed exactly
    per residue class with sum_k 1/(c+kN)^2 = pi^2/(N^2 sin^2(pi c/N))."""
    N = 2 ** m
    s = len(z)
    d = np.arange(N)
    S = []
    for j in range(s):
        v = np.empty(N)
        v[0] = 1.0 + gamma[j] / (6.0 * N ** 2)
        v[1:] = gamma[j] / (2.0 * N ** 2 * np.sin(np.pi * d[1:] / N) ** 2)
        S.append(v)
    # sum over residue vectors (d_1..d_s) with sum d_j z_j = 0 mod N
    tot = np.zeros(N)  # tot[c] = sum over d_1..d_j with sum d z = c
    tot[0] = 1.0
    for j in range(s):
        new = np.zeros(N)
        for dj in range(N):
            new += S[j][dj] * np.roll(tot, (dj * int(z[j])) % N)
        tot = new
    return tot[0] - 1.0


def test_cbc_one_dimension_closed_form():
    for m in [1, 3, 6, 10]:
        z, e2 = O.cbc(1, m)
        assert z[0] == 1
        # -1 + mean(...) of N terms near 1 cancels: the bound is absolute, N ulps of 1
        assert abs(e2[0] - 1.0 / (6 * 4 ** m)) < (2 ** m) * 2.0 ** -52


@pytest.mark.parametrize("m", [4, 5, 6])
def test_cbc_criterion_dual_lattice(m):
    gamma = np.array([1.0 / (j + 1) ** 2 for j in range(3)])
    z, e2 = O.cbc(3, m, gamma)
    for j in range(3):
        dual = _dual_criterion(z[:j + 1], m, gamma)
        assert abs(e2[j] - dual) < 1e-12 * abs(dual) + (2 ** m) * 2.0 ** -52
    # component-by-component optimality of the last component, by brute force
    N = 2 ** m
    best = min(((_dual_criterion(list(z[:2]) + [c], m, gamma), c) for c in range(1, N // 2 + 1, 2)))
    assert abs(best[0] - e2[2]) < 1e-12 * best[0] + (2 ** m) * 2.0 ** -52


def test_cbc_symmetry_and_config_vector():
    gamma = np.array([1.0 / (j + 1) ** 2 for j in range(4)])
    z, _ = O.cbc(4, 6, gamma)
    zz = z.copy()
    zz[2] = 64 - zz[2]
    assert abs(O.cbc_criterion(z, 6, gamma) - O.cbc_criterion(zz, 6, gamma)) < 1e-15
    z2, e2 = O.cbc(100, 10)
    assert np.all(z2 % 2 == 1) and np.all(z2 <= 512) and z2[0] == 1
    assert np.all(np.diff(e2) > 0)


def test_randomly_shifted_lattice_is_unbiased_on_toy_integrands():
    # Sec. 3.2: with a uniform random shift the rank-1 lattice rule is an
    # unbiased estimator of the integral. Toy integrands of the normals with
    # known means: f(y) = sum_j 2^-j y_j^2 (mean sum_j 2^-j) and the lognormal
    # g(y) = exp(sum_j a_j y_j) (mean exp(sum_j a_j^2 / 2)). Over R shifts the
    # mean of the R rule estimates is within 4 standard errors (from the
    # replicates) of the exact value, and for the smooth g the spread over
    # shifts is well below plain Monte Carlo's with as many points.
    s, m, R = 8, 8, 64
    z, _ = O.cbc(s, m)
    o = O.Oracle(n_levels=1, n0=4, s=s, sampler="lattice", seed=11, R=R, genvec=z, log2_nmax=m)
    N = 1 << m
    w = 2.0 ** -np.arange(1, s + 1)
    a = 0.3 / np.arange(1, s + 1)
    f_exact = w.sum()
    g_exact = np.exp(0.5 * np.sum(a * a))
    Qf, Qg, g_all = np.zeros(R), np.zeros(R), []
    for r in range(R):
        Y = np.array([o.normals(0, r, n) for n in range(N)])
        Qf[r] = np.mean(Y ** 2 @ w)
        gv = np.exp(Y @ a)
        Qg[r] = gv.mean()
        g_all.append(gv)
    for Q, exact in ((Qf, f_exact), (Qg, g_exact)):
        se = Q.std(ddof=1) / np.sqrt(R)
        assert se > 0
        assert abs(Q.mean() - exact) <= 4.0 * se
    mc_se = np.concatenate(g_all).std(ddof=1) / np.sqrt(N)   # one plain-MC estimate of N points
    assert Qg.std(ddof=1) < 0.25 * mc_se   # measured 0.16; random points give about 1
