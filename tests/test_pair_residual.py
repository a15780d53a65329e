"""The FP32-pair residual of the mixed forms' interpolation step: with every
input an FP32 number (the FMG interpolant, the faces, b = 1, c = n^2), the
residual r = 1 - c sum_j k_j (u_P - u_j) formed with FP32 error-free
transformations (TwoSum, the FMA product error, cascaded summation) and
rounded once is within one FP32 ulp of the exact residual, including heavy
cancellation, where the plain FP32 evaluation is off by many ulps. Pinned
against exact rational arithmetic; the arithmetic is emulated in numpy
float32 (an FMA as the exact double product plus the addend, rounded once:
the product of two floats is exact in double)."""
from fractions import Fraction

import numpy as np

f32 = np.float32


def _fma(a, b, c):
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def _two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    return s, f32(f32(a - f32(s - bb)) + f32(b - bb))


def _pair_residual(k, up, u, c):
    ph, pl = [], []
    for j in range(4):
        dh, dl = _two_sum(up, f32(-u[j]))
        p = f32(k[j] * dh)
        ph.append(p)
        pl.append(_fma(k[j], dl, _fma(k[j], dh, -p)))
    sh, sl = ph[0], pl[0]
    for j in range(1, 4):
        sh, e = _two_sum(sh, ph[j])
        sl = f32(sl + f32(e + pl[j]))
    ah = f32(c * sh)
    al = _fma(c, sl, _fma(c, sh, -ah))
    rh, re = _two_sum(f32(1.0), f32(-ah))
    return f32(rh + f32(re - al))


def _plain_fp32(k, up, u, c):
    acc = f32(0.0)
    for j in range(4):
        acc = f32(acc + f32(k[j] * f32(up - u[j])))
    return f32(f32(1.0) - f32(c * acc))


def _exact(k, up, u, c):
    acc = sum(Fraction(float(k[j])) * (Fraction(float(up)) - Fraction(float(u[j]))) for j in range(4))
    return Fraction(1) - Fraction(float(c)) * acc, sum(abs(Fraction(float(k[j])) * (Fraction(float(up)) -
                                                                                      Fraction(float(u[j]))))
                                                     for j in range(4)) * Fraction(float(c))


def _ulp(x):
    x = abs(f32(x))
    return float(np.nextafter(x, f32(np.inf)) - x) if x > 0 else float(np.finfo(np.float32).smallest_subnormal)


def _cases(rng, count, n):
    c = f32(n * n)
    for _ in range(count):
        k = [f32(v) for v in np.exp(rng.standard_normal(4))]
        up = f32(rng.uniform(0.01, 0.08))
        # neighbours within a few grid steps' change, then one of them moved so
        # that c sum_j k_j (u_P - u_j) lands near 1 (heavy cancellation in r)
        u = [f32(up * (1.0 + rng.uniform(-4.0, 4.0) / n)) for _ in range(4)]
        part = sum(float(k[j]) * (float(up) - float(u[j])) for j in range(3))
        target = (1.0 + rng.uniform(-1.0, 1.0) * 2.0 ** -rng.integers(2, 18)) / float(c)
        u[3] = f32(float(up) - (target - part) / float(k[3]))
        yield k, up, u, c


def test_pair_residual_error_bound():
    # beyond its one final rounding the error is a few units of 2^-48 of the
    # term magnitudes c sum_j |k_j (u_P - u_j)| (an FP64 evaluation: 2^-53), so
    # within one ulp of r wherever the terms cancel by less than 2^20; plain
    # FP32 is off by 2^-24 of the terms
    rng = np.random.default_rng(20180614)
    worst_pair, worst_plain, worst_ulp, cancel_max = 0.0, 0.0, 0.0, 0.0
    for n in (16, 256, 1024):
        for k, up, u, c in _cases(rng, 400, n):
            ex, mag = _exact(k, up, u, c)
            exf, mag = float(ex), float(mag)
            if exf == 0.0:
                continue
            cancel = mag / abs(exf)
            cancel_max = max(cancel_max, cancel)
            ulp = _ulp(exf)
            err = abs(float(_pair_residual(k, up, u, c)) - exf)
            worst_pair = max(worst_pair, (err - ulp) / mag)
            worst_plain = max(worst_plain, (abs(float(_plain_fp32(k, up, u, c)) - exf) - ulp) / mag)
            if cancel < 2.0 ** 20:
                worst_ulp = max(worst_ulp, err / ulp)
    assert cancel_max > 2.0 ** 24          # the cases cancel heavily
    assert worst_pair <= 2.0 ** -46
    assert worst_ulp <= 1.0
    assert worst_plain >= 2.0 ** -30


def test_pair_residual_exact_on_the_boundary_and_zero_neighbours():
    # Dirichlet neighbours enter as 0: the terms k_j u_P; all inputs exact
    rng = np.random.default_rng(7)
    for n in (8, 64, 512):
        c = f32(n * n)
        for _ in range(200):
            k = [f32(v) for v in np.exp(rng.standard_normal(4))]
            up = f32(rng.uniform(1e-6, 0.08))
            u = [f32(0.0), f32(up * 0.75), f32(0.0), f32(up * 1.25)]
            ex, _ = _exact(k, up, u, c)
            got = _pair_residual(k, up, u, c)
            assert abs(float(got) - float(ex)) <= _ulp(float(ex))
