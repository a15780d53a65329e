"""Level sizes other than n0 * 2^t with n0 a power of two: coarse grids of 6
and 2 cells per side, so that levels are 6, 12, 24, 48, 96 (generic level-0
factorisation and coarse solves, the plain red-black kernel on sides no
shared-memory smoother takes, three TMA tiles per side on 96) and 2..64."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from test_parity_gpu import EXP_SLACK, MIXED, _field_bound, _pair, _rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("n0,levels,qoi", [(6, 5, "mean"), (2, 6, "center"), (6, 4, "center")])
def test_fp64_solutions_match_oracle(n0, levels, qoi):
    cfg, ctx, orc = _pair(W.LATTICE_6LEVEL, n0=n0, n_levels=levels, s=20, R=2, qoi=qoi, log2_nmax=8)
    for (lv, r, n) in [(levels - 1, 1, 3), (levels - 2, 0, 0)]:
        sols, F = ctx.sample_solution(lv, r, n)
        ref = orc.sample(lv, r, n, want_u=True)
        assert ref["status"] == O.OK
        for t in range(lv + 1):
            assert _rel(sols[t].cpu().numpy(), ref["u"][t]) < 1e-12, (lv, t)
        assert _rel(F.cpu().numpy(), ref["F"]) < 1e-12
    ctx.check_device()


@pytest.mark.parametrize("precision,ufun", MIXED)
def test_mixed_qoi_on_non_power_of_two_levels(precision, ufun):
    cfg, ctx, orc = _pair(W.PRECISION_1024, n0=6, n_levels=5, s=40, R=2, precision=precision, log2_nmax=8)
    names = [k for k, _ in ctx.smoother_info()]
    assert names[4] == "tma" or names[4] == "stream" or names[4] == "tile"
    for (lv, r, n) in [(4, 1, 2), (2, 0, 5)]:
        _, F = ctx.sample_solution(lv, r, n)
        ref = orc.sample(lv, r, n, want_u=True)
        assert ref["status"] == O.OK
        y = orc.normals(lv, r, n)
        # field rounding bound, plus the mixed forms' FP32 normals (a few ulp of 2^-24 each)
        eta = _field_bound(orc, cfg, y, ufun(cfg["s"]) + 2.0 ** -21) + EXP_SLACK
        Fg = F.cpu().numpy()
        for t in range(lv + 1):
            u = ref["u"][t]
            ratio = math.sqrt(np.mean(u ** 2)) / np.mean(u)
            tol = math.expm1(eta) + 2 * cfg["rtol"] * ratio
            assert abs(Fg[t] / ref["F"][t] - 1.0) <= tol, (t, Fg[t], ref["F"][t], tol)
    ctx.check_device()
