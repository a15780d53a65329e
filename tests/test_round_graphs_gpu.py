"""Round graphs: a call of mlqmc_sample_levels that is not a repeat (one
adaptive round of Algorithm 1, Sec. 3.3) runs as one graph launch, the
converged forms' refinement loops as conditional WHILE nodes on the device.

Same kernels in the same order as the launch-by-launch path, so sums, per
sample F and the refinement iteration counts must be bit-identical to it, over
a sequence of rounds of changing shapes (updates of an instantiated graph and
new instantiations), and Algorithm 1 must take the same decisions.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
M = pytest.importorskip("paper_1806_05619_gb300")

ROUNDS = [
    [(0, 0, 1, 0, 2)],
    [(1, 0, 1, 0, 2)],
    [(0, 1, 2, 0, 2)],                      # same shape as the first: an in-place update
    [(5, 0, 2, 0, 2), (3, 1, 5, 0, 1)],     # several levels in one round
    [(2, 0, 3, 0, 2)],
    [(2, 3, 6, 0, 2)],                      # same shape, other points
    [(2, 3, 6, 0, 2)],                      # a repeat
    [(4, 0, 1, 1, 2), (0, 2, 9, 0, 2)],
]


def _context(precision, rtol):
    # one context for both paths: two contexts could tune different smoothers
    # (the choice changes FP32 rounding)
    cfg = W.scaled(W.LATTICE_6LEVEL, R=2, s=24, precision=precision, rtol=rtol, max_cycles=30)
    z, _ = M.cbc_genvec(cfg["s"], cfg["log2_nmax"])
    ctx = M.Context.from_config(cfg, genvec=z)
    ctx.set_round_graphs("on")  # the fixed-cycle forms too (their default is launch by launch)
    return cfg, ctx


def _call(ctx, cfg, work):
    nl = cfg["n_levels"]
    ns = sum((ne - nb) * (re_ - rb) for (_, nb, ne, rb, re_) in work)
    sums = torch.zeros(nl * cfg["R"] * 2, dtype=torch.float64, device="cuda")
    F = torch.zeros(ns * nl, dtype=torch.float64, device="cuda")
    ctx.sample_levels(work, sums, F)
    torch.cuda.synchronize()
    ctx.check_device()
    return sums.cpu().numpy(), F.cpu().numpy()


@pytest.mark.parametrize("precision,rtol", [("fp64", 0.0), ("mixed_tf32", 0.0), ("fp64", 1e-10),
                                            ("mixed_tf32", 1e-10)])
def test_rounds_equal_direct_path(precision, rtol):
    cfg, ctx = _context(precision, rtol)
    on = [_call(ctx, cfg, work) for work in ROUNDS]
    it_on = ctx.last_iterations()
    st = ctx.graph_stats()
    assert st["round_launches"] >= len(ROUNDS) - 1
    assert st["round_updates"] >= 2 and st["round_instantiations"] >= 1
    ctx.set_graphs(False)
    off = [_call(ctx, cfg, work) for work in ROUNDS]
    assert ctx.graph_stats()["round_launches"] == st["round_launches"]
    for work, a, b in zip(ROUNDS, on, off):
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), work
    if rtol > 0:
        assert it_on == ctx.last_iterations()


@pytest.mark.parametrize("precision", ["fp64", "mixed_tf32"])
def test_algorithm1_same_with_and_without_round_graphs(precision):
    cfg = W.scaled(W.ADAPTIVE_7LEVEL, n_levels=5, s=24, precision=precision, log2_nmax=12)
    z, _ = M.cbc_genvec(cfg["s"], cfg["log2_nmax"])
    ctx = M.Context.from_config(cfg, genvec=z)
    ctx.set_round_graphs("on")
    a = ctx.estimate(3e-3)
    sa = ctx.graph_stats()
    ctx.set_graphs(False)
    b = ctx.estimate(3e-3)
    sb = ctx.graph_stats()
    ctx.close()
    assert a["L"] == b["L"] and a["rounds"] == b["rounds"] and a["N"] == b["N"]
    assert a["Q"] == b["Q"] and a["varQ"] == b["varQ"]
    assert sa["round_launches"] == a["rounds"] and sb["round_launches"] == sa["round_launches"]
