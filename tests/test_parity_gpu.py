"""GPU path against the FP64 oracle through the C ABI.

Tolerances (FP64 form): lattice bits bit-exact; normals 1e-14 relative (CUDA's
normcdfinv against AS 241, both within a few ulp); fields, solutions and F_t
1e-12 relative; reuse sums within 1e-12 of the sum of |F_t| + |F_{t-1}| over
the samples entering them (dF_t cancels, and the two sides add in different
orders).
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
M = pytest.importorskip("paper_1806_05619_gb300")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import os
    if not os.path.exists(M.LIB_PATH):
        M.build()
    assert torch.cuda.is_available()


def _genvec(cfg):
    if cfg["sampler"] != "lattice":
        return None
    z, _ = M.cbc_genvec(cfg["s"], cfg["log2_nmax"])
    zo, _ = O.cbc(cfg["s"], cfg["log2_nmax"])
    assert np.array_equal(z, zo)
    return z


def _pair(cfg, **over):
    cfg = W.scaled(cfg, **over)
    z = _genvec(cfg)
    ctx = M.Context.from_config(cfg, genvec=z)
    orc = O.Oracle(n_levels=cfg["n_levels"], n0=cfg["n0"], s=cfg["s"], sigma=cfg["sigma"],
                   corr_len=cfg["corr_len"], qoi=cfg["qoi"], mu0=cfg["mu0"], nu1=cfg["nu1"], nu2=cfg["nu2"],
                   rtol=cfg["rtol"] if cfg["precision"] == "fp64" else 1e-12,
                   max_cycles=max(cfg["max_cycles"], 100), sampler=cfg["sampler"], seed=cfg["seed"], R=cfg["R"],
                   genvec=z, log2_nmax=cfg["log2_nmax"], reuse=cfg["reuse"])
    return cfg, ctx, orc


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


# --------------------------------------------------------------------------- #
# a1: lattice points and normals                                              #
# --------------------------------------------------------------------------- #


@pytest.mark.parametrize("pid", [1, 2])
def test_point_bits_bit_exact(pid):
    cfg, ctx, orc = _pair(W.PROBLEMS[pid])
    for level, r, nb, cnt in [(0, 0, 0, 64), (3, 5 % cfg["R"], 17, 45), (cfg["n_levels"] - 1, cfg["R"] - 1, 0, 7)]:
        bits = ctx.point_bits(level, r, nb, cnt).cpu().numpy().view(np.uint64)
        for i in range(cnt):
            n = nb + i
            for j in range(cfg["s"]):
                if cfg["sampler"] == "lattice":
                    want = O.lattice_bits(int(orc._z[j]), n, O.shift_bits(cfg["seed"], level, r, j))
                else:
                    want = O.mc_bits(cfg["seed"], level, r, n, j)
                assert int(bits[i, j]) == want, (level, r, n, j)


def test_lattice_index_end_of_sequence():
    cfg, ctx, orc = _pair(W.LATTICE_6LEVEL)
    N = 2 ** cfg["log2_nmax"]
    bits = ctx.point_bits(2, 1, N - 3, 3).cpu().numpy().view(np.uint64)
    for i in range(3):
        for j in range(cfg["s"]):
            assert int(bits[i, j]) == O.lattice_bits(int(orc._z[j]), N - 3 + i, O.shift_bits(cfg["seed"], 2, 1, j))
    with pytest.raises(M.MlqmcError) as e:
        ctx.point_bits(2, 1, N - 2, 3)
    assert e.value.code == 4


@pytest.mark.parametrize("pid", [1, 2])
def test_normals(pid):
    cfg, ctx, orc = _pair(W.PROBLEMS[pid])
    y = ctx.normals(2, 0, 5, 40).cpu().numpy()
    for i in range(40):
        want = orc.normals(2, 0, 5 + i)
        assert np.max(np.abs(y[i] - want) / np.maximum(np.abs(want), 1e-3)) < 1e-14


# --------------------------------------------------------------------------- #
# a2: KL field                                                                #
# --------------------------------------------------------------------------- #


def test_modes_match():
    cfg, ctx, orc = _pair(W.LATTICE_6LEVEL)
    a, b, th = ctx.modes()
    ao, bo, tho, _ = orc.modes()
    assert np.array_equal(a, ao) and np.array_equal(b, bo)
    assert _rel(th, tho) < 1e-13


@pytest.mark.parametrize("pid,levels", [(1, [0, 3]), (2, [0, 2, 4]), (3, [0, 3])])
def test_fields_fp64(pid, levels):
    cfg, ctx, orc = _pair(W.PROBLEMS[pid], precision="fp64", rtol=0.0)
    Y = W.random_normals(cfg["s"], 3, tag=20 + pid)
    for t in levels:
        k = ctx.fields(t, torch.from_numpy(Y)).cpu().numpy()
        for i in range(3):
            want = orc.field(t, Y[i])
            assert np.max(np.abs(k[i] / want - 1.0)) < 1e-12


# --------------------------------------------------------------------------- #
# a3-a6: FMG solutions and F_t, FP64 form                                     #
# --------------------------------------------------------------------------- #


@pytest.mark.parametrize("pid,level,r,n", [(1, 3, 0, 5), (2, 0, 0, 0), (2, 3, 2, 7), (2, 5, 15, 3)])
def test_single_sample_solutions_fp64(pid, level, r, n):
    cfg, ctx, orc = _pair(W.PROBLEMS[pid])
    sols, F = ctx.sample_solution(level, r, n)
    ref = orc.sample(level, r, n, want_u=True)
    assert ref["status"] == O.OK
    for t in range(level + 1):
        assert _rel(sols[t].cpu().numpy(), ref["u"][t]) < 1e-12, t
    assert _rel(F.cpu().numpy(), ref["F"]) < 1e-12


def _check_sums(cfg, ctx, orc, work):
    R, nl = cfg["R"], cfg["n_levels"]
    nsamp = sum((ne - nb) * (re_ - rb) for (_, nb, ne, rb, re_) in work)
    sums = torch.zeros(nl * R * 2, dtype=torch.float64, device="cuda")
    F = torch.zeros(max(1, nsamp) * nl, dtype=torch.float64, device="cuda")
    ctx.sample_levels(work, sums, F)
    ctx.check_device()
    torch.cuda.synchronize()
    ref = orc.sample_levels(work, want_F=True)
    Fg = F.cpu().numpy().reshape(-1, nl)[:nsamp]
    assert _rel(Fg, ref["F"]) < 1e-12
    # bound for the sums: dF_t = F_t - F_{t-1} cancels, so each term carries
    # 1e-12 of |F_t| + |F_{t-1}|
    # and a square dF_t^2 carries 2 |dF_t| times that
    absd = np.zeros((nl, R))
    absd2 = np.zeros((nl, R))
    i = 0
    for (lv, nb, ne, rb, re_) in work:
        for r in range(rb, re_):
            for _ in range(nb, ne):
                for t in range(lv + 1):
                    if cfg["reuse"] or t == lv:
                        mag = abs(ref["F"][i, t]) + (abs(ref["F"][i, t - 1]) if t else 0.0)
                        d = ref["F"][i, t] - (ref["F"][i, t - 1] if t else 0.0)
                        absd[t, r] += mag
                        absd2[t, r] += 2 * abs(d) * mag + d * d
                i += 1
    s = sums.cpu().numpy().reshape(nl, R, 2)
    assert np.all(np.abs(s[:, :, 0] - ref["sums"][:, :, 0]) <= 1e-12 * absd + 1e-300)
    assert np.all(np.abs(s[:, :, 1] - ref["sums"][:, :, 1]) <= 1e-12 * absd2 + 1e-300)
    return s, Fg


def test_config1_full_sums():
    cfg, ctx, orc = _pair(W.MC_4LEVEL)
    work = W.fixed_count_work(cfg["counts"], cfg["R"])
    _check_sums(cfg, ctx, orc, work)


@pytest.mark.parametrize("reuse", [True, False])
def test_config2_ragged_work(reuse):
    cfg, ctx, orc = _pair(W.LATTICE_6LEVEL, R=4, reuse=reuse)
    work = [(0, 0, 13, 0, 3), (1, 5, 9, 1, 4), (2, 0, 3, 0, 4), (3, 2, 4, 2, 3), (4, 0, 1, 0, 2), (5, 0, 1, 3, 4),
            (2, 7, 7, 0, 4)]
    _check_sums(cfg, ctx, orc, work)


def test_chunked_calls_equal_single_call():
    cfg = W.scaled(W.LATTICE_6LEVEL, R=2)
    z = _genvec(cfg)
    work = [(0, 0, 40, 0, 2), (2, 0, 9, 0, 2), (3, 0, 3, 0, 2)]
    outs = []
    for ms in [65536, 7]:
        ctx = M.Context.from_config(cfg, genvec=z, max_samples=ms)
        sums = torch.zeros(cfg["n_levels"] * 2 * 2, dtype=torch.float64, device="cuda")
        F = torch.zeros(104 * cfg["n_levels"], dtype=torch.float64, device="cuda")
        ctx.sample_levels(work, sums, F)
        torch.cuda.synchronize()
        outs.append((sums.cpu().numpy(), F.cpu().numpy()))
    assert np.array_equal(outs[0][1], outs[1][1])
    assert np.allclose(outs[0][0], outs[1][0], rtol=1e-13, atol=1e-18)


def test_empty_and_invalid_work():
    cfg, ctx, orc = _pair(W.LATTICE_6LEVEL, R=2)
    sums = torch.zeros(cfg["n_levels"] * 2 * 2, dtype=torch.float64, device="cuda")
    ctx.sample_levels([], sums)
    ctx.sample_levels([(1, 4, 4, 0, 2)], sums)
    torch.cuda.synchronize()
    assert torch.count_nonzero(sums).item() == 0
    for bad, code in [((6, 0, 1, 0, 1), 1), ((0, 3, 2, 0, 1), 1), ((0, 0, 1, 0, 3), 1), ((0, 0, 1025, 0, 1), 4)]:
        with pytest.raises(M.MlqmcError) as e:
            ctx.sample_levels([bad], sums)
        assert e.value.code == code


def test_full_config2_launch_sampled_against_oracle():
    """The bench's workload in its launch configuration: all 32256 samples of
    the fixed counts; sampled F rows against the oracle one by one, and the
    sums against a host recomputation from the per-sample F (any size)."""
    cfg, ctx, orc = _pair(W.LATTICE_6LEVEL)
    work = W.fixed_count_work(cfg["counts"], cfg["R"])
    nl, R = cfg["n_levels"], cfg["R"]
    nsamp = sum((ne - nb) * (re_ - rb) for (_, nb, ne, rb, re_) in work)
    sums = torch.zeros(nl * R * 2, dtype=torch.float64, device="cuda")
    F = torch.zeros(nsamp * nl, dtype=torch.float64, device="cuda")
    ctx.sample_levels(work, sums, F)
    ctx.check_device()
    torch.cuda.synchronize()
    Fg = F.cpu().numpy().reshape(nsamp, nl)
    index = []
    for (lv, nb, ne, rb, re_) in work:
        for r in range(rb, re_):
            for n in range(nb, ne):
                index.append((lv, r, n))
    rg = W.rng(33)
    picks = list(rg.choice(nsamp, 10, replace=False)) + [nsamp - 1, nsamp - 2, 0]
    for q in picks:
        lv, r, n = index[q]
        ref = orc.sample(lv, r, n)
        assert _rel(Fg[q, :lv + 1], ref["F"]) < 1e-12
        assert np.all(Fg[q, lv + 1:] == 0.0)
    # sums from the per-sample F (telescoped differences) in FP64 on the host
    want = np.zeros((nl, R))
    absd = np.zeros((nl, R))
    for q, (lv, r, n) in enumerate(index):
        d = np.diff(np.concatenate([[0.0], Fg[q, :lv + 1]]))
        want[:lv + 1, r] += d
        absd[:lv + 1, r] += np.abs(Fg[q, :lv + 1]) + np.abs(np.concatenate([[0.0], Fg[q, :lv]]))
    s = sums.cpu().numpy().reshape(nl, R, 2)
    assert np.all(np.abs(s[:, :, 0] - want) <= 1e-12 * absd)


# --------------------------------------------------------------------------- #
# a7-a8: estimator and Algorithm 1                                            #
# --------------------------------------------------------------------------- #


def test_algorithm1_matches_oracle():
    cfg, ctx, orc = _pair(W.LATTICE_6LEVEL, n_levels=5, n0=4, s=6, R=4, seed=11, log2_nmax=10)
    eps = 4e-4
    g = ctx.estimate(eps)
    o = orc.estimate(eps)
    assert o["status"] == O.OK
    assert g["L"] == o["L"] and g["rounds"] == o["rounds"]
    assert g["N"] == o["N"]
    assert abs(g["Q"] - o["Q"]) <= 1e-12 * abs(o["Q"])
    assert abs(g["varQ"] - o["varQ"]) <= 1e-9 * o["varQ"]
    assert g["varQ"] <= eps ** 2 / 2


def test_device_status_not_converged():
    cfg, ctx, orc = _pair(W.LATTICE_6LEVEL, R=1, rtol=1e-30, max_cycles=0)
    sums = torch.zeros(cfg["n_levels"] * 2, dtype=torch.float64, device="cuda")
    ctx.sample_levels([(2, 0, 2, 0, 1)], sums)
    assert ctx.device_status() == 5
    assert ctx.device_status() == 0  # reading clears it


# --------------------------------------------------------------------------- #
# Mixed precision (a2 in FP32, a4 FP32 V-cycles inside a5 FP64 refinement)     #
# --------------------------------------------------------------------------- #


def _field_bound(orc, cfg, y, u_in):
    """Rounding bound on |z_mixed - z_64|: u_in * sum_m |sqrt(theta_m) y_m| M_a M_b with
    M_k = sqrt((w_k^2 + c^2)/N_k) >= max |psi_k|."""
    a, b, th, K1 = orc.modes()
    w, _, nr = O.kl1d(cfg["corr_len"], K1)
    c = 1.0 / cfg["corr_len"]
    Mk = np.sqrt((w ** 2 + c ** 2) / nr)
    return u_in * np.sum(np.sqrt(th) * np.abs(y) * Mk[a] * Mk[b])


def _tf32_u(s):
    """Error factor of the TF32 contraction: both operands rounded to TF32
    (2 * 2^-11) and an FP32 accumulation over s terms (s * 2^-24)."""
    return 2 * 2.0 ** -11 + s * 2.0 ** -24


def _bf16x3_u(s):
    """Error factor of the split-BF16 contraction: each operand x = hi + lo + d
    with |d| <= 2^-16 |x| (8-bit significands, unit roundoff 2^-8 twice), the
    dropped lo*lo product <= 2^-16 |ab|, the FP32 rounding of both operands
    (2 * 2^-24) and an FP32 accumulation over the 3s products (3s * 2^-24)."""
    return 3 * 2.0 ** -16 + 2 * 2.0 ** -24 + 3 * s * 2.0 ** -24


EXP_SLACK = 2.0 ** -20  # FP32 exp and the FP32 face arithmetic
MIXED = [("mixed_tf32", _tf32_u), ("mixed_bf16x3", _bf16x3_u)]


@pytest.mark.parametrize("precision,ufun", MIXED)
def test_mixed_fields_within_bound(precision, ufun):
    cfg, ctx, orc = _pair(W.PRECISION_1024, n_levels=4, precision=precision)
    Y = W.random_normals(cfg["s"], 2, tag=40)
    for t in [0, 3]:
        k = ctx.fields(t, torch.from_numpy(Y)).cpu().numpy()
        for i in range(2):
            want = orc.field(t, Y[i])
            eta = _field_bound(orc, cfg, Y[i], ufun(cfg["s"]))
            assert np.max(np.abs(np.log(k[i] / want))) <= eta + EXP_SLACK


def test_split_bf16_more_accurate_than_tf32():
    """Same normals, level of 256 x 256 cells (tensor-core path): the split-BF16
    field's largest log-error is at least 8x below the TF32 one."""
    errs = {}
    for precision in ["mixed_tf32", "mixed_bf16x3"]:
        cfg, ctx, orc = _pair(W.PRECISION_1024, n_levels=6, precision=precision)
        Y = W.random_normals(cfg["s"], 3, tag=42)
        k = ctx.fields(5, torch.from_numpy(Y)).cpu().numpy()
        errs[precision] = max(np.max(np.abs(np.log(k[i] / orc.field(5, Y[i])))) for i in range(3))
    assert errs["mixed_bf16x3"] * 8 <= errs["mixed_tf32"], errs


@pytest.mark.parametrize("precision,ufun", MIXED)
def test_tensor_core_fields_many_samples(precision, ufun):
    """More samples than one tensor-core tile (256) and several cell tiles."""
    cfg, ctx, orc = _pair(W.PRECISION_1024, n_levels=4, precision=precision)
    Y = W.random_normals(cfg["s"], 300, tag=41)
    k = ctx.fields(2, torch.from_numpy(Y)).cpu().numpy()
    assert np.all(np.isfinite(k)) and np.all(k > 0)
    for i in [0, 1, 255, 256, 299]:
        want = orc.field(2, Y[i])
        eta = _field_bound(orc, cfg, Y[i], ufun(cfg["s"]))
        err = np.max(np.abs(np.log(k[i] / want)))
        assert err <= eta + EXP_SLACK, (i, err, eta)
    ctx.check_device()


@pytest.mark.parametrize("precision,ufun", MIXED)
def test_mixed_qoi_within_bound(precision, ufun):
    cfg, ctx, orc = _pair(W.PRECISION_1024, n_levels=5, R=2, precision=precision)
    for (lv, r, n) in [(4, 0, 3), (2, 1, 0)]:
        sols, F = ctx.sample_solution(lv, r, n)
        ref = orc.sample(lv, r, n, want_u=True)
        assert ref["status"] == O.OK
        y = orc.normals(lv, r, n)
        eta = _field_bound(orc, cfg, y, ufun(cfg["s"])) + EXP_SLACK
        Fg = F.cpu().numpy()
        for t in range(lv + 1):
            u = ref["u"][t]
            ratio = math.sqrt(np.mean(u ** 2)) / np.mean(u)
            tol = math.expm1(eta) + 2 * cfg["rtol"] * ratio
            assert abs(Fg[t] / ref["F"][t] - 1.0) <= tol, (t, Fg[t], ref["F"][t], tol)
    ctx.check_device()


# --------------------------------------------------------------------------- #
# Smoothers of the FP32 V-cycles: same sweeps whichever kernel runs them      #
# --------------------------------------------------------------------------- #


def _force(ctx, name):
    for t in range(1, ctx.n_levels):
        try:
            ctx.set_smoother(t, name)
        except M.MlqmcError:
            pass  # this smoother does not handle the level; the tuned one stays


def _mixed_F(ctx, cfg, work, names):
    out = {}
    ns = sum((ne - nb) * (re_ - rb) for (_, nb, ne, rb, re_) in work)
    for name in names:
        _force(ctx, name)
        sums = torch.zeros(cfg["n_levels"] * cfg["R"] * 2, dtype=torch.float64, device="cuda")
        F = torch.zeros(ns * cfg["n_levels"], dtype=torch.float64, device="cuda")
        ctx.sample_levels(work, sums, F)
        torch.cuda.synchronize()
        ctx.check_device()
        out[name] = F.cpu().numpy().reshape(ns, cfg["n_levels"])
    return out


def test_fp32_interpolant_path_matches_fp64_store():
    """Fixed-cycle mixed form with the mean QoI: a plain sampling call carries
    the FMG interpolant of the TMA levels (128x128, 256x256) in FP32 and forms
    each level's one refinement update as an exact FP32 pair; a call that asks
    for the solution keeps the FP64 store (u64 += e in FP64). Both are the
    same update of the same numbers, so per-level F agree to the FP32 pair
    sum's accuracy (1e-12 relative), and both match the oracle within the
    TF32 field bound."""
    cfg, ctx, orc = _pair(W.LATTICE_6LEVEL, R=2, precision="mixed_tf32")
    nl = cfg["n_levels"]
    for (lv, r, n) in [(5, 0, 0), (5, 1, 3), (4, 0, 1)]:
        sums = torch.zeros(nl * cfg["R"] * 2, dtype=torch.float64, device="cuda")
        F = torch.zeros(nl, dtype=torch.float64, device="cuda")
        ctx.sample_levels([(lv, n, n + 1, r, r + 1)], sums, F)
        torch.cuda.synchronize()
        ctx.check_device()
        _, Fs = ctx.sample_solution(lv, r, n)
        a = F.cpu().numpy()[:lv + 1]
        b = Fs.cpu().numpy()
        assert _rel(a, b) <= 1e-12, (lv, r, n, a, b)
        ref = orc.sample(lv, r, n)
        eta = _field_bound(orc, cfg, orc.normals(lv, r, n), _tf32_u(cfg["s"])) + EXP_SLACK
        assert np.max(np.abs(a / ref["F"] - 1)) <= math.expm1(eta) + 1e-9


def test_smoothers_agree_fixed_cycles():
    """Mixed form, fixed cycles (6 levels up to 256x256): the wavefront and
    whole-sample smoothers (residual and correction fused), TMA-tile and
    plain-tile smoothers run the same red-black sweeps; per-sample F agree to
    FP32 rounding of the residual's summation order (1e-5 relative)."""
    cfg = W.scaled(W.LATTICE_6LEVEL, R=2, precision="mixed_tf32")
    z = _genvec(cfg)
    ctx = M.Context.from_config(cfg, genvec=z)
    work = [(5, 0, 3, 0, 2), (4, 1, 4, 0, 2), (3, 0, 5, 1, 2), (1, 2, 6, 0, 1)]
    F = _mixed_F(ctx, cfg, work, ["stream", "tma", "tile", "whole"])
    mask = F["tile"] != 0
    for name in ["stream", "tma", "whole"]:
        assert np.array_equal(F[name] != 0, mask)
        assert _rel(F[name][mask], F["tile"][mask]) <= 1e-5, name


def test_smoothers_agree_converged():
    """Converged mixed form (rtol 1e-10, levels up to 128x128, samples leave
    the refinement loop at different steps): per-sample F of the wavefront and
    TMA-tile smoothers agree within 1e-8 relative."""
    cfg = W.scaled(W.PRECISION_1024, n_levels=5, R=2)
    z = _genvec(cfg)
    ctx = M.Context.from_config(cfg, genvec=z)
    work = [(4, 0, 6, 0, 2), (3, 0, 3, 0, 1)]
    F = _mixed_F(ctx, cfg, work, ["stream", "tma", "whole"])
    mask = F["stream"] != 0
    assert _rel(F["tma"][mask], F["stream"][mask]) <= 1e-8
    assert _rel(F["whole"][mask], F["stream"][mask]) <= 1e-8


def test_autotuner_report():
    cfg = W.scaled(W.LATTICE_6LEVEL, R=2, precision="mixed_tf32")
    ctx = M.Context.from_config(cfg, genvec=_genvec(cfg), max_samples=2048)
    info = ctx.smoother_info()
    assert info[0][0] == "gs"
    for t, (name, ms) in enumerate(info[1:], start=1):
        n = cfg["n0"] << t
        assert name in ("stream", "tma", "tile", "whole")
        if len(ms) >= 2:
            assert name == min(ms, key=ms.get), (t, name, ms)
        if n > 256:
            assert name == "tma"
    with pytest.raises(M.MlqmcError):
        ctx.set_smoother(1, "tma")  # 16 x 16: no whole TMA tile with its halo inside the grid
    c64 = M.Context.from_config(W.scaled(W.LATTICE_6LEVEL, R=2), genvec=_genvec(cfg))
    for t, (k, _) in enumerate(c64.smoother_info()):
        assert k == "gs" or (k == "whole" and (cfg["n0"] << t) <= 64)
    with pytest.raises(M.MlqmcError):
        c64.set_smoother(3, "stream")  # FP64 form: kb_gs, the whole-sample smoother or the plain tiles


def test_batch_schedule_report_and_results():
    """The autotuner's batch-size schedule: a small-batch smoother per level
    (the fastest of its timings on 64 samples) and a KL tile width (128 or 256
    samples) per level and batch class (the faster of the two timings; every
    level's field is a tensor-core contraction in the mixed forms, a level of
    fewer than 128 cells in one zero-padded tile); calls of either class still
    match the oracle within the TF32 field bound."""
    cfg, ctx, orc = _pair(W.PRECISION_1024, n_levels=6, R=2, precision="mixed_tf32", rtol=1e-10)
    info = ctx.schedule_info()
    for t, row in enumerate(info):
        n = cfg["n0"] << t
        if t > 0:
            assert row["smoother_small"] in ("stream", "tma", "tile", "whole")
            if len(row["small_ms"]) >= 2:
                assert row["smoother_small"] == min(row["small_ms"], key=row["small_ms"].get), (t, row)
        for cls in range(2):
            assert row["kl_nt"][cls] in (128, 256), (t, n, row)
            ms = row["kl_ms"][cls]
            assert min(ms) > 0 and row["kl_nt"][cls] == (128 if ms[0] < ms[1] else 256)
    for (lv, r, n) in [(5, 0, 1), (5, 1, 2)]:
        _, F = ctx.sample_solution(lv, r, n)
        ref = orc.sample(lv, r, n)
        eta = _field_bound(orc, cfg, orc.normals(lv, r, n), _tf32_u(cfg["s"])) + EXP_SLACK
        assert np.max(np.abs(F.cpu().numpy() / ref["F"] - 1)) <= math.expm1(eta) + 1e-9
    work = [(5, 0, 20, 0, 2), (2, 0, 200, 0, 2)]  # 440 samples reach levels 0..2: the large class there
    sums = torch.zeros(cfg["n_levels"] * cfg["R"] * 2, dtype=torch.float64, device="cuda")
    F = torch.zeros(440 * cfg["n_levels"], dtype=torch.float64, device="cuda")
    ctx.sample_levels(work, sums, F)
    torch.cuda.synchronize()
    ctx.check_device()
    Fg = F.cpu().numpy().reshape(440, cfg["n_levels"])
    for q, (lv, r, n) in [(0, (5, 0, 0)), (439, (2, 1, 199))]:
        ref = orc.sample(lv, r, n)
        eta = _field_bound(orc, cfg, orc.normals(lv, r, n), _tf32_u(cfg["s"])) + EXP_SLACK
        assert np.max(np.abs(Fg[q, :lv + 1] / ref["F"] - 1)) <= math.expm1(eta) + 1e-9


def test_fp64_whole_sample_smoother_matches_gs():
    """FP64 form: the whole-sample smoother (levels up to 64 x 64) multiplies by
    the stored 1/D like kb_gs and fuses residual and correction with the same
    arithmetic: per-sample F agree with the kb_gs path to 1e-13."""
    cfg = W.scaled(W.LATTICE_6LEVEL, R=2)
    ctx = M.Context.from_config(cfg, genvec=_genvec(cfg))
    work = [(5, 0, 2, 0, 2), (3, 0, 3, 0, 2), (2, 0, 4, 1, 2)]
    ns = sum((ne - nb) * (re_ - rb) for (_, nb, ne, rb, re_) in work)
    out = {}
    for name in ["gs", "whole"]:
        for t in (1, 2, 3):
            ctx.set_smoother(t, name)
        sums = torch.zeros(cfg["n_levels"] * 2 * 2, dtype=torch.float64, device="cuda")
        F = torch.zeros(ns * cfg["n_levels"], dtype=torch.float64, device="cuda")
        ctx.sample_levels(work, sums, F)
        torch.cuda.synchronize()
        out[name] = F.cpu().numpy()
    mask = out["gs"] != 0
    assert _rel(out["whole"][mask], out["gs"][mask]) <= 1e-13
    ctx.check_device()


@pytest.mark.parametrize("pid,precision", [(2, "fp64"), (6, "fp64"), (2, "mixed_tf32"), (6, "mixed_tf32")])
def test_level0_split_kernel_matches_thread_per_sample(pid, precision):
    """The level-0 exact solve of calls with fewer than 16,384 samples splits
    every factorisation step over the warps of a CTA (kb_level0_split); larger
    calls take one thread per sample (kb_level0_fixed). Both perform the same
    operations in the same order: F_0 of the same samples is bit-identical in
    the FP64 form (n0 = 8 and n0 = 4) and, in the mixed form, agrees to 1e-13
    (the tensor-core fields of the two calls may use other tile widths), and
    the small call stays within 1e-12 of the oracle (FP64 form)."""
    cfg, ctx, orc = _pair(W.PROBLEMS[pid], precision=precision)
    R, npts = cfg["R"], 16384 // cfg["R"]
    nl = cfg["n_levels"]
    out = {}
    for name, work in (("big", [(0, 0, npts, 0, R)]), ("small", [(0, 0, 64, 0, 2)])):
        ns = sum((ne - nb) * (re_ - rb) for (_, nb, ne, rb, re_) in work)
        S = torch.zeros(nl * R * 2, dtype=torch.float64, device="cuda")
        F = torch.zeros(ns * nl, dtype=torch.float64, device="cuda")
        ctx.sample_levels(work, S, F)
        torch.cuda.synchronize()
        ctx.check_device()
        out[name] = F.cpu().numpy().reshape(ns, nl)[:, 0]
    big = np.concatenate([out["big"][r * npts: r * npts + 64] for r in range(2)])
    if precision == "fp64":
        assert np.array_equal(out["small"], big)
        for q, (r, n) in [(0, (0, 0)), (70, (1, 6)), (127, (1, 63))]:
            ref = orc.sample(0, r, n)
            assert abs(out["small"][q] / ref["F"][0] - 1) <= 1e-12, (r, n)
    else:
        assert _rel(out["small"], big) <= 1e-13


def test_fp64_tile_smoother_matches_gs():
    """FP64 form: the plain-tile smoother (one full red-black sweep per launch
    on 32 x 32 tiles, the coarse-grid correction added to the staged tile)
    performs kb_gs's operations in kb_gs's order, an outside neighbour being a
    staged zero; with it on the 128 x 128 and 256 x 256 levels, per-sample F
    and the reuse sums agree with two kb_gs launches per sweep (the default
    there) to 1e-13, and stay within 1e-12 of the oracle."""
    cfg, ctx, orc = _pair(W.LATTICE_6LEVEL, R=2)
    assert [k for k, _ in ctx.smoother_info()][4:6] == ["gs", "gs"]
    work = [(5, 0, 3, 0, 2), (4, 1, 4, 0, 2), (2, 0, 4, 1, 2)]
    ns = sum((ne - nb) * (re_ - rb) for (_, nb, ne, rb, re_) in work)
    out, sums = {}, {}
    for name in ["tile", "gs"]:
        for t in (4, 5):
            ctx.set_smoother(t, name)
        S = torch.zeros(cfg["n_levels"] * 2 * 2, dtype=torch.float64, device="cuda")
        F = torch.zeros(ns * cfg["n_levels"], dtype=torch.float64, device="cuda")
        ctx.sample_levels(work, S, F)
        torch.cuda.synchronize()
        ctx.check_device()
        out[name] = F.cpu().numpy().reshape(ns, cfg["n_levels"])
        sums[name] = S.cpu().numpy()
    mask = out["gs"] != 0
    assert _rel(out["tile"][mask], out["gs"][mask]) <= 1e-13
    assert _rel(sums["tile"], sums["gs"]) <= 1e-13
    for q, (lv, r, n) in [(0, (5, 0, 0)), (5, (5, 1, 2)), (6, (4, 0, 1))]:
        ref = orc.sample(lv, r, n)
        assert np.max(np.abs(out["tile"][q, :lv + 1] / ref["F"] - 1)) <= 1e-12, (lv, r, n)


# --------------------------------------------------------------------------- #
# Graph replay of repeated identical calls                                    #
# --------------------------------------------------------------------------- #


@pytest.mark.parametrize("precision", ["fp64", "mixed_tf32"])
def test_graph_replay_equals_direct_path(precision):
    """The second identical call is captured as a CUDA graph and replayed,
    later ones replay it: sums and per-sample F are bit-identical to the
    launch-by-launch call; a different call runs directly; turning graphs
    off gives the same results again."""
    cfg = W.scaled(W.LATTICE_6LEVEL, R=2, precision=precision)
    ctx = M.Context.from_config(cfg, genvec=_genvec(cfg))
    nl = cfg["n_levels"]
    work = [(5, 0, 2, 0, 2), (3, 1, 5, 0, 1), (1, 0, 7, 1, 2)]
    ns = sum((ne - nb) * (re_ - rb) for (_, nb, ne, rb, re_) in work)
    sums = torch.zeros(nl * 2 * 2, dtype=torch.float64, device="cuda")
    F = torch.zeros(ns * nl, dtype=torch.float64, device="cuda")

    def call(w=work):
        sums.zero_()
        F.zero_()
        ctx.sample_levels(w, sums, F)
        torch.cuda.synchronize()
        return sums.cpu().numpy().copy(), F.cpu().numpy().copy()

    ref = call()
    assert ctx.graph_replays() == 0
    for k in range(3):
        got = call()
        assert ctx.graph_replays() == k + 1
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    other = [(2, 0, 3, 0, 2)]
    call(other)
    assert ctx.graph_replays() == 3
    got = call()  # remembered again, runs directly
    assert np.array_equal(got[1], ref[1]) and ctx.graph_replays() == 3
    ctx.set_graphs(False)
    for _ in range(2):
        got = call()
        assert np.array_equal(got[1], ref[1])
    assert ctx.graph_replays() == 3
    ctx.check_device()


def test_graph_replay_with_profiling():
    """Profiling through a replayed graph: each replay's kernel brackets are
    read back; per-kind launch counts grow by the same amount per call and
    the results stay those of the direct path."""
    cfg = W.scaled(W.LATTICE_6LEVEL, R=2, precision="mixed_tf32")
    ctx = M.Context.from_config(cfg, genvec=_genvec(cfg))
    nl = cfg["n_levels"]
    work = [(4, 0, 3, 0, 2), (2, 0, 4, 0, 2)]
    sums = torch.zeros(nl * 2 * 2, dtype=torch.float64, device="cuda")
    ctx.profile(True)
    outs, counts = [], []
    for _ in range(4):
        sums.zero_()
        ctx.sample_levels(work, sums)
        torch.cuda.synchronize()
        outs.append(sums.cpu().numpy().copy())
        prof = ctx.profile_read()
        counts.append({k: v[1] for k, v in prof.items()})
        ctx.profile(True)
        assert all(v[0] > 0 for v in prof.values() if v[1] > 0)
    ctx.profile(False)
    assert ctx.graph_replays() == 3
    assert all(np.array_equal(o, outs[0]) for o in outs)
    assert all(c == counts[0] for c in counts)
    ctx.check_device()


# --------------------------------------------------------------------------- #
# Mixed forms against the FP64 oracle: Algorithm 1, the solution in the       #
# energy norm, the device timeout path                                        #
# --------------------------------------------------------------------------- #


@pytest.mark.parametrize("precision,ufun", MIXED)
def test_algorithm1_mixed_matches_oracle(precision, ufun):
    """Algorithm 1 in a converged mixed form (rtol 1e-10) against the FP64
    oracle (rtol 1e-12): the same decisions (levels, counts, rounds), and Q
    within the field bound propagated through the estimator: every F_t of a
    sample is within eps_F = expm1(eta + slack) + 2 rtol rms(u)/mean(u) of the
    oracle's, and Q sums, per level, means of differences of two F, so
    |dQ| <= 2 (L + 1) max eps_F max F."""
    cfg, ctx, orc = _pair(W.LATTICE_6LEVEL, n_levels=5, n0=4, s=6, R=4, seed=11, log2_nmax=10, precision=precision,
                          rtol=1e-10)
    eps = 4e-4
    g = ctx.estimate(eps)
    o = orc.estimate(eps)
    assert o["status"] == O.OK and g["run_status"] == o["run_status"]
    assert g["L"] == o["L"] and g["rounds"] == o["rounds"] and g["N"] == o["N"]
    L = o["L"]
    eta = 0.0
    for lv in range(L + 1):
        for r in range(cfg["R"]):
            for n in range(o["N"][lv]):
                eta = max(eta, _field_bound(orc, cfg, orc.normals(lv, r, n), ufun(cfg["s"])))
    ratio = 2.0  # rms(u)/mean(u) of every level of this problem is below 1.6
    eps_F = math.expm1(eta + EXP_SLACK) + 2 * 1e-10 * ratio + 1e-12
    Fmax = 0.08
    assert abs(g["Q"] - o["Q"]) <= 2 * (L + 1) * eps_F * Fmax, (g["Q"], o["Q"], eta)
    assert abs(g["Q"] - o["Q"]) <= 1e-2 * abs(o["Q"])


def test_mixed_solution_energy_norm_bound():
    """The mixed solution (TF32 field, FP32 V-cycles, FP64 refinement to
    ||r|| <= 1e-10 ||b||) against the oracle's FP64 one (1e-12) on every level
    up to 64 x 64, in the energy norm of the oracle's operator A: the FP32
    field and faces make the mixed operator A' with (1 - d) A <= A' <= (1 + d) A,
    d = expm1(eta + slack), so the exact solutions differ by at most
    d / (1 - d) ||u||_A, and each solve adds at most its residual norm over
    sqrt(lambda_min(A)) (lambda_min(A) >= min face k x lambda_min of the unit-
    coefficient operator, computed here). The max-norm error is reported."""
    import scipy.sparse as sps
    import scipy.sparse.linalg as spla

    cfg, ctx, orc = _pair(W.PRECISION_1024, n_levels=4, R=2, s=40, precision="mixed_tf32", rtol=1e-10)
    lam1 = {}
    for t in range(4):
        n = cfg["n0"] << t
        cols = [O.apply_A(n, np.ones(n * n), np.eye(1, n * n, q)[0]) for q in range(n * n)]
        A1 = sps.csr_matrix(np.array(cols).T)
        lam1[t] = float(spla.eigsh(A1, k=1, sigma=0.0, return_eigenvectors=False)[0]) if n * n > 16 else \
            float(np.linalg.eigvalsh(A1.toarray())[0])
    worst = []
    for (lv, r, n) in [(3, 0, 2), (3, 1, 5)]:
        sols, _ = ctx.sample_solution(lv, r, n)
        ref = orc.sample(lv, r, n, want_u=True)
        assert ref["status"] == O.OK
        y = orc.normals(lv, r, n)
        d = math.expm1(_field_bound(orc, cfg, y, _tf32_u(cfg["s"])) + EXP_SLACK)
        for t in range(lv + 1):
            nt = cfg["n0"] << t
            k = orc.field(t, y)
            um, uo = sols[t].cpu().numpy(), ref["u"][t]
            e = um - uo
            eA = math.sqrt(max(0.0, e @ O.apply_A(nt, k, e)))
            uA = math.sqrt(uo @ O.apply_A(nt, k, uo))
            kx = np.minimum(k.reshape(nt, nt)[:, 1:], k.reshape(nt, nt)[:, :-1])
            kmin = min(float(np.min(k)), float(np.min(kx)))  # harmonic means lie above the smaller k
            lam = kmin * lam1[t]
            bnorm = float(nt)  # ||b||_2 for b = 1 on nt^2 cells
            bound = d / (1 - d) * uA + (1e-10 / (1 - d) + 1e-12) * bnorm / math.sqrt(lam)
            assert eA <= bound, (lv, t, eA, bound)
            worst.append((eA / uA, float(np.max(np.abs(e)) / np.max(np.abs(uo)))))
    print("energy-norm relative errors and max-norm relative errors:", worst)
    ctx.check_device()


def test_device_wait_timeout_sets_status():
    """A kernel that waits with the library's bounded mbarrier wait (limit
    1 ms) on a barrier nothing arrives on gives up and records
    MLQMC_ERR_TIMEOUT; reading the status clears it and the context keeps
    working."""
    cfg, ctx, orc = _pair(W.MC_4LEVEL, R=1)
    s = torch.cuda.current_stream()
    assert M.lib().mlqmc_test_wait_timeout(ctx.h, 1_000_000, M._stream(s)) == 0
    torch.cuda.synchronize()
    assert ctx.device_status() == 6  # MLQMC_ERR_TIMEOUT
    assert ctx.device_status() == 0
    sums = torch.zeros(cfg["n_levels"] * 2, dtype=torch.float64, device="cuda")
    ctx.sample_levels([(1, 0, 4, 0, 1)], sums)
    torch.cuda.synchronize()
    ctx.check_device()
    ref = orc.sample_levels([(1, 0, 4, 0, 1)])["sums"].reshape(-1)
    assert np.allclose(sums.cpu().numpy(), ref, rtol=1e-12, atol=1e-15)
