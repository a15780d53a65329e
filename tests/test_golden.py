"""Stored expected values (tests/golden/, written by tests/golden/make_golden.py
from the oracle alone): the oracle still reproduces them, the library's host
CBC matches them, and (GPU) the device lattice bits match them bit for bit and
the FP64 normals to 1e-14."""
import os

import numpy as np
import pytest

import oracle as O
import workloads as W

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLD, name)) as f:
        return [ln.split() for ln in f if not ln.startswith("#")]


def test_oracle_reproduces_the_stored_cbc_vector():
    rows = _rows("cbc_s100_m10.txt")
    z, e2 = O.cbc(100, 10)
    assert [int(r[1]) for r in rows] == [int(v) for v in z]
    assert [float.fromhex(r[2]) for r in rows] == [float(v) for v in e2]


def test_library_cbc_matches_the_stored_vector():
    M = pytest.importorskip("paper_1806_05619_gb300")
    z, _ = M.cbc_genvec(100, 10)
    assert [int(r[1]) for r in _rows("cbc_s100_m10.txt")] == [int(v) for v in z]


def test_oracle_reproduces_the_stored_points_and_normals():
    z = [int(r[1]) for r in _rows("cbc_s100_m10.txt")]
    cfg = W.LATTICE_6LEVEL
    orc = O.Oracle(n_levels=cfg["n_levels"], n0=cfg["n0"], s=cfg["s"], sampler="lattice", seed=cfg["seed"],
                   R=cfg["R"], genvec=z, log2_nmax=cfg["log2_nmax"])
    for lv, r, n, j, bits, y in _rows("lattice_bits_problem2.txt"):
        lv, r, n, j = int(lv), int(r), int(n), int(j)
        assert O.lattice_bits(z[j], n, O.shift_bits(cfg["seed"], lv, r, j)) == int(bits, 16)
        assert orc.normals(lv, r, n)[j] == float.fromhex(y)


@pytest.mark.gpu
def test_device_points_and_normals_match_the_stored_values():
    pytest.importorskip("torch")
    import paper_1806_05619_gb300 as M

    z = [int(r[1]) for r in _rows("cbc_s100_m10.txt")]
    ctx = M.Context.from_config(W.LATTICE_6LEVEL, genvec=z)
    for lv, r, n, j, bits, y in _rows("lattice_bits_problem2.txt"):
        lv, r, n, j = int(lv), int(r), int(n), int(j)
        b = int(ctx.point_bits(lv, r, n, 1).cpu().numpy()[0, j]) & 0xFFFFFFFFFFFFFFFF
        assert b == int(bits, 16), (lv, r, n, j)
        yg = float(ctx.normals(lv, r, n, 1).cpu().numpy()[0, j])
        assert abs(yg - float.fromhex(y)) <= 1e-14 * max(1.0, abs(float.fromhex(y))), (lv, r, n, j)
