"""Constants of the FP64 exponential in the device code (Tang's table-driven
method): the table holds 2^(j/64) rounded to nearest, the reduction splits
ln2/64 into a 32-bit head and a tail, and 64/ln2 is rounded to nearest.
Checked against 60-digit decimal arithmetic; no GPU needed."""
import os
import re
from decimal import Decimal, getcontext

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_1806_05619_gb300", "csrc", "fmg_device.cuh")


def _source():
    with open(SRC) as f:
        return f.read()


def _ln2():
    getcontext().prec = 60
    return Decimal(2).ln()


def test_exp2_table_is_correctly_rounded():
    body = re.search(r"kExp2Tab\[64\] = \{(.*?)\};", _source(), re.S).group(1)
    vals = [float.fromhex(v) for v in re.findall(r"0x[0-9a-fA-F.]+p[+-]\d+", body)]
    assert len(vals) == 64
    ln2 = _ln2()
    for j, v in enumerate(vals):
        exact = (ln2 * j / 64).exp()
        assert v == float(exact), j  # float(Decimal) rounds to nearest


def test_reduction_constants():
    src = _source()

    def const(name):
        return float.fromhex(re.search(name + r" = (0x[0-9a-fA-F.]+p[+-]\d+);", src).group(1))

    ln2 = _ln2()
    inv_l, l1, l2 = const("kInvL"), const("kL1"), const("kL2")
    assert inv_l == float(64 / ln2)
    m = int(l1 * 2.0 ** 38)  # kL1 = m * 2^-38 with m below 2^32: products n * kL1 exact for |n| < 2^21
    assert m * 2.0 ** -38 == l1 and m < 2 ** 32
    assert abs(Decimal(l1) + Decimal(l2) - ln2 / 64) < Decimal(2) ** -90
