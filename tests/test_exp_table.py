"""The 2^(j/64) double-double table of the table-driven exp (Tang 1989) against
a 60-digit decimal evaluation."""
import os
import re
from decimal import Decimal, getcontext

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_exp_table_entries():
    src = open(os.path.join(ROOT, "paper_2210_07094_gb300", "csrc", "fastexp.cuh")).read()
    rows = re.findall(r"\{(-?0x[0-9a-fp.+-]+), (-?0x[0-9a-fp.+-]+)\}", src)
    assert len(rows) == 64
    getcontext().prec = 60
    ln2 = Decimal(2).ln()
    for j, (hi, lo) in enumerate(rows):
        exact = (Decimal(j) / 64 * ln2).exp()
        h, l = float.fromhex(hi), float.fromhex(lo)
        assert h == float(exact)                       # hi rounded to nearest
        assert abs(Decimal(h) + Decimal(l) - exact) < Decimal(2) ** -104
    L1 = float.fromhex(re.search(r"L1 = (0x[0-9a-fp.+-]+)", src).group(1))
    L2 = float.fromhex(re.search(r"L2 = (0x[0-9a-fp.+-]+)", src).group(1))
    assert abs(Decimal(L1) + Decimal(L2) - ln2 / 64) < Decimal(2) ** -110
