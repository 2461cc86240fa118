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
    # the reduction constants of both tables: L1 + L2 = ln 2 / 2^B, INV_L = 2^B / ln 2
    m = re.search(r"INV_L = B == 8 \? (0x[0-9a-fp.+-]+) : (0x[0-9a-fp.+-]+);", src)
    l1 = re.search(r"L1 = B == 8 \? (0x[0-9a-fp.+-]+) : (0x[0-9a-fp.+-]+);", src)
    l2 = re.search(r"L2 = B == 8 \? (0x[0-9a-fp.+-]+) : (0x[0-9a-fp.+-]+);", src)
    for g, B in ((1, 8), (2, 6)):
        inv = float.fromhex(m.group(g))
        L1, L2 = float.fromhex(l1.group(g)), float.fromhex(l2.group(g))
        assert inv == float(Decimal(2 ** B) / ln2)
        assert abs(Decimal(L1) + Decimal(L2) - ln2 / 2 ** B) < Decimal(2) ** -(104 + B)


def test_exp_table256_entries():
    """The 256-entry table of the generated kernels (fastexp_table256.inc,
    written by gen_exptab.py) against a 60-digit evaluation of 2^(j/256)."""
    src = open(os.path.join(ROOT, "paper_2210_07094_gb300", "csrc", "fastexp_table256.inc")).read()
    rows = re.findall(r"\{(-?0x[0-9a-fp.+-]+), (-?0x[0-9a-fp.+-]+)\}", src)
    assert len(rows) == 256
    getcontext().prec = 60
    ln2 = Decimal(2).ln()
    for j, (hi, lo) in enumerate(rows):
        exact = (Decimal(j) / 256 * ln2).exp()
        h, l = float.fromhex(hi), float.fromhex(lo)
        assert h == float(exact)
        assert abs(Decimal(h) + Decimal(l) - exact) < Decimal(2) ** -104
