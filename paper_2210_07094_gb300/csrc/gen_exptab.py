"""Writes fastexp_table256.inc: the 256-entry table 2^(j/256), j = 0..255, of
the table-driven exponential in fastexp.cuh (the variant with a degree-4
polynomial), each entry a double-double: hi the double nearest to the value
evaluated with 60 significant digits, lo the double nearest to the
remainder.  Run from this directory: python gen_exptab.py"""
from decimal import Decimal, getcontext

getcontext().prec = 60


def nearest(v: Decimal) -> float:
    # float(Decimal) rounds to nearest
    return float(v)


def main():
    ln2 = Decimal(2).ln()
    out = ["// generated by gen_exptab.py: {2^(j/256) hi, lo}"]
    for j in range(256):
        v = (Decimal(j) / 256 * ln2).exp()
        hi = nearest(v)
        lo = nearest(v - Decimal(hi))
        out.append(f"    {{{hi.hex()}, {lo.hex()}}},")
    with open("fastexp_table256.inc", "w") as f:
        f.write("\n".join(out) + "\n")


if __name__ == "__main__":
    main()
