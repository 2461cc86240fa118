"""Writes fastlog_table.inc: the 128-entry table of the table-driven logarithm
in fastlog.cuh.  Entry j covers mantissas y in [1 + j/128, 1 + (j+1)/128):
r_j is the double nearest to 1/F_j with F_j = 1 + (j + 1/2)/128, and
-ln(r_j) of that exact double is evaluated with 60 significant digits and
split into a double-double (hi + lo).  Also ln 2 split so that m * hi is exact
for |m| <= 1100.  Run from this directory: python gen_logtab.py"""
import mpmath as mp

mp.mp.dps = 60


def dd(v):
    hi = float(v)
    lo = float(v - mp.mpf(hi))
    return hi, lo


def main():
    out = ["// generated by gen_logtab.py: {r_j, -ln(r_j) hi, -ln(r_j) lo}"]
    for j in range(128):
        F = mp.mpf(1) + (mp.mpf(j) + mp.mpf("0.5")) / 128
        r = float(1 / F)
        hi, lo = dd(-mp.log(mp.mpf(r)))
        out.append(f"    {{{r.hex()}, {hi.hex()}, {lo.hex()}}},")
    ln2 = mp.log(2)
    # ln2_hi with its 12 lowest mantissa bits zero
    hi = float(ln2)
    m, e = mp.frexp(mp.mpf(hi))
    hi = float(mp.ldexp(mp.floor(mp.ldexp(m, 41)), e - 41))
    lo = float(ln2 - mp.mpf(hi))
    out.append(f"// ln 2 = LN2_HI + LN2_LO: {hi.hex()} {lo.hex()}")
    with open("fastlog_table.inc", "w") as f:
        f.write("\n".join(out) + "\n")


if __name__ == "__main__":
    main()
