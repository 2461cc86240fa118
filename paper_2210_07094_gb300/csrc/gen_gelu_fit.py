"""Coefficients of the GELU's normal-tail exponent in tc_gemm.cuh.

Phi(-a) = 2^(-a^2 log2(e) / 2 + Q(a)) for a >= 0, with
Q(a) = log2(Phi(-a)) + a^2 log2(e) / 2, a smooth, slowly varying function
(-1 at a = 0, about -3.3 at a = 4).  Q is interpolated on [0, A] at the
Chebyshev points of the variable x = 2a/A - 1 by a polynomial of degree D,
then converted to monomials in x for Horner evaluation in FP32.
log_ndtr (scipy) gives log Phi to full double precision.

    python gen_gelu_fit.py        # prints the table and its FP32 error
"""
import numpy as np
from numpy.polynomial import chebyshev as cheb
from scipy.special import log_ndtr, ndtr

A, D = 4.0, 8
L2E = 1.0 / np.log(2.0)


def fit():
    x = np.cos(np.pi * (np.arange(4096) + 0.5) / 4096)
    a = (x + 1.0) * A / 2.0
    q = log_ndtr(-a) * L2E + 0.5 * a * a * L2E
    return cheb.cheb2poly(cheb.chebfit(x, q, D)).astype(np.float32)


def fp32_error(c):
    a = np.linspace(0.0, A, 400001)
    x = (a / np.float32(A / 2.0) - np.float32(1.0)).astype(np.float32)
    acc = np.float32(c[-1])
    for k in range(D - 1, -1, -1):
        acc = (acc * x + c[k]).astype(np.float32)
    e = (acc - np.float32(0.5 * L2E) * (a.astype(np.float32) ** 2)).astype(np.float32)
    return np.max(np.abs(np.exp2(e.astype(np.float64)) / ndtr(-a) - 1.0))


if __name__ == "__main__":
    c = fit()
    for k, v in enumerate(c):
        print(f"  c[{k}] = {float(v)!r}f")
    print("max relative error of Phi(-a) on [0, A] in FP32 Horner:", fp32_error(c))
