"""Fit the FP32 complementary error function used by the formal-solve kernel.

erfc(x) = exp(-x^2) * erfcx(x) for x >= 0, and erfcx(x) = t P(s) with
t = 1 / (1 + 0.4 x) and s = 2 t - 1 in [-1, 1].  P is a degree-10 polynomial
from a relative-error-weighted Chebyshev least-squares fit of erfcx(x) / t
(scipy.special.erfcx) on t in (0, 1], returned in monomial form in s for a
Horner evaluation.  Prints the coefficients (lowest degree first) and the
maximum relative error of an FP32 Horner evaluation on [0, 9.5].

    python paper_2411_03040_gb300/csrc/fit_erfcx.py
"""
import numpy as np
from numpy.polynomial import chebyshev as C
from scipy.special import erfcx

P_SCALE = 0.4
DEGREE = 10


def fit():
    t = np.linspace(1e-5, 1.0, 40001)
    x = (1.0 / t - 1.0) / P_SCALE
    y = erfcx(x) / t
    cf = C.chebfit(2.0 * t - 1.0, y, DEGREE, w=1.0 / y)
    return C.cheb2poly(cf)


def eval_fp32(coef, x):
    x = np.asarray(x, np.float32)
    t = (np.float32(1.0) / (np.float32(1.0) + np.float32(P_SCALE) * np.abs(x))).astype(np.float32)
    s = (np.float32(2.0) * t - np.float32(1.0)).astype(np.float32)
    c = np.asarray(coef, np.float32)
    acc = np.full_like(s, c[-1])
    for k in c[-2::-1]:
        acc = (acc * s + k).astype(np.float32)
    return (t * acc).astype(np.float32)


if __name__ == "__main__":
    coef = fit()
    xx = np.linspace(0.0, 9.5, 400001)
    rel = np.abs(eval_fp32(coef, xx).astype(np.float64) / erfcx(xx) - 1.0)
    print("coefficients:", ", ".join(f"{c:.9e}f" for c in coef))
    print("max relative error (fp32 Horner):", rel.max())
