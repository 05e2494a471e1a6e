"""The FP32 erfc of the formal-solve kernel against scipy (CPU).

The kernel evaluates erfc(|x|) = exp(-x^2) t P(2t - 1), t = 1/(1 + 0.4|x|),
with the coefficients written in mgt_erfc.cuh; here the same coefficients, read
from the source, are evaluated in FP32 Horner form and compared with
scipy.special.erfcx / erfc.
"""
import os
import re
import sys

import numpy as np
from scipy.special import erfc, erfcx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2411_03040_gb300", "csrc")
sys.path.insert(0, CSRC)
import fit_erfcx  # noqa: E402


def kernel_coefficients():
    src = open(os.path.join(CSRC, "mgt_erfc.cuh")).read()
    body = src[src.index("float kErfcP[11] = {"):]
    body = body[:body.index("};")]
    vals = [float(v) for v in re.findall(r"([-+]?\d\.\d+e[-+]\d+)f", body)]
    assert len(vals) == 11
    # the array lists the leading (highest-degree) coefficient first
    return np.array(vals[::-1])


def test_kernel_coefficients_match_the_fit():
    np.testing.assert_allclose(kernel_coefficients(), fit_erfcx.fit(), rtol=1e-8, atol=1e-12)


def test_scaled_form_relative_error():
    c = kernel_coefficients()
    x = np.linspace(0.0, 9.5, 200001)
    rel = np.abs(fit_erfcx.eval_fp32(c, x) / erfcx(x) - 1)
    assert rel.max() < 5e-7


def test_erfc_with_fp32_exponential():
    c = kernel_coefficients()
    x = np.linspace(-6.0, 6.0, 120001).astype(np.float32)
    ax = np.abs(x)
    r = fit_erfcx.eval_fp32(c, ax) * np.exp(-(ax * ax).astype(np.float32)).astype(np.float32)
    got = np.where(x < 0, np.float32(2.0) - r, r).astype(np.float64)
    ref = erfc(x.astype(np.float64))
    rel = np.abs(got / ref - 1)
    # exp(-x^2) with x^2 rounded to FP32: relative error up to about |x|^2 * 6e-8
    assert np.all(rel < 5e-7 + 1.2e-7 * ax.astype(np.float64) ** 2)
