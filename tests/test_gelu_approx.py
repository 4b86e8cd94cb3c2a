"""The erf of the tcgen05 FFN kernel's GELU epilogue (csrc/pt_gemm_tc.cu, gelu_erf2):
Abramowitz and Stegun, Handbook of Mathematical Functions, formula 7.1.26,
erf(a) = 1 - (a1 t + a2 t^2 + a3 t^3 + a4 t^4 + a5 t^5) exp(-a^2), t = 1 / (1 + p a), a >= 0, with
the handbook's error bound 1.5e-7. The coefficients below are read from the kernel's source, so a
mistyped digit there fails this test; the bound is checked against math.erf on a dense grid, and
the resulting GELU against the erf form within the bfloat16 rounding the kernel applies after it."""
import math
import re
from pathlib import Path

import numpy as np

SRC = Path(__file__).resolve().parents[1] / "paper_2509_23043_gb300" / "csrc" / "pt_gemm_tc.cu"


def _coefficients():
    body = SRC.read_text()
    body = body[body.index("__device__ __forceinline__ void gelu_erf2"):]
    body = body[:body.index("\n}\n")]
    nums = [float(x) for x in re.findall(r"[-+]?\d+\.\d+(?:e[-+]?\d+)?", body)]
    # in order of appearance: 1/sqrt 2, p, then a5, a4, a3, a2, a1 (Horner order)
    return nums


def test_coefficients_are_the_handbooks():
    nums = _coefficients()
    assert nums[0] == 0.70710678118654752
    p, a5, a4, a3, a2, a1 = nums[1], nums[2], nums[3], nums[4], nums[5], nums[6]
    assert (p, a1, a2, a3, a4, a5) == (0.3275911, 0.254829592, -0.284496736, 1.421413741,
                                       -1.453152027, 1.061405429)


def test_erf_within_the_published_bound():
    p, a5, a4, a3, a2, a1 = _coefficients()[1:7]
    a = np.linspace(0.0, 6.0, 300001)
    t = 1.0 / (1.0 + p * a)
    poly = ((((a5 * t + a4) * t + a3) * t + a2) * t + a1) * t        # the kernel's Horner order
    e = 1.0 - poly * np.exp(-a * a)
    ref = np.array([math.erf(x) for x in a])
    assert np.abs(e - ref).max() <= 1.5e-7


def test_gelu_within_bfloat16_rounding():
    p, a5, a4, a3, a2, a1 = _coefficients()[1:7]
    x = np.linspace(-8.0, 8.0, 160001)
    a = np.abs(x) / math.sqrt(2.0)
    t = 1.0 / (1.0 + p * a)
    poly = ((((a5 * t + a4) * t + a3) * t + a2) * t + a1) * t
    g = 0.5 * x * (1.0 + np.copysign(1.0 - poly * np.exp(-a * a), x))
    ref = np.array([0.5 * v * (1.0 + math.erf(v / math.sqrt(2.0))) for v in x])
    err = np.abs(g - ref)
    # the erf bound carried through GELU: |error| <= |x| / 2 * 1.5e-7 (+ float64 rounding)
    assert np.all(err <= 0.5 * np.abs(x) * 1.5e-7 + 1e-15)
    # and within an eighth of a bfloat16 unit of the result (relative 2^-9 / 8), the relative
    # error being largest in the negative tail, where 1 + erf cancels
    assert np.all(err <= 2.0 ** -9 / 8 * np.maximum(np.abs(ref), 1e-3))
