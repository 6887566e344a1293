"""The arithmetic probes on the GPU: the float64 trace kernel's table
exponential against the CUDA library's exp and against e^x to 40 digits,
and the pipe-rate probes (FP64 FMA, FP32 FMA, FP64 warp-level MMA) return
plausible rates."""
import math
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

from paper_2010_08482_gb300 import ctq

pytestmark = pytest.mark.gpu
getcontext().prec = 50


def test_table_exponential_against_library_and_exact():
    rng = np.random.default_rng(7)
    x = np.concatenate([[0.0, -0.0, -1e-300, -1e-17, -708.4, -745.1, -746.0, -np.inf],
                        -rng.uniform(0, 1, 20000), -rng.uniform(0, 60, 20000), -rng.exponential(5.0, 20000),
                        -rng.uniform(600, 745, 2000)])
    yt, yl = ctq.probe_exp(x)
    normal = yl >= 2.0 ** -1022
    ulp = np.spacing(yl[normal])
    d_lib = np.abs(yt[normal] - yl[normal]) / ulp
    assert d_lib.max() <= 3.0, d_lib.max()  # each within 2 ulp (table) and 1 ulp (library) of e^x
    assert np.all(np.abs(yt[~normal] - yl[~normal]) <= 2.0 ** -1073)
    assert yt[6] == 0.0 and yt[7] == 0.0 and yt[0] == 1.0 and yt[1] == 1.0  # e^-746, e^-inf, e^0, e^-0
    worst = 0.0
    for k in rng.choice(np.nonzero(normal)[0], 400, replace=False):
        ref = Fraction(Decimal(float(x[k])).exp())
        worst = max(worst, float(abs(Fraction(float(yt[k])) - ref) / Fraction(math.ulp(float(ref)))))
    assert worst <= 2.0, worst
    print(f"\ntable exp: max {d_lib.max():.1f} ulp from the library's exp, max {worst:.2f} ulp from e^x (sample)")


def test_pipe_rate_probes():
    r64 = ctq.probe_fma_rate(0, 0)
    r32 = ctq.probe_fma_rate(0, 1)
    rmma = ctq.probe_fma_rate(0, 2, iters=4000)
    print(f"\nFP64 FMA {r64 / 1e12:.3f} TFLOP/s, FP32 FMA {r32 / 1e12:.1f} TFLOP/s, "
          f"FP64 mma.sync.m8n8k4 {rmma / 1e12:.3f} TFLOP/s")
    assert r64 > 1e11 and r32 > r64 and rmma > 1e11
