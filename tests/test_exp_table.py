"""The float64 trace kernel's table-driven exponential (csrc/exp_tang.cuh,
Tang's method with 64 entries) on the CPU: its table holds the float64
values nearest to 2^(j/64), its reduction constants split ln2/64 as stated,
and the algorithm, emulated step by step with exactly rounded fused
multiply-adds, stays within 2 ulp of e^x computed to 40 digits."""
import math
import os
import random
import re
from decimal import Decimal, getcontext
from fractions import Fraction

HDR = os.path.join(os.path.dirname(__file__), "..", "paper_2010_08482_gb300", "csrc", "exp_tang.cuh")
getcontext().prec = 50


def _header():
    with open(HDR) as f:
        return f.read()


def _table():
    body = _header().split("kExp2Frac64[64] = {", 1)[1].split("};", 1)[0]
    return [float.fromhex(t) for t in re.findall(r"0x[0-9a-fA-F.]+p[+-]\d+", body)]


def _const(name):
    m = re.search(name + r"\s*=\s*(0x[0-9a-fA-F.]+p[+-]?\d+)", _header())
    return float.fromhex(m.group(1))


def _fma(a, b, c):
    """fl(a b + c) with one rounding (exact rationals, correctly rounded)."""
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def _exp_nonpos(x, tab):
    """The device function's steps, in the same order and roundings."""
    inv, hi, lo, sh = _const("INV_STEP"), _const("STEP_HI"), _const("STEP_LO"), float.fromhex("0x1.8p52")
    if not x >= -745.2:
        return x if x != x else 0.0
    t = _fma(x, inv, sh)
    n = int(t - sh)  # exact: the low bits of t
    nd = t - sh
    r = _fma(-nd, hi, x)
    r = _fma(-nd, lo, r)
    q = _fma(r, 1.0 / 120.0, 1.0 / 24.0)
    for c in (1.0 / 6.0, 0.5, 1.0, 1.0):
        q = _fma(r, q, c)
    j, m = n & 63, n >> 6
    v = tab[j] * q
    if m >= -1020:
        return math.ldexp(v, m)  # exact: the result stays normal
    return float(Fraction(v) * Fraction(2) ** (m + 60) * Fraction(1, 2 ** 60))


def _ulps(a, ref):
    return abs(Fraction(a) - ref) / Fraction(math.ulp(float(ref)))


def test_table_is_nearest_to_the_exact_powers():
    tab = _table()
    assert len(tab) == 64
    for j, v in enumerate(tab):
        exact = Decimal(2) ** (Decimal(j) / 64)
        assert v == float(exact), j  # float(Decimal) rounds to nearest


def test_reduction_constants():
    hi, lo, inv = _const("STEP_HI"), _const("STEP_LO"), _const("INV_STEP")
    step = Decimal(2).ln() / 64
    mant = Fraction(hi) / Fraction(2) ** (math.frexp(hi)[1] - 53)
    assert mant.denominator == 1 and int(mant) % (1 << 21) == 0  # at most 32 significant bits
    assert abs(Decimal(hi) + Decimal(lo) - step) <= Decimal(math.ulp(lo)) / 2  # lo rounded to nearest
    assert abs(Decimal(inv) - 1 / step) < Decimal(10) ** -14


def test_algorithm_within_two_ulp():
    tab = _table()
    rng = random.Random(2010)
    xs = [0.0, -0.0, -1e-300, -1e-17, -0.0054, -0.0109, -math.log(2) / 128, -1.0, -math.log(2), -700.0,
          -708.4, -709.0, -744.0, -745.1]
    xs += [-rng.uniform(0, 1) for _ in range(300)] + [-rng.uniform(0, 50) for _ in range(300)]
    xs += [-rng.uniform(700, 745) for _ in range(100)]
    worst = 0.0
    for x in xs:
        got = _exp_nonpos(x, tab)
        ref = Fraction(Decimal(x).exp())
        if ref < Fraction(2) ** -1022:  # subnormal results: absolute error within 1 ulp of the smallest normal
            assert abs(Fraction(got) - ref) <= Fraction(2) ** -1074, x
            continue
        u = float(_ulps(got, ref))
        worst = max(worst, u)
        assert u <= 2.0, (x, u)
    assert _exp_nonpos(-746.0, tab) == 0.0 and _exp_nonpos(-math.inf, tab) == 0.0
    assert math.isnan(_exp_nonpos(math.nan, tab))
    print(f"\nworst {worst:.2f} ulp over {len(xs)} arguments")
