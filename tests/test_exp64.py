"""The FP64 attenuation factor e^{-x} of Eq. 3 (table-driven, Tang 1989).

CPU: the constants in moc_exp64.cuh against their definitions, computed in
60-digit decimal arithmetic (2^{j/64} = hi + lo, ln2/64 = hi + lo with a
29-bit hi, 64/ln2, 1/k!).  GPU: the device function against e^{-x} in long
double, within 1 ulp over |x| < 700, next to CUDA's exp(-x); 0 at and above
x = 700, NaN passed through."""
import os
import re
from decimal import Decimal, getcontext

import numpy as np
import pytest

HDR = os.path.join(os.path.dirname(__file__), "..", "paper_2503_17743_gb300", "csrc", "moc_exp64.cuh")
HEX = r"(-?0x[0-9a-fA-F.]+p[+-]?\d+|0\.0)"


def header():
    return open(HDR).read()


def constant(name):
    m = re.search(r"constexpr double %s = %s;" % (name, HEX), header())
    assert m, name
    return float.fromhex(m.group(1))


def table():
    body = header().split("kTable[64] = {", 1)[1].split("};", 1)[0]
    rows = re.findall(r"\{%s, %s\}" % (HEX, HEX), body)
    return [(float.fromhex(a), float.fromhex(b)) for a, b in rows]


def D(v):
    return Decimal(v)  # exact value of a double


def test_table_is_two_to_the_j_over_64():
    getcontext().prec = 60
    rows = table()
    assert len(rows) == 64
    for j, (hi, lo) in enumerate(rows):
        exact = Decimal(2) ** (Decimal(j) / Decimal(64))
        assert hi == float(exact), j  # hi: the nearest double
        assert lo == float(exact - D(hi)), j  # lo: the nearest double to the rest
        assert abs(D(hi) + D(lo) - exact) < Decimal(2) ** -105


def test_reduction_constants():
    getcontext().prec = 60
    ln2 = Decimal(2).ln()
    hi, lo = constant("kStepHi"), constant("kStepLo")
    # hi: ln2/64 to the nearest double with the low 24 of its 52 fraction
    # bits cleared (29 significant bits: n * hi exact for |n| < 2^24)
    bits = int(np.float64(float(ln2 / 64)).view(np.uint64))
    assert hi == float(np.uint64(bits >> 24 << 24).view(np.float64))
    assert lo == float(ln2 / 64 - D(hi))  # lo: the nearest double to the rest
    assert constant("kInvStep") == float(64 / ln2)
    assert constant("kShift") == 1.5 * 2.0 ** 52
    fact = {2: 2, 3: 6, 4: 24, 5: 120}
    for k, f in fact.items():
        assert constant("kC%d" % k) == float(Decimal(1) / f)
    assert int(re.search(r"kHiCut = (0x[0-9A-Fa-f]+)", header()).group(1), 16) == \
        int(np.float64(700.0).view(np.uint64)) >> 32


def ulp_error(y, x):
    exact = np.exp(-x.astype(np.longdouble))
    ulp = np.spacing(exact.astype(np.float64))
    return np.abs((y.astype(np.longdouble) - exact) / ulp.astype(np.longdouble)).astype(np.float64)


@pytest.mark.gpu
def test_device_exp_within_one_ulp():
    from paper_2503_17743_gb300 import eval_attenuation_f64
    if np.finfo(np.longdouble).nmant < 60:
        pytest.skip("long double has no more precision than double here")
    rng = np.random.default_rng(17)
    x = np.concatenate([
        rng.uniform(0.0, 1.0, 400000),
        rng.uniform(0.0, 40.0, 400000),
        rng.uniform(0.0, 699.9, 200000),
        np.ldexp(rng.uniform(0.5, 1.0, 100000), -rng.integers(1, 60, 100000)),
        # around the reduction's break points n ln2 / 64 +- ln2 / 128
        (np.arange(1, 20001) + 0.5) * np.log(2.0) / 64 * (1 + rng.uniform(-1e-12, 1e-12, 20000)),
        np.array([0.0, 5e-324, 1e-300, 699.0, 699.99]),
    ])
    y, y_lib = eval_attenuation_f64(x)
    err = ulp_error(y, x)
    err_lib = ulp_error(y_lib, x)
    assert err.max() <= 1.0, (err.max(), x[err.argmax()])
    assert err_lib.max() <= 1.0 + 1e-9  # CUDA's stated bound for exp, as a check of the measure
    assert y[x == 0.0][0] == 1.0
    assert np.all(np.diff(y[:400000][np.argsort(x[:400000])]) <= 0.0)  # monotone on [0, 1)


@pytest.mark.gpu
def test_device_exp_outside_domain():
    from paper_2503_17743_gb300 import eval_attenuation_f64
    x = np.array([700.0, 745.2, 1e6, 1e300, np.inf, np.nan, -np.nan])
    y, y_lib = eval_attenuation_f64(x)
    assert np.all(y[:5] == 0.0)
    assert np.isnan(y[5]) and np.isnan(y[6])
    assert np.all(eval_attenuation_f64(np.zeros(0))[0].shape == (0,))
