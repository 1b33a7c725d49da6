"""The float-float helpers of the reaction kernels (split of a double into
a float pair on its bit pattern, exact widening of a float, float-float sum
and products), run on the host against exact rational arithmetic (no GPU
needed)."""
import math
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2104_05024_gb300", "csrc")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("ffloat") / "ffloat_host")
    subprocess.run(["g++", "-O2", "-std=c++17", "-fno-strict-aliasing", "-ffp-contract=off", "-I", CSRC,
                    os.path.join(HERE, "host", "ffloat_host.cpp"), "-o", exe], check=True)
    return exe


def _inputs():
    rng = np.random.default_rng(5)
    xs = list(rng.uniform(-1.5, 1.5, 4000))
    xs += list(rng.choice([-1.0, 1.0], 4000) * 10.0 ** rng.uniform(-25, 28, 4000))
    xs += [0.0, -0.0, 1.0, -1.0, 0.1, 2.0 ** -60, -(2.0 ** -60), 2.0 ** -61, 2.0 ** -60 * (1 - 2 ** -52),
           2.0 ** 99 * 1.75, 2.0 ** 100, -(2.0 ** 100), 2.0 ** 127 * 1.999, 2.0 ** 128, -(2.0 ** 129),
           1e300, math.inf, -math.inf, math.nan,
           1.0 + 2.0 ** -52, 1.0 - 2.0 ** -53, float.fromhex("0x1.fffffffffffffp-1"),
           float.fromhex("0x1.00000ffffffffp0"), float.fromhex("0x1.000001fffffffp0")]
    return xs


def test_split_widen_and_products_exact_bounds(harness):
    xs = _inputs()
    inp = "\n".join(repr(float(x)) if math.isfinite(x) else ("nan" if math.isnan(x) else ("inf" if x > 0 else "-inf"))
                    for x in xs)
    out = subprocess.run([harness], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    u = Fraction(1, 2 ** 24)
    for x, line in zip(xs, out):
        f = line.split()
        ok = f[0] == "1"
        h, l, hw, sh, sl, qh, ql, rh, rl, nw = (float.fromhex(t) if t not in ("nan", "-nan") else math.nan
                                                for t in f[1:])
        if not math.isfinite(x) or abs(x) >= 2.0 ** 128:
            assert not ok, x
            # narrowing: infinities, NaN for NaN
            assert math.isnan(nw) if math.isnan(x) else nw == math.copysign(math.inf, x)
            continue
        assert ok, x
        if abs(x) < 2.0 ** -60:
            assert h == 0.0 and l == 0.0 and nw == 0.0, x
            continue
        # narrowing: the nearest float, or a neighbour of it within 2^-48 |x| of a tie
        if abs(x) < 2.0 ** 127:
            near = float(np.float32(x))
            assert nw == near or (abs(Fraction(x) - (Fraction(near) + Fraction(nw)) / 2)
                                  <= abs(Fraction(x)) * Fraction(1, 2 ** 48)), (x, nw, near)
        X = Fraction(x)
        H, L = Fraction(h), Fraction(l)
        # hi: x truncated to 24 significant bits
        assert abs(H) <= abs(X) and abs(X - H) < Fraction(2) ** (math.frexp(x)[1] - 24), x
        assert h == 0.0 or math.copysign(1.0, h) == math.copysign(1.0, x)
        # hi + lo within 2^-48 |x|
        assert abs(X - (H + L)) <= abs(X) * u * u, x
        # widening is exact
        assert hw == h
        P = H + L
        # float-float sum and products within a few units of 2^-48 of the
        # exact values, while they stay in the float range (the reaction's
        # values are O(1); an absolute slack covers products near the
        # subnormal floats)
        if abs(x) > 2.0 ** 60:
            continue
        for (a, b), ref in (((sh, sl), 2 * P), ((qh, ql), P * P), ((rh, rl), P * H)):
            got = Fraction(a) + Fraction(b)
            assert abs(got - ref) <= abs(ref) * 8 * u * u + Fraction(1, 2 ** 140), (x, float(got), float(ref))
