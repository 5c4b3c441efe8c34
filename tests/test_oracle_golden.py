"""The oracle still reproduces its stored regression values
(tests/golden/oracle_2d32_rk4.txt, written by tests/golden/make_golden.py)."""
import os
import re
import sys

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_matches_its_regression_fixture():
    sys.path.insert(0, os.path.join(HERE, "golden"))
    import make_golden

    stored = open(os.path.join(HERE, "golden", "oracle_2d32_rk4.txt")).read().split("\n")
    got = make_golden.compute()
    num = re.compile(r"=(-?[0-9.e+-]+)")
    for a, b in zip(got, stored):
        assert a.split("=")[0] == b.split("=")[0]
        for x, y in zip(num.findall(a), num.findall(b)):
            if "." in x or "e" in x:
                assert abs(float(x) - float(y)) <= 1e-13 * max(1.0, abs(float(y))), (a, b)
            else:
                assert x == y
