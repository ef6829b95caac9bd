"""The parameter rule of Sec. 5.6 (evaluate.params) against every (instance,
n, c_d, c_b) row of Table 7 and every entry of Table 3, with d and log2 b
evaluated by hand from the printed formula (tests/golden/param_rule.txt)."""
import math
import os

import pytest

from paper_2601_09477_gb300 import evaluate

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "param_rule.txt")


def _rows():
    out = []
    with open(GOLDEN) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            name, n, cd, cb, d, L = line.split()[:6]
            out.append((name, int(n), float(cd), float(cb), int(d), int(L)))
    return out


ROWS = _rows()


def test_golden_covers_both_tables():
    assert len(ROWS) == 27 + 9
    assert {r[0] for r in ROWS} == {"logunit", "diagonal", "covariance", "lightbulb"}


@pytest.mark.parametrize("name,n,c_d,c_b,d,log2b", ROWS)
def test_params_match_tables(name, n, c_d, c_b, d, log2b):
    assert evaluate.params(n, c_d, c_b) == (d, log2b)
    # every row's b = c_b n is already a power of two: no rounding was applied
    assert (1 << log2b) == c_b * n
    assert d % 2 == 1


def test_formula_reading_not_the_words():
    # "the next odd number >= c_d log2 n" would give 5 at n = 2^15, c_d = 0.25
    # (3.75 -> 5); the printed formula gives 3 (reading c9)
    d, _ = evaluate.params(1 << 15, 0.25, 0.25)
    assert d == 3
    words = lambda x: int(math.ceil(x)) | 1
    assert words(0.25 * 15) == 5
