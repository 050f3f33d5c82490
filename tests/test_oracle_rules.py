"""Pins of the oracle's quadrature rules against closed forms (CPU).

- 7-point rule (Sec. 3.1 footnote): exact for total degree <= 3 on the
  reference triangle; the printed weights; not exact for degree 4.
- 16-point conical product rule (reading of the unspecified 16-point rule):
  exact for total degree <= 7, not for 8.
- 5-point Gauss-Legendre on (0,1) (Sec. 3.1: tensor rule for the transforms):
  exact for degree <= 9 against int_0^1 x^n = 1/(n+1).
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import rules as R

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))


def mono_exact(a, b):
    # int over {x, y >= 0, x + y <= 1} of x^a y^b = a! b! / (a + b + 2)!
    return math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)


def integrate(rule, a, b):
    x = rule[:, 1]
    y = rule[:, 2]
    return float(np.sum(rule[:, 3] * x ** a * y ** b))


@pytest.mark.parametrize("n,deg", [(7, 3), (16, 7)])
def test_rule_exact_up_to_degree(n, deg):
    q = R.rule(n)
    assert q.shape == (n, 4)
    assert np.allclose(q[:, :3].sum(1), 1.0, atol=2e-16)
    assert abs(q[:, 3].sum() - 0.5) < 1e-16
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            assert abs(integrate(q, a, b) - mono_exact(a, b)) < 2e-16, (a, b)
    worst = max(abs(integrate(q, a, deg + 1 - a) - mono_exact(a, deg + 1 - a)) for a in range(deg + 2))
    assert worst > 1e-8  # the degree is exactly deg, so a dropped point or weight would show


def test_rule7_weights_match_paper():
    q = R.rule7()
    want = GOLD["rule7"]["weights_barycenter_vertex_midside"]
    assert q[0, 3] == pytest.approx(want[0], abs=1e-17)
    assert np.allclose(q[1:4, 3], want[1], atol=1e-17)
    assert np.allclose(q[4:7, 3], want[2], atol=1e-17)
    # points: barycentre, the three vertices, the three mid-sides
    assert np.allclose(q[0, :3], 1.0 / 3.0)
    assert sorted(map(tuple, q[1:4, :3])) == sorted([(1, 0, 0), (0, 1, 0), (0, 0, 1)])
    assert sorted(map(tuple, q[4:7, :3])) == sorted([(.5, .5, 0), (0, .5, .5), (.5, 0, .5)])


def test_rule16_points_inside_and_positive():
    q = R.rule16()
    assert (q[:, :3] > 0).all() and (q[:, 3] > 0).all()
    assert len({tuple(r) for r in q[:, :2]}) == 16


@pytest.mark.parametrize("n", [5, 8, 12])
def test_gauss01(n):
    x, w = R.gauss01(n)
    assert (x > 0).all() and (x < 1).all()
    for k in range(2 * n):
        assert abs(np.sum(w * x ** k) - 1.0 / (k + 1)) < 2e-15, k
    if n == 5:  # degree exactly 2n - 1
        assert abs(np.sum(w * x ** (2 * n)) - 1.0 / (2 * n + 1)) > 1e-8


def test_gauss5_closed_form_matches_library():
    x, w = R.gauss01(5)
    t, v = np.polynomial.legendre.leggauss(5)
    assert np.allclose(x, 0.5 * (t + 1), atol=2e-16)
    assert np.allclose(w, 0.5 * v, atol=2e-16)
