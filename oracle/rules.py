"""Quadrature rules for the oracle (test infrastructure; independent of the CUDA path).

- 7-point rule on the reference triangle: barycentre, vertices and edge midpoints
  with weights 27/60 * 1/2, 3/60 * 1/2 and 8/60 * 1/2 (Sec. 3.1, footnote to the
  truncated fractional diffusion example). Exact for total degree <= 3.
- 16-point rule: the paper names none. The reading used here is the Stroud
  conical product of a 4-point Gauss-Jacobi rule (weight 1 - u on [0, 1]) and a
  4-point Gauss-Legendre rule, exact for total degree <= 7. Nodes are polished
  by Newton's method in 50-digit decimal arithmetic and rounded once to double.
  Parity unpinned against the paper, which prints no 16-point rule: the rule is pinned
  to its own definition only (exact for total degree <= 7, positive weights, points inside).
- Gauss-Legendre rules on [0, 1] for the tensor rule of the regularising
  transforms (Sec. 3.1: a tensor product of a 5-point Gauss rule).

A rule is an array [n, 4] of (l0, l1, l2, w): barycentric coordinates of the
point and its weight; the weights sum to 1/2, the area of the reference triangle.
"""
from __future__ import annotations

from decimal import Decimal, getcontext
from functools import lru_cache

import numpy as np

getcontext().prec = 50


def rule7() -> np.ndarray:
    third = 1.0 / 3.0
    pts = [
        (third, third, third, 27.0 / 120.0),
        (1.0, 0.0, 0.0, 3.0 / 120.0),
        (0.0, 1.0, 0.0, 3.0 / 120.0),
        (0.0, 0.0, 1.0, 3.0 / 120.0),
        (0.5, 0.5, 0.0, 8.0 / 120.0),
        (0.0, 0.5, 0.5, 8.0 / 120.0),
        (0.5, 0.0, 0.5, 8.0 / 120.0),
    ]
    return np.array(pts, dtype=np.float64)


def _jacobi(n: int, a: int, b: int, t: Decimal):
    """P_n^{(a,b)}(t) and P_{n-1}^{(a,b)}(t) by the three-term recurrence."""
    p0 = Decimal(1)
    if n == 0:
        return p0, Decimal(0)
    p1 = Decimal(a + 1) + Decimal(a + b + 2) * (t - 1) / 2
    for k in range(2, n + 1):
        c = 2 * k + a + b
        a1 = 2 * k * (k + a + b) * (c - 2)
        a2 = (c - 1) * (c * (c - 2) * t + a * a - b * b)
        a3 = 2 * (k + a - 1) * (k + b - 1) * c
        p0, p1 = p1, (a2 * p1 - a3 * p0) / a1
    return p1, p0


def _jacobi_deriv(n, a, b, t):
    pn, pm = _jacobi(n, a, b, t)
    c = 2 * n + a + b
    return pn, (n * ((a - b) - c * t) * pn + 2 * (n + a) * (n + b) * pm) / (c * (1 - t * t))


def _gauss_jacobi(n: int, a: int, b: int, guesses):
    """Nodes t_i in (-1, 1) and weights for weight (1-t)^a (1+t)^b, by Newton polishing."""
    from math import gamma
    nodes, weights = [], []
    for g in guesses:
        t = Decimal(repr(float(g)))
        for _ in range(100):
            pn, dp = _jacobi_deriv(n, a, b, t)
            dt = pn / dp
            t -= dt
            if abs(dt) < Decimal(10) ** -45:
                break
        _, dp = _jacobi_deriv(n, a, b, t)
        # w_i = G(n+a+1) G(n+b+1) / (G(n+a+b+1) n!) * 2^(a+b+1) / ((1 - t^2) P_n'(t)^2)
        cst = Decimal(gamma(n + a + 1)) * Decimal(gamma(n + b + 1)) / \
            (Decimal(gamma(n + a + b + 1)) * Decimal(gamma(n + 1)))
        w = cst * Decimal(2) ** (a + b + 1) / ((1 - t * t) * dp * dp)
        nodes.append(t)
        weights.append(w)
    return nodes, weights


@lru_cache(maxsize=None)
def rule16() -> np.ndarray:
    """Conical product rule, 4 x 4 points, degree 7 on the reference triangle."""
    from scipy.special import roots_jacobi, roots_legendre
    gj, _ = roots_jacobi(4, 1, 0)
    gl, _ = roots_legendre(4)
    tj, wj = _gauss_jacobi(4, 1, 0, gj)
    tl, wl = _gauss_jacobi(4, 0, 0, gl)
    pts = []
    half, quarter = Decimal(1) / 2, Decimal(1) / 4
    for t_u, w_u in zip(tj, wj):
        u = (1 + t_u) * half          # weight (1 - u) on [0, 1]
        wu = w_u * quarter
        for t_v, w_v in zip(tl, wl):
            v = (1 + t_v) * half
            wv = w_v * half
            l1 = u
            l2 = (1 - u) * v
            l0 = (1 - u) * (1 - v)
            pts.append((float(l0), float(l1), float(l2), float(wu * wv)))
    return np.array(pts, dtype=np.float64)


def rule(n: int) -> np.ndarray:
    if n == 7:
        return rule7()
    if n == 16:
        return rule16()
    raise ValueError(f"no {n}-point triangle rule")


def gauss01(n: int):
    """Gauss-Legendre points and weights on (0, 1)."""
    if n == 5:
        # closed form: 0, +-(1/3) sqrt(5 -+ 2 sqrt(10/7)); weights 128/225, (322 +- 13 sqrt 70)/900
        s = Decimal(10) / 7
        a = (Decimal(5) - 2 * s.sqrt()).sqrt() / 3
        b = (Decimal(5) + 2 * s.sqrt()).sqrt() / 3
        w0 = Decimal(128) / 225
        wa = (Decimal(322) + 13 * Decimal(70).sqrt()) / 900
        wb = (Decimal(322) - 13 * Decimal(70).sqrt()) / 900
        t = [-b, -a, Decimal(0), a, b]
        w = [wb, wa, w0, wa, wb]
        x = np.array([float((1 + ti) / 2) for ti in t])
        ww = np.array([float(wi / 2) for wi in w])
        return x, ww
    t, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (t + 1.0), 0.5 * w
