"""Pins of the oracle's ball approximations (Defs. 2.1, 2.2) on the CPU.

The exact area of disk-intersect-triangle is computed here independently
(sectors and triangles around the centre). The nocaps polygon misses exactly
the circular segments cut off by its chords; approxcaps adds one triangle per
cap, so its area lies between nocaps and exact. The fan triangulation of the
polygon must reproduce the shoelace area. Over all elements of a fine mesh the
nocaps ball converges to the disk area pi delta^2 at second order in h
(Sec. 2.2: the symmetric difference is O(h^2)).
"""
import math

import numpy as np
import pytest

import oracle
from synth import meshes


def shoelace(P):
    x, y = P[:, 0], P[:, 1]
    return 0.5 * float(np.sum(x * np.roll(y, -1) - y * np.roll(x, -1)))


def disk_triangle_area(V, c, r):
    """Exact area of disk(c, r) intersected with the CCW triangle V (independent formula)."""
    def seg_area(a, b):
        # signed area of disk intersect triangle (c, a, b), c at origin
        a = np.asarray(a, float); b = np.asarray(b, float)
        d = b - a
        A = d @ d; B = a @ d; C = a @ a - r * r
        disc = B * B - A * C
        ts = [0.0]
        if disc > 0:
            s = math.sqrt(disc)
            for t in sorted([(-B - s) / A, (-B + s) / A]):
                if 0 < t < 1:
                    ts.append(t)
        ts.append(1.0)
        tot = 0.0
        for t0, t1 in zip(ts[:-1], ts[1:]):
            p = a + t0 * d; q = a + t1 * d
            m = a + 0.5 * (t0 + t1) * d
            cr = p[0] * q[1] - p[1] * q[0]
            if m @ m <= r * r:
                tot += 0.5 * cr
            else:
                ang = math.atan2(cr, p @ q)
                tot += 0.5 * r * r * ang
        return tot
    V = np.asarray(V, float) - np.asarray(c, float)
    return sum(seg_area(V[i], V[(i + 1) % 3]) for i in range(3))


def on_circle(p, c, r):
    return abs(math.hypot(p[0] - c[0], p[1] - c[1]) - r) < 1e-9 * r


def on_edge(p, q, V):
    m = 0.5 * (p + q)
    for i in range(3):
        a, b = V[i], V[(i + 1) % 3]
        cr = (b[0] - a[0]) * (m[1] - a[1]) - (b[1] - a[1]) * (m[0] - a[0])
        if abs(cr) < 1e-12 * np.dot(b - a, b - a) ** 0.5:
            return True
    return False


def segment_area(p, q, r):
    chord = math.hypot(q[0] - p[0], q[1] - p[1])
    th = 2 * math.asin(min(1.0, chord / (2 * r)))
    return 0.5 * r * r * (th - math.sin(th))


def random_cases(n, seed=1):
    rng = np.random.default_rng(seed)
    for _ in range(n):
        V = rng.uniform(-1, 1, size=(3, 2))
        if (V[1, 0] - V[0, 0]) * (V[2, 1] - V[0, 1]) - (V[1, 1] - V[0, 1]) * (V[2, 0] - V[0, 0]) < 0:
            V[[1, 2]] = V[[2, 1]]
        c = rng.uniform(-1.2, 1.2, size=2)
        r = rng.uniform(0.2, 1.5)
        yield V, c, r


def test_nocaps_misses_exactly_the_segments():
    checked = 0
    for V, c, r in random_cases(400):
        P, full = oracle.clip(V, c, r, caps=False)
        exact = disk_triangle_area(V, c, r)
        if full:
            assert abs(exact - shoelace(V)) < 1e-12
            continue
        if len(P) < 3:
            assert exact < 1e-6 or len(P) == 2  # a chord alone bounds a lone cap
            continue
        A = shoelace(P)
        assert A > -1e-14
        missing = sum(segment_area(P[i], P[(i + 1) % len(P)], r) for i in range(len(P))
                      if on_circle(P[i], c, r) and on_circle(P[(i + 1) % len(P)], c, r)
                      and not on_edge(P[i], P[(i + 1) % len(P)], V))
        assert abs((exact - A) - missing) < 1e-11, (V, c, r)
        checked += 1
    assert checked > 50


def test_approxcaps_between_nocaps_and_exact():
    n = 0
    for V, c, r in random_cases(400, seed=2):
        Pn, full = oracle.clip(V, c, r, caps=False)
        Pa, _ = oracle.clip(V, c, r, caps=True)
        if full:
            continue
        exact = disk_triangle_area(V, c, r)
        An = shoelace(Pn) if len(Pn) >= 3 else 0.0
        Aa = shoelace(Pa) if len(Pa) >= 3 else 0.0
        assert An - 1e-13 <= Aa <= exact + 1e-12
        # every added point is a cap centre on the circle
        extra = [p for p in Pa if not any(np.array_equal(p, q) for q in Pn)]
        assert all(on_circle(p, c, r) for p in extra)
        n += len(extra) > 0
    assert n > 30


def test_fan_triangulation_area():
    # the oracle integrates the fan (P0, Pi, Pi+1); its area equals the shoelace area
    for V, c, r in random_cases(200, seed=3):
        for caps in (False, True):
            P, full = oracle.clip(V, c, r, caps)
            if len(P) < 3:
                continue
            fan = sum(0.5 * abs((P[i][0] - P[0][0]) * (P[i + 1][1] - P[0][1]) -
                                (P[i][1] - P[0][1]) * (P[i + 1][0] - P[0][0])) for i in range(1, len(P) - 1))
            assert abs(fan - shoelace(P)) < 1e-13


def test_clip_special_cases():
    V = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    P, full = oracle.clip(V, (0.2, 0.2), 5.0, False)
    assert full and len(P) == 3
    P, full = oracle.clip(V, (5.0, 5.0), 1.0, True)
    assert not full and len(P) == 0
    # vertex exactly on the circle, both edges leaving: a single point, no area
    P, full = oracle.clip(V, (-1.0, 0.0), 1.0, True)
    assert len(P) < 3
    # a chord across one edge only: nocaps has 2 points (empty), approxcaps adds the cap centre
    V2 = np.array([[-1.0, 0.0], [1.0, 0.0], [0.0, 2.0]])
    P, _ = oracle.clip(V2, (0.0, -0.5), 0.7, False)
    assert len(P) == 2
    P, _ = oracle.clip(V2, (0.0, -0.5), 0.7, True)
    assert len(P) == 3 and np.allclose(P[2], (0.0, 0.2))
    # vertex on the circle reached by an edge: the crossing snaps to the vertex
    V3 = np.array([[0.3, 0.5], [0.4, 0.5], [0.4, 0.6]])
    P, _ = oracle.clip(V3, (0.3, 0.3), 0.2, True)
    assert len(P) == 1 and np.array_equal(P[0], V3[0])


@pytest.mark.parametrize("caps", [False, True])
def test_ball_area_converges_second_order(caps):
    # sum over elements of |E_l cut by the ball around x| -> pi delta^2 (Sec. 2.2, O(h^2))
    delta = 0.3
    errs = []
    for n in (8, 16, 32):
        m = meshes.structured(-0.5, 0.5, n)
        x = np.array([0.0123, -0.0311])
        tot = 0.0
        for e in m.elems:
            P, full = oracle.clip(m.verts[e], x, delta, caps)
            if len(P) >= 3:
                tot += shoelace(P)
        errs.append(abs(tot - math.pi * delta ** 2))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > 1.5, (errs, rates)
    if caps:
        nocap = []
        # approxcaps has the smaller geometric error
        m = meshes.structured(-0.5, 0.5, 16)
        x = np.array([0.0123, -0.0311])
        tot = sum(shoelace(P) for P, _ in (oracle.clip(m.verts[e], x, delta, False) for e in m.elems)
                  if len(P) >= 3)
        nocap.append(abs(tot - math.pi * delta ** 2))
        assert errs[1] < nocap[0]
