"""Pins of the oracle's infinity norm ball (Sec. 2.2, Def. of the infinity norm ball) on the CPU.

The infinity ball is cut exactly (no geometric error), so:
- over all elements of a mesh covering the square, the clipped areas add up to (2 delta)^2
  to rounding, on jittered meshes and on structured meshes whose lines the square's sides
  hit exactly (the tie cases);
- each clipped area equals the area of the square clipped by the triangle's three
  half-planes, computed here the other way round (square as the subject polygon);
- every polygon point lies in both the triangle and the square, and the polygon is convex
  and counter-clockwise;
- special cases: the square inside a large triangle, the triangle inside the square,
  disjoint, touching along an edge or at a corner only.
"""
import numpy as np
import pytest

import oracle
from synth import meshes


def shoelace(P):
    x, y = P[:, 0], P[:, 1]
    return 0.5 * float(np.sum(x * np.roll(y, -1) - y * np.roll(x, -1)))


def square_by_triangle_area(V, c, d):
    """Area of the square |y - c|_inf <= d intersected with the CCW triangle V: the square is
    clipped successively by the triangle's three inner half-planes (independent of the oracle)."""
    P = [np.array(c, float) + np.array(q) for q in ((-d, -d), (d, -d), (d, d), (-d, d))]
    V = np.asarray(V, float)
    for i in range(3):
        a, b = V[i], V[(i + 1) % 3]
        f = lambda p: (b[0] - a[0]) * (p[1] - a[1]) - (b[1] - a[1]) * (p[0] - a[0])
        out = []
        for j in range(len(P)):
            S, E = P[j - 1], P[j]
            fs, fe = f(S), f(E)
            if (fs >= 0) != (fe >= 0):
                out.append(S + (fs / (fs - fe)) * (E - S))
            if fe >= 0:
                out.append(E)
        P = out
        if not P:
            return 0.0
    return shoelace(np.array(P)) if len(P) >= 3 else 0.0


def tri_area(V):
    V = np.asarray(V, float)
    return 0.5 * ((V[1, 0] - V[0, 0]) * (V[2, 1] - V[0, 1]) - (V[1, 1] - V[0, 1]) * (V[2, 0] - V[0, 0]))


def clip_area(V, c, d):
    P, full = oracle.clip(V, c, d, ball="infinity")
    if full:
        return tri_area(V)
    return shoelace(P) if len(P) >= 3 else 0.0


def test_areas_match_square_clipped_by_triangle():
    rng = np.random.default_rng(7)
    for _ in range(3000):
        V = rng.uniform(-1, 1, size=(3, 2))
        if tri_area(V) < 0:
            V[[1, 2]] = V[[2, 1]]
        c = rng.uniform(-1.2, 1.2, size=2)
        d = rng.uniform(0.05, 1.2)
        got, want = clip_area(V, c, d), square_by_triangle_area(V, c, d)
        assert abs(got - want) <= 1e-13 * max(1.0, 4 * d * d), (V, c, d, got, want)


def test_points_inside_convex_ccw():
    rng = np.random.default_rng(8)
    for _ in range(2000):
        V = rng.uniform(-1, 1, size=(3, 2))
        if tri_area(V) < 0:
            V[[1, 2]] = V[[2, 1]]
        c = rng.uniform(-1, 1, size=2)
        d = rng.uniform(0.05, 1.0)
        P, full = oracle.clip(V, c, d, ball="infinity")
        if full or len(P) < 3:
            continue
        assert len(P) <= 7
        assert np.all(np.abs(P - c) <= d * (1 + 1e-12))
        for i in range(3):
            a, b = V[i], V[(i + 1) % 3]
            cr = (b[0] - a[0]) * (P[:, 1] - a[1]) - (b[1] - a[1]) * (P[:, 0] - a[0])
            assert np.all(cr >= -1e-12), (V, c, d, P)
        n = len(P)
        for i in range(n):
            p, q, r = P[i], P[(i + 1) % n], P[(i + 2) % n]
            turn = (q[0] - p[0]) * (r[1] - q[1]) - (q[1] - p[1]) * (r[0] - q[0])
            assert turn >= -1e-12, (V, c, d, P)


@pytest.mark.parametrize("kind", ["jittered", "structured"])
@pytest.mark.parametrize("d", [0.05, 0.125, 0.3])
def test_partition_sums_to_square_area(kind, d):
    if kind == "jittered":
        m = meshes.jittered_delaunay(-0.5, 1.5, 40, 0.2, seed=3)
    else:
        m = meshes.structured(-0.5, 1.5, 40)          # spacing 0.05: sides on mesh lines
    rng = np.random.default_rng(11)
    centres = list(rng.uniform(0.2, 0.8, size=(6, 2))) + [m.verts[len(m.verts) // 2]]
    for c in centres:
        tot = 0.0
        for e in m.elems:
            tot += clip_area(m.verts[e], c, d)
        assert abs(tot - 4 * d * d) <= 1e-13 * 4 * d * d, (c, tot, 4 * d * d)


def test_special_cases():
    d = 0.1
    big = np.array([[-5.0, -5.0], [5.0, -5.0], [0.0, 5.0]])
    P, full = oracle.clip(big, (0.0, 0.0), d, ball="infinity")
    assert not full and len(P) == 4 and abs(shoelace(P) - 4 * d * d) < 1e-15
    small = np.array([[0.0, 0.0], [0.05, 0.0], [0.0, 0.05]])
    P, full = oracle.clip(small, (0.01, 0.01), d, ball="infinity")
    assert full
    P, full = oracle.clip(small, (1.0, 1.0), d, ball="infinity")
    assert not full and len(P) == 0
    # an edge on the square's right side, the triangle outside: fewer than 3 points
    edge = np.array([[0.1, 0.0], [0.6, 0.0], [0.1, 0.5]])
    P, full = oracle.clip(edge, (0.0, 0.0), d, ball="infinity")
    assert len(P) == 0
    # touching at the corner (0.1, 0.1) only
    corner = np.array([[0.1, 0.1], [0.5, 0.1], [0.1, 0.5]])
    P, full = oracle.clip(corner, (0.0, 0.0), d, ball="infinity")
    assert len(P) == 0
    # vertex on the boundary counts as inside: the whole triangle
    onb = np.array([[0.1, 0.0], [0.0, 0.1], [-0.1, -0.1]])
    P, full = oracle.clip(onb, (0.0, 0.0), d, ball="infinity")
    assert full
