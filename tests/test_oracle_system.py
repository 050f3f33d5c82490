"""System-level pins of the oracle (CPU): pair search, invariants, convergence.

- P9: the traversal of Alg. 2 finds exactly the pairs of a brute-force search
  over all element pairs with the same predicate.
- P10: on the "/"-split grid every interior element has 1 identical, 3 common
  edge and 9 common vertex partners (Sec. 2.4, the first BFS layer).
- P5: A is symmetric bit for bit (Rem. 2.4), A 1 = 0 (Neumann null space,
  Sec. 1 and Rem. 2.4), the peridynamic operator annihilates rigid motions,
  and the diagonal is positive.
- P7: with the constants of Sec. 3 the discrete operator reproduces -Delta on
  x^2 + y^2 row by row, up to the O(h^2) ball approximation error (Z1: the
  factor 2 of eq. strongL), and the peridynamic one -(pi/4) Delta u - (pi/2) grad div u
  on u = (y^2, x^2 y).
- P6: the manufactured solutions of Sec. 3.1 / 3.2 converge at second order
  (Tabs. tab:hto0fractionalCG and tab:hto0peridynamicsCG).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from synth import meshes

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))


@pytest.mark.parametrize("mesh_kind,ball,nq", [("structured", "nocaps", 7), ("jittered", "approxcaps", 7),
                                              ("jittered", "nocaps", 16), ("structured", "approxcaps", 16),
                                              ("structured", "infinity", 7), ("jittered", "infinity", 16)])
def test_bfs_pairs_equal_brute_force(mesh_kind, ball, nq):
    m = meshes.structured(0.0, 1.0, 7) if mesh_kind == "structured" else \
        meshes.jittered_delaunay(0.0, 1.0, 7, 0.1, seed=3)
    delta = 2.0 / 7 if ball != "infinity" else 1.5 / 7   # square sides on mesh lines when structured
    a = oracle.pairs(m, kernel="constant", delta=delta, ball=ball, quad_outer=nq, mode="bfs")
    b = oracle.pairs(m, kernel="constant", delta=delta, ball=ball, quad_outer=nq, mode="brute")
    assert len(a) == len(b) > m.K
    assert set(map(tuple, a)) == set(map(tuple, b))


def test_classification_counts_structured():
    n = 8
    m = meshes.structured(0.0, 1.0, n)
    S = oracle.assemble(m, kernel="constant", delta=2.5 / n)
    c = m.verts[m.elems].mean(1)
    interior = np.flatnonzero((c.min(1) > 1.5 / n) & (c.max(1) < 1 - 1.5 / n))
    for k in interior:
        sel = S.pclass[S.pairs[:, 0] == k]
        assert (sel == 3).sum() == 1 and (sel == 2).sum() == 3 and (sel == 1).sum() == 9


CASES = [
    dict(kernel="constant", delta=0.3, ball="nocaps"),
    dict(kernel="constant", delta=0.3, ball="infinity"),
    dict(kernel="fractional", s=0.25, delta=0.2, ball="infinity"),
    dict(kernel="constant", delta=0.3, ball="approxcaps", quad_outer=16, quad_inner=16),
    dict(kernel="fractional", s=0.5, delta=0.3, ball="approxcaps"),
    dict(kernel="fractional", s=0.75, delta=0.3, ball="nocaps", quad_outer=16, quad_inner=7),
    dict(kernel="peridynamic", delta=0.3, ball="nocaps"),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c['kernel']}-{c['ball']}")
def test_invariants(case):
    m = meshes.jittered_delaunay(0.0, 1.0, 8, 0.1, seed=5)
    S = oracle.assemble(m, **case)
    A = S.scipy()
    assert (A != A.T).nnz == 0                       # bitwise symmetric
    d = A.diagonal()
    assert (d > 0).all()
    scale = abs(A).max()
    if S.ndof == 1:
        assert np.abs(A @ np.ones(S.N)).max() < 1e-13 * scale
    else:
        x, y = m.verts[:, 0], m.verts[:, 1]
        for mode in (np.stack([np.ones_like(x), 0 * x], 1), np.stack([0 * x, np.ones_like(x)], 1),
                     np.stack([-y, x], 1)):
            assert np.abs(A @ mode.reshape(-1)).max() < 1e-13 * scale * max(1.0, np.abs(mode).max())


def test_constant_kernel_reproduces_laplacian_rowwise():
    # P7: (A I_h u)_i / int phi_i -> -Delta u = -4 for interior rows, u = x^2 + y^2, fixed delta
    delta = 0.2
    errs = []
    for n in (10, 20, 40):
        m = meshes.structured(-delta, 1 + delta, int(round((1 + 2 * delta) * n)))
        S = oracle.assemble(m, kernel="constant", delta=delta, ball="approxcaps",
                            f_nodal=np.ones(m.M))   # F_i = int_Omega phi_i
        g = m.verts[:, 0] ** 2 + m.verts[:, 1] ** 2
        r = S.scipy() @ g
        x, y = m.verts[:, 0], m.verts[:, 1]
        inner = (x > 0.3) & (x < 0.7) & (y > 0.3) & (y < 0.7)
        errs.append(np.max(np.abs(r[inner] / S.F[inner] + 4.0)))
    assert errs[-1] < 0.05
    assert math.log2(errs[0] / errs[1]) > 1.5 and math.log2(errs[1] / errs[2]) > 1.5, errs


def test_peridynamic_kernel_reproduces_navier_rowwise():
    # P7 for peridynamics: with c = 3 / delta^3 the operator is -(pi/4) Delta u - (pi/2) grad div u
    # (the factor-2 reading of eq. strongL); for u = (y^2, x^2 y) that is -(pi/2) (1 + 2x, y), and
    # (A I_h u)_i / int phi_i approaches it row by row at second order (fixed delta)
    delta = 0.2
    errs = []
    for n in (8, 16, 32):
        m = meshes.structured(-delta, 1 + delta, int(round((1 + 2 * delta) * n)))
        x, y = m.verts[:, 0], m.verts[:, 1]
        S = oracle.assemble(m, kernel="peridynamic", delta=delta, ball="approxcaps",
                            f_nodal=np.stack([np.ones(m.M), np.ones(m.M)], 1))
        g = np.stack([y * y, x * x * y], 1).reshape(-1)
        inner = (x > 0.3) & (x < 0.7) & (y > 0.3) & (y < 0.7)
        r = (S.scipy() @ g).reshape(-1, 2)[inner] / S.F.reshape(-1, 2)[inner]
        want = -0.5 * math.pi * np.stack([1.0 + 2.0 * x, y], 1)[inner]
        errs.append(np.max(np.abs(r - want)))
    assert errs[-1] < 0.05, errs
    assert math.log2(errs[0] / errs[1]) > 1.5 and math.log2(errs[1] / errs[2]) > 1.5, errs

def test_load_vector_partition_of_unity():
    m = meshes.jittered_delaunay(-0.2, 1.2, 10, 0.1, seed=9)
    S = oracle.assemble(m, kernel="constant", delta=0.3, f_nodal=2.0 + 3.0 * m.verts[:, 0])
    # sum_i F_i = int_Omega f, exact for the 7-point rule and linear f
    P = m.verts[m.elems[m.elem_label == 1]]
    area = 0.5 * np.abs((P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1]) -
                        (P[:, 1, 1] - P[:, 0, 1]) * (P[:, 2, 0] - P[:, 0, 0]))
    want = np.sum(area * (2.0 + 3.0 * P[:, :, 0].mean(1)))
    assert abs(S.F.sum() - want) < 1e-13 * abs(want)
    assert np.all(S.F[S.dirichlet & ~np.isin(np.arange(m.M), m.elems[m.elem_label == 1])] == 0)


def test_load_vector_closed_form_for_linear_f():
    # F_i = sum over Omega elements E of int_E f phi_i, and for f in P1 with nodal values f_a
    # the element integral is |E| (2 f_a + f_b + f_c) / 12 (exact for the 7- and 16-point rules)
    m = meshes.jittered_delaunay(-0.2, 1.2, 10, 0.1, seed=9)
    f = 2.0 + 3.0 * m.verts[:, 0] - 5.0 * m.verts[:, 1]
    want = np.zeros(m.M)
    for e in np.flatnonzero(m.elem_label == 1):
        t = m.elems[e]
        P = m.verts[t]
        area = 0.5 * abs((P[1, 0] - P[0, 0]) * (P[2, 1] - P[0, 1]) - (P[1, 1] - P[0, 1]) * (P[2, 0] - P[0, 0]))
        for a in range(3):
            want[t[a]] += area * (2.0 * f[t[a]] + f[t[(a + 1) % 3]] + f[t[(a + 2) % 3]]) / 12.0
    for nq in (7, 16):
        S = oracle.assemble(m, kernel="constant", delta=0.3, f_nodal=f, quad_outer=nq)
        assert np.abs(S.F - want).max() < 1e-14 * np.abs(want).max()


def _e1(level):
    a = GOLD["E1_fractional_cg"]["a"][level]
    m = meshes.paper_square(0.2, a)
    S = oracle.assemble(m, kernel="fractional", delta=0.2, s=0.5, ball="approxcaps",
                        f_nodal=-2.0 * (m.verts[:, 1] + 1.0))
    ue = lambda x, y: x * x * y + y * y
    u = oracle.solve_dirichlet(S, ue(m.verts[:, 0], m.verts[:, 1]))
    return int((~S.dirichlet).sum()), oracle.l2_error(m, u, ue)


def _e3(level):
    a = GOLD["E3_peridynamics_cg"]["a"][level]
    m = meshes.paper_square(0.1, a)
    x, y = m.verts[:, 0], m.verts[:, 1]
    f = -0.5 * math.pi * np.stack([1.0 + 2.0 * x, y], 1)
    S = oracle.assemble(m, kernel="peridynamic", delta=0.1, ball="approxcaps", f_nodal=f)
    ue = lambda x, y: np.stack([y * y, x * x * y])
    g = np.stack([y * y, x * x * y], 1).reshape(-1)
    u = oracle.solve_dirichlet(S, g)
    return int((~np.repeat(S.dirichlet, 2)).sum()), oracle.l2_error(m, u, ue, ndof=2)


def _check(tab, runs):
    dofs = [r[0] for r in runs]
    errs = [r[1] for r in runs]
    for i, d in enumerate(dofs):
        assert abs(d - tab["dof"][i]) <= 0.005 * tab["dof"][i] + 1     # printed with 3 digits
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    for i, r in enumerate(rates):
        assert 1.85 < r < 2.25, (rates, errs)
    # The paper states neither the triangulation of its grids nor how the L2 error is
    # evaluated; the printed errors sit below the interpolation error of a "/"-split
    # grid. Only the order of magnitude is pinned.
    for i, e in enumerate(errs):
        assert 0.4 * tab["l2"][i] < e < 2.5 * tab["l2"][i], (errs, tab["l2"])
    return rates


def test_paper_E1_fractional_rates():
    runs = [_e1(k) for k in range(3)]
    _check(GOLD["E1_fractional_cg"], runs)


def test_paper_E3_peridynamic_rates():
    runs = [_e3(k) for k in range(3)]
    _check(GOLD["E3_peridynamics_cg"], runs)


def _e6(level):
    # Sec. 3.3, delta = 2a (h = sqrt(2) a the element diameter): u = sin(4 pi x) sin(4 pi y),
    # f = -Delta u given at the nodes, constant kernel c = 3 / (4 delta^4) on the infinity ball
    a = 0.1 / 2 ** level              # printed h = sqrt(2) a
    delta = GOLD["E6_infinity_delta_h"]["delta"][level]
    m = meshes.paper_square(delta, a)
    ue = lambda x, y: np.sin(4 * math.pi * x) * np.sin(4 * math.pi * y)
    x, y = m.verts[:, 0], m.verts[:, 1]
    S = oracle.assemble(m, kernel="constant", delta=delta, ball="infinity",
                        f_nodal=32 * math.pi ** 2 * ue(x, y))
    u = oracle.solve_dirichlet(S, ue(x, y))
    return oracle.l2_error(m, u, ue)


def test_paper_E6_infinity_ball_rates():
    tab = GOLD["E6_infinity_delta_h"]
    errs = [_e6(k) for k in range(4)]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    for i, r in enumerate(rates):
        assert abs(r - tab["rate"][i + 1]) < 0.15, (rates, errs)
    # the printed errors include the paper's (unstated) load quadrature of the oscillating f;
    # with f given at the nodes they come out about 20% larger: the magnitude is pinned
    for i, e in enumerate(errs):
        assert 0.5 * tab["l2"][i] < e < 2.0 * tab["l2"][i], (errs, tab["l2"])


@pytest.mark.slow
def test_paper_E1_fractional_rates_level3():
    runs = [_e1(k) for k in range(4)]
    _check(GOLD["E1_fractional_cg"], runs)


def test_l2_error_closed_forms():
    # the error norm of the convergence pins: Omega = (0, 1)^2 exactly (grid lines at 0 and 1),
    # ||1|| = 1, ||x|| = 1/sqrt(3), ||(1, x)|| = 2/sqrt(3) (the 7-point rule is exact for degree 2),
    # and a linear function is reproduced by its P1 interpolant
    m = meshes.structured(-0.2, 1.2, 14)
    x, y = m.verts[:, 0], m.verts[:, 1]
    z = np.zeros(m.M)
    assert abs(oracle.l2_error(m, z, lambda x, y: 1.0 + 0 * x) - 1.0) < 1e-14
    assert abs(oracle.l2_error(m, z, lambda x, y: x) - 1.0 / math.sqrt(3.0)) < 1e-14
    assert abs(oracle.l2_error(m, np.zeros(2 * m.M), lambda x, y: np.stack([1.0 + 0 * x, x]), ndof=2)
               - 2.0 / math.sqrt(3.0)) < 1e-14
    assert oracle.l2_error(m, 2.0 - 3.0 * x + 5.0 * y, lambda x, y: 2.0 - 3.0 * x + 5.0 * y) < 1e-13
