"""Pins of the oracle's label-dependent kernel (Sec. 1: the kernel may depend on element
labels, interface problems): Psi on E_k x E_l is scaled by s[m_k][m_l] for a symmetric table s.

- A table of ones reproduces the unlabelled matrix bit for bit; a uniform table c gives c A.
- The matrix is linear in the table: the sum of the assemblies with the indicator tables
  of the interior block, the exterior block and the coupling equals the full table's matrix.
- Every labelled matrix stays bitwise symmetric with A 1 = 0 (the symmetrised form, Rem. 2.4).
- Closed form: with every pair inside the ball, the constant kernel on the pairs of different
  materials only is 2c (|Omega_1| M0 + |Omega_0| M1) - 2c (m0 m1^T + m1 m0^T) (the linearity and
  symmetry pins alone would not see a table read at (m_k, m_k) instead of (m_k, m_l)).
"""
import numpy as np
import pytest

import oracle
from synth import meshes


@pytest.fixture(scope="module")
def case():
    m = meshes.jittered_delaunay(0.0, 1.0, 9, 0.1, seed=14)
    c = m.verts[m.elems].mean(1)
    mat = (c[:, 0] > 0.5).astype(np.int8)         # two materials split at x = 0.5
    return m, mat


@pytest.mark.parametrize("kw", [dict(kernel="constant", delta=0.25, ball="approxcaps"),
                                dict(kernel="fractional", s=0.5, delta=0.25, ball="nocaps")],
                         ids=lambda k: k["kernel"])
def test_material_table_linear_symmetric(case, kw):
    m, mat = case
    A0 = oracle.assemble(m, **kw)
    ones = oracle.assemble(m, materials=mat, material_scale=np.ones((2, 2)), **kw)
    assert np.array_equal(ones.val, A0.val) and np.array_equal(ones.col, A0.col)
    u = oracle.assemble(m, materials=mat, material_scale=3.0 * np.ones((2, 2)), **kw)
    assert np.allclose(u.val, 3.0 * A0.val, rtol=1e-13, atol=1e-14 * np.abs(u.val).max())
    tab = np.array([[1.0, 0.35], [0.35, 4.0]])
    full = oracle.assemble(m, materials=mat, material_scale=tab, **kw)
    parts = [np.array([[1.0, 0], [0, 0]]), np.array([[0, 0], [0, 4.0]]), np.array([[0, 0.35], [0.35, 0]])]
    tot = sum(oracle.assemble(m, materials=mat, material_scale=t, **kw).val for t in parts)
    assert np.allclose(full.val, tot, rtol=1e-13, atol=1e-13 * np.abs(full.val).max())
    A = full.scipy()
    assert (A != A.T).nnz == 0
    assert np.abs(A @ np.ones(full.N)).max() < 1e-13 * np.abs(full.val).max()
    # the coupling changes the matrix only near the interface
    assert not np.allclose(full.val, A0.val)


def test_coupling_table_closed_form():
    # with every pair inside the ball, the constant kernel c restricted to pairs of different
    # materials (table [[0, 1], [1, 0]]) is
    #   2c (|Omega_1| M0 + |Omega_0| M1) - 2c (m0 m1^T + m1 m0^T),
    # Mj the mass matrix and mj the vector of int phi_i over the elements of material j
    m = meshes.jittered_delaunay(0.0, 1.0, 5, 0.1, seed=15)
    c = m.verts[m.elems].mean(1)
    mat = (c[:, 1] > 0.45).astype(np.int8)
    X, T = m.verts, m.elems
    area = 0.5 * np.abs((X[T[:, 1], 0] - X[T[:, 0], 0]) * (X[T[:, 2], 1] - X[T[:, 0], 1])
                        - (X[T[:, 2], 0] - X[T[:, 0], 0]) * (X[T[:, 1], 1] - X[T[:, 0], 1]))
    M = [np.zeros((m.M, m.M)), np.zeros((m.M, m.M))]
    mv = [np.zeros(m.M), np.zeros(m.M)]
    for k in range(m.K):
        j = mat[k]
        for a in range(3):
            mv[j][T[k, a]] += area[k] / 3.0
            for b in range(3):
                M[j][T[k, a], T[k, b]] += area[k] / 12.0 * (1.0 + (a == b))
    Om = [area[mat == 0].sum(), area[mat == 1].sum()]
    delta = 5.0
    cc = 4.0 / (np.pi * delta ** 4)
    ref = 2 * cc * (Om[1] * M[0] + Om[0] * M[1]) - 2 * cc * (np.outer(mv[0], mv[1]) + np.outer(mv[1], mv[0]))
    A = oracle.assemble(m, kernel="constant", delta=delta, materials=mat,
                        material_scale=np.array([[0.0, 1.0], [1.0, 0.0]]))
    assert np.abs(A.dense() - ref).max() < 1e-13 * np.abs(ref).max()
