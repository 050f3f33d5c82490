"""Pins of the oracle's label-dependent kernel (Sec. 1: the kernel may depend on element
labels, interface problems): Psi on E_k x E_l is scaled by s[m_k][m_l] for a symmetric table s.

- A table of ones reproduces the unlabelled matrix bit for bit; a uniform table c gives c A.
- The matrix is linear in the table: the sum of the assemblies with the indicator tables
  of the interior block, the exterior block and the coupling equals the full table's matrix.
- Every labelled matrix stays bitwise symmetric with A 1 = 0 (the symmetrised form, Rem. 2.4).
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
