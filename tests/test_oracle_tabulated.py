"""Pins of the oracle's user-defined (tabulated radial) kernel, gamma = c g(|x - y|) with g
linear between table values at r_i = i delta / (n - 1) (the Conclusion: user-defined kernels).

- A constant table g = 1 with c = 4 / (pi delta^4) reproduces the constant kernel bit for bit
  (all three balls).
- The matrix is linear in the table values; symmetry and A 1 = 0 hold for any table.
- Tables of g(r) = r^2 with 2, 4, 8, 16 intervals: the interpolation error is at most
  (delta / (n - 1))^2 / 4, so successive matrices approach each other at second order.
- A table of g(r) = r is interpolated exactly: it reproduces c |z|^(-2-2s) at s = -3/2.
"""
import numpy as np
import pytest

import oracle
from synth import meshes


@pytest.fixture(scope="module")
def mesh():
    return meshes.jittered_delaunay(0.0, 1.0, 8, 0.1, seed=19)


def test_constant_table_is_the_constant_kernel(mesh):
    d = 0.3
    for ball in ("nocaps", "approxcaps", "infinity"):
        A = oracle.assemble(mesh, kernel="constant", delta=d, ball=ball, kconst=4 / (np.pi * d ** 4))
        B = oracle.assemble(mesh, kernel="tabulated", delta=d, ball=ball, kconst=4 / (np.pi * d ** 4),
                            kernel_table=np.ones(5))
        assert np.array_equal(A.col, B.col) and np.array_equal(A.val, B.val)


def test_linear_in_table_and_invariants(mesh):
    d = 0.3
    rng = np.random.default_rng(2)
    t1, t2 = rng.uniform(0.5, 2.0, 9), rng.uniform(-1.0, 1.0, 9)
    A1 = oracle.assemble(mesh, kernel="tabulated", delta=d, ball="approxcaps", kernel_table=t1)
    A2 = oracle.assemble(mesh, kernel="tabulated", delta=d, ball="approxcaps", kernel_table=t2)
    A12 = oracle.assemble(mesh, kernel="tabulated", delta=d, ball="approxcaps", kernel_table=t1 + t2)
    scale = np.abs(A12.val).max()
    assert np.allclose(A12.val, A1.val + A2.val, rtol=0, atol=1e-13 * scale)
    S = A1.scipy()
    assert (S != S.T).nnz == 0
    assert np.abs(S @ np.ones(A1.N)).max() < 1e-13 * np.abs(A1.val).max()


def test_piecewise_linear_table_converges_second_order(mesh):
    # g(r) = r^2 tabulated with n nodes: the interpolation error is at most (delta/(n-1))^2/4,
    # so the matrices of successive tables approach each other at second order in 1/(n-1)
    d = 0.3
    vals = []
    for n in (3, 5, 9, 17):
        r = np.linspace(0.0, d, n)
        vals.append(oracle.assemble(mesh, kernel="tabulated", delta=d, ball="nocaps", kernel_table=r * r).val)
    diffs = [np.abs(vals[i + 1] - vals[i]).max() for i in range(3)]
    rates = [np.log2(diffs[i] / diffs[i + 1]) for i in range(2)]
    assert all(1.7 < q < 2.3 for q in rates), (diffs, rates)


def test_linear_table_is_the_power_kernel(mesh):
    # g(r) = r is interpolated exactly by the table, and c |z|^(-2-2s) with s = -3/2 is c |z|:
    # both assemblies agree to rounding wherever every point lies within delta (Euclidean balls)
    d = 0.3
    for ball in ("nocaps", "approxcaps"):
        A = oracle.assemble(mesh, kernel="fractional", s=-1.5, delta=d, ball=ball, kconst=2.0)
        B = oracle.assemble(mesh, kernel="tabulated", delta=d, ball=ball, kconst=2.0,
                            kernel_table=np.linspace(0.0, d, 7))
        assert np.array_equal(A.col, B.col)
        assert np.abs(A.val - B.val).max() < 1e-13 * np.abs(A.val).max()
