"""Pins of the oracle's pure Neumann-type solve (CPU).

The full matrix is singular with the null space N of Rem. 2.4: the constants for a
scalar kernel, the rigid motions for the peridynamic kernel. The oracle returns the
minimum-norm solution of A u = F - P_N F. Pinned without the oracle's own solve:
- for F = A v the answer is v minus its orthogonal projection onto N (closed form with
  the null-space basis written out here, not taken from the oracle);
- the answer is orthogonal to every rigid motion and solves the projected equation.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from synth import meshes


def rigid_modes(verts, ndof):
    x, y = verts[:, 0], verts[:, 1]
    if ndof == 1:
        return [np.ones_like(x)]
    z = np.zeros_like(x)
    return [np.stack([np.ones_like(x), z], 1).reshape(-1), np.stack([z, np.ones_like(x)], 1).reshape(-1),
            np.stack([-y, x], 1).reshape(-1)]


def project_out(v, modes):
    Q, _ = np.linalg.qr(np.stack(modes, 1))
    return v - Q @ (Q.T @ v)


@pytest.mark.parametrize("kw", [dict(kernel="constant", delta=0.3, ball="approxcaps"),
                                dict(kernel="fractional", s=0.5, delta=0.3, ball="nocaps"),
                                dict(kernel="peridynamic", delta=0.3, ball="nocaps")],
                         ids=lambda k: k["kernel"])
def test_neumann_recovers_projected_vector(kw):
    m = meshes.jittered_delaunay(0.0, 1.0, 7, 0.1, seed=12)
    S = oracle.assemble(m, **kw)
    rng = np.random.default_rng(3)
    v = rng.standard_normal(S.N)
    modes = rigid_modes(m.verts, S.ndof)
    v += 5.0 * modes[-1]                       # a large null-space component to remove
    S2 = dataclasses.replace(S, F=S.scipy() @ v)
    u = oracle.solve_neumann(S2, m.verts)
    want = project_out(v, modes)
    assert np.linalg.norm(u - want) <= 1e-8 * np.linalg.norm(want)


def test_neumann_projects_an_incompatible_load():
    m = meshes.structured(0.0, 1.0, 8)
    S = oracle.assemble(m, kernel="constant", delta=0.25, f_nodal=1.0 + m.verts[:, 0])
    u = oracle.solve_neumann(S, m.verts)
    assert abs(u.sum()) <= 1e-12 * np.abs(u).sum()
    b = project_out(S.F, rigid_modes(m.verts, 1))
    assert np.linalg.norm(S.scipy() @ u - b) <= 1e-10 * np.linalg.norm(b)
