"""Fault handling of the solver on the host side: an iteration cap that the CG cannot meet ends
the solve with NLFEM_ERR_NOT_CONVERGED (status -6), the last iterate in u and the residual in
the info; the system stays usable and the next solve converges."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2207_03921_gb300 import Mesh, assemble  # noqa: E402
from synth import meshes  # noqa: E402


def test_iteration_cap_reports_not_converged():
    m = meshes.jittered_delaunay(-0.2, 1.2, 14, 0.05, seed=2207039211)
    S = assemble(Mesh.from_synth(m), kernel="constant", delta=0.3, ball="approxcaps", precision="fp64",
                 f_nodal=np.full(m.M, -4.0))
    g = m.verts[:, 0] ** 2 + m.verts[:, 1] ** 2
    u, info = S.solve(g, tol_rel=1e-12, max_iter=3)
    assert info["status"] == -6, info
    assert info["iterations"] == 3 and info["rel_residual"] > 1e-12, info
    assert bool(torch.isfinite(u).all())
    u2, info2 = S.solve(g, tol_rel=1e-10)
    assert info2["status"] == 0 and info2["rel_residual"] <= 1e-10, info2
