"""The arithmetic of the FP32-bulk path, each setting pinned against the FP64 oracle.

- Singular rule (Sec. 2.3.2, Tab. 1 club): FP64 by default, FP32 on request. With a horizon
  far below the mesh size only intersecting pairs interact, so the whole matrix is the
  singular rule: in FP64 the bulk result then equals the oracle up to the fixed-point
  rounding (about 1e-12 of the largest contribution), in FP32 it carries the FP32 rounding
  of the transform points and sums.
- Cut geometry (Defs. 2.1, 2.2): FP32 decisions and positions by default, every cut outer
  point cut in FP64 on request. Both stay within the 1e-5 bar, and their difference is the
  geometry's FP32 contribution; structured grids with delta a multiple of h put vertices on
  the circle (ties) and are covered too.
- The FP64 path ignores both settings.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2207_03921_gb300 import Mesh, assemble  # noqa: E402
from synth import meshes  # noqa: E402


def vals(S):
    rp, col, val = (t.cpu().numpy() for t in S.csr())
    return rp, col, val


def rel(val, ref):
    return np.linalg.norm(val - ref) / np.linalg.norm(ref)


@pytest.mark.parametrize("s", [0.5, 0.25, 0.75])
def test_singular_rule_precision(s):
    m = meshes.jittered_delaunay(-0.1, 1.1, 16, 0.05, seed=31)
    kw = dict(kernel="fractional", s=s, delta=0.004, ball="approxcaps", quad_outer=7, quad_inner=7)
    ref = oracle.assemble(m, **kw)
    assert ref.counts["pairs_separated"] == 0  # every interacting pair shares a vertex
    mesh = Mesh.from_synth(m)
    errs = {}
    for sp in ("fp64", "fp32"):
        S = assemble(mesh, precision="fp32_bulk", singular_precision=sp, **kw)
        rp, col, val = vals(S)
        assert np.array_equal(rp, ref.row_ptr) and np.array_equal(col, ref.col)
        errs[sp] = rel(val, ref.val)
    assert errs["fp64"] <= 1e-10, errs
    assert 1e-9 < errs["fp32"] <= 1e-5, errs


def test_singular_rule_precision_in_the_full_problem():
    # the configuration-2 shape at small size: both settings within the bar, FP64 no worse
    m = meshes.jittered_delaunay(-0.1, 1.1, 30, 0.03, seed=2207039212)
    kw = dict(kernel="fractional", s=0.5, delta=0.1, ball="approxcaps", quad_outer=16, quad_inner=16)
    ref = oracle.assemble(m, **kw)
    mesh = Mesh.from_synth(m)
    e = {}
    for sp in ("fp64", "fp32"):
        _, _, val = vals(assemble(mesh, precision="fp32_bulk", singular_precision=sp, **kw))
        e[sp] = rel(val, ref.val)
    assert e["fp64"] <= 1e-5 and e["fp32"] <= 1e-5, e
    assert e["fp64"] <= e["fp32"] * 1.05, e


JIT = ("jittered", lambda: meshes.jittered_delaunay(-0.1, 1.1, 24, 0.03, seed=2207039213))
# structured grids with delta a multiple of h: vertices lie exactly on the circle or on a side
# of the square for the outer points at vertices (ties)
TIES = ("structured_ties", lambda: meshes.structured(-0.2, 1.2, 28))


@pytest.mark.parametrize("mesh,kw", [
    (JIT, dict(kernel="constant", delta=0.1, ball="nocaps")),
    (JIT, dict(kernel="fractional", s=0.5, delta=0.1, ball="approxcaps", quad_outer=16, quad_inner=16)),
    (JIT, dict(kernel="peridynamic", delta=0.12, ball="nocaps")),
    (JIT, dict(kernel="constant", delta=0.1, ball="infinity")),
    (TIES, dict(kernel="constant", delta=0.25, ball="nocaps")),
    (TIES, dict(kernel="constant", delta=0.2, ball="approxcaps")),
    (TIES, dict(kernel="peridynamic", delta=0.2, ball="nocaps")),
    (TIES, dict(kernel="constant", delta=0.1, ball="infinity")),
], ids=lambda v: v[0] if isinstance(v, tuple) else "-".join(str(x) for x in v.values()))
def test_geometry_precision(mesh, kw):
    m = mesh[1]()
    ndof = 2 if kw["kernel"] == "peridynamic" else 1
    ref = oracle.assemble(m, **kw)
    mesh = Mesh.from_synth(m, ndof)
    out = {}
    for gp in ("fp32", "fp64"):
        S = assemble(mesh, precision="fp32_bulk", geometry_precision=gp, **kw)
        rp, col, val = vals(S)
        assert np.array_equal(rp, ref.row_ptr) and np.array_equal(col, ref.col)
        out[gp] = val
        assert rel(val, ref.val) <= 1e-5, (gp, rel(val, ref.val))
        # the result is the same bits in every run whatever the setting
        _, _, again = vals(assemble(mesh, precision="fp32_bulk", geometry_precision=gp, **kw))
        assert np.array_equal(again, val)
    d = rel(out["fp32"], out["fp64"])
    assert 0.0 < d <= 1e-6, d  # the switch changes the positions, by FP32 rounding only


def test_fp64_path_ignores_the_bulk_settings():
    m = meshes.jittered_delaunay(-0.1, 1.1, 16, 0.05, seed=31)
    kw = dict(kernel="fractional", s=0.5, delta=0.15, ball="approxcaps")
    mesh = Mesh.from_synth(m)
    _, _, a = vals(assemble(mesh, precision="fp64", **kw))
    _, _, b = vals(assemble(mesh, precision="fp64", singular_precision="fp32", geometry_precision="fp64", **kw))
    assert np.array_equal(a, b)
