"""Parity at full size on the benchmark configurations other than the 720k mesh, sampled rows.

A row i of A only receives contributions from ordered pairs (E_k, E_l) with node i among
the vertices of E_k or E_l. Interacting elements satisfy |c_k - c_l| <= R + r_k + r_l
(centroids c, radii r, R = delta for the Euclidean balls and sqrt(2) delta for the infinity
ball), so every outer element of such a pair has its centroid within R + 3 r_max of node i.
The oracle assembles those outer elements only and keeps only the pairs that touch a sampled
node (node_keep), which leaves the sampled rows exactly those of the full assembly. The GPU
assembles the whole mesh in the configuration bench.py times (FP32 bulk with its cached
pattern) and in plain FP64.

- cfg2: jittered Delaunay h = 0.01 (28,800 triangles), fractional s = 1/2, delta = 0.1
  (delta / h = 10: more than 512 partners per element, so the block-per-segment sort and the
  large-row pattern build run), approxcaps, 16-point rules, singular rule on touching pairs
  (Sec. 3.1 kernel, Tab. 1 club).
- cfg3: bond-based peridynamics on the structured h = 0.005 mesh (86,528 triangles, two dofs
  per node, Tab. 1 diamond on intersecting pairs; Sec. 3.2 kernel).
- inf_e5: the Sec. 3.3 infinity-ball problem at delta = 0.2 on spacing 0.00625 (41,472
  triangles, delta / h = 32, about 9,000 partners per element).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2207_03921_gb300 import Mesh, assemble  # noqa: E402
from synth import meshes  # noqa: E402

CASES = {
    "cfg2": dict(mesh=meshes.cfg2_mesh, ndof=1, reach=0.1, big_rows=True, nrand=6,
                 kw=dict(kernel="fractional", s=0.5, delta=0.1, ball="approxcaps", quad_outer=16, quad_inner=16)),
    "cfg3": dict(mesh=meshes.cfg3_mesh, ndof=2, reach=0.02, big_rows=False, nrand=6,
                 kw=dict(kernel="peridynamic", delta=0.02, ball="nocaps", quad_outer=7, quad_inner=7)),
    "inf_e5": dict(mesh=lambda: meshes.paper_square(0.2, 0.00625), ndof=1, reach=0.2 * math.sqrt(2.0),
                   big_rows=True, nrand=3,
                   kw=dict(kernel="constant", delta=0.2, ball="infinity", quad_outer=7, quad_inner=7)),
}


def sample_nodes(m, nrand, seed=11):
    rng = np.random.default_rng(seed)
    x, y = m.verts[:, 0], m.verts[:, 1]
    picks = [int(v) for v in rng.choice(m.M, size=nrand, replace=False)]
    lo, hi = x.min(), x.max()
    mid = 0.5 * (lo + hi)
    picks.append(int(np.argmin(x + y)))                                  # corner of the base domain
    picks.append(int(np.argmin(np.abs(x - 0.0) + np.abs(y - mid))))     # on the boundary of Omega
    picks.append(int(np.argmin(np.abs(x - mid) + np.abs(y - mid))))     # centre
    return sorted(set(picks))


def load_data(m, ndof):
    if ndof == 2:
        return np.tile(np.array([0.0, -1.0]), m.M)   # body force (0, -1) of configuration 3
    return -4.0 * np.ones(m.M)


def gpu_rows(S, rows):
    rp, col, val = S.csr_views()
    rp_h = rp.cpu().numpy()
    F = S.rhs()
    out = {}
    for r in rows:
        s, e = int(rp_h[r]), int(rp_h[r + 1])
        out[r] = (col[s:e].cpu().numpy(), val[s:e].cpu().numpy(), float(F[r]))
    return out


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    name = request.param
    cfg = CASES[name]
    m = cfg["mesh"]()
    ndof = cfg["ndof"]
    nodes = sample_nodes(m, cfg["nrand"])
    rows = [i * ndof + d for i in nodes for d in range(ndof)]
    f = load_data(m, ndof)
    mesh = Mesh.from_synth(m, ndof)
    got = {}
    bulk = assemble(mesh, precision="fp32_bulk", f_nodal=f, **cfg["kw"])
    del bulk
    bulk = assemble(mesh, precision="fp32_bulk", f_nodal=f, **cfg["kw"])   # cached pattern, as timed
    got["bulk"] = gpu_rows(bulk, rows)
    info = bulk.info()
    del bulk
    plain = assemble(mesh, precision="fp64", f_nodal=f, **cfg["kw"])
    got["plain"] = gpu_rows(plain, rows)
    del plain
    k, _ = mesh.pairs()
    partners = torch.bincount(k.long(), minlength=m.K).cpu().numpy()
    del mesh, k
    torch.cuda.empty_cache()
    # the oracle's rows: outer elements near the sampled nodes, pairs touching them
    c = m.verts[m.elems].mean(1)
    r = np.sqrt(((m.verts[m.elems] - c[:, None, :]) ** 2).sum(-1)).max()
    near = np.zeros(m.K, dtype=bool)
    for i in nodes:
        near |= np.hypot(c[:, 0] - m.verts[i, 0], c[:, 1] - m.verts[i, 1]) <= cfg["reach"] + 3 * r + 1e-12
    keep = np.zeros(m.M, dtype=bool)
    keep[nodes] = True
    ref = oracle.assemble(m, elem_subset=np.flatnonzero(near).astype(np.int32), node_keep=keep, f_nodal=f,
                          **cfg["kw"])
    return dict(name=name, m=m, cfg=cfg, nodes=nodes, rows=rows, got=got, ref=ref, info=info,
                partners=partners)


def test_rows_match_oracle(case):
    ref = case["ref"]
    for r in case["rows"]:
        s, e = ref.row_ptr[r], ref.row_ptr[r + 1]
        col_ref, val_ref, F_ref = ref.col[s:e], ref.val[s:e], ref.F[r]
        assert len(col_ref) > 0
        for name in ("plain", "bulk"):
            col, val, F = case["got"][name][r]
            assert np.array_equal(col, col_ref), f"{case['name']} {name}: pattern of row {r} differs"
            if name == "plain":
                # entrywise 1e-12, floored at 1e-3 of the row's largest entry
                floor = 1e-3 * np.abs(val_ref).max()
                err = np.abs(val - val_ref) / np.maximum(np.abs(val_ref), floor)
                assert err.max() <= 1e-12, (case["name"], r, err.max())
            else:
                err = np.linalg.norm(val - val_ref) / np.linalg.norm(val_ref)
                assert err <= 1e-5, (case["name"], r, err)
            assert abs(F - F_ref) <= 1e-12 * max(1.0, abs(F_ref)), (case["name"], name, r, F, F_ref)


def test_row_sums_vanish(case):
    # A 1 = 0 (scalar) and A t = 0 for the translations (peridynamics) hold row by row
    ndof = case["cfg"]["ndof"]
    for name in ("plain", "bulk"):
        for r in case["rows"]:
            col, val, _ = case["got"][name][r]
            for d in range(ndof):
                sel = (col % ndof) == d
                tol = (1e-13 if name == "plain" else 1e-6) * np.abs(val).max() * math.sqrt(len(val))
                assert abs(val[sel].sum()) <= tol, (case["name"], name, r, d, val[sel].sum())


def test_sampled_rows_reach_the_large_row_paths(case):
    # delta / h of configuration 2 and of the Sec. 3.3 problem gives elements with more than
    # 512 partners: the pair lists are sorted by the block-per-segment sort and the pattern
    # rows are long; the sampled rows contain such elements
    if not case["cfg"]["big_rows"]:
        pytest.skip("delta / h = 4: fewer than 512 partners per element by construction")
    m = case["m"]
    star = np.isin(m.elems, case["nodes"]).any(1)
    assert case["partners"].max() > 512
    assert case["partners"][star].max() > 512
    assert case["info"]["npairs"] == int(case["partners"].sum())
