"""GPU parity: the CUDA path against the FP64 oracle on the same seeded meshes.

Bars: the CSR pattern (row_ptr, col) and the interaction graph are bit-exact; FP64
values agree entrywise to 1e-12 relative, floored at 1e-3 of the row's largest entry
(tiny entries come from sliver sub-triangles whose relative error is ill-conditioned);
FP32-bulk values agree to 1e-5 in relative Frobenius norm; A is symmetric bit for bit
and identical from run to run; the load vectors agree to 1e-12 (FP64).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2207_03921_gb300 import Mesh, NlfemError, assemble  # noqa: E402
from synth import meshes  # noqa: E402


def gpu_csr(S):
    rp, col, val = (t.cpu().numpy() for t in S.csr())
    return rp, col, val


def rowmax(rp, val):
    out = np.zeros(len(val))
    for i in range(len(rp) - 1):
        s, e = rp[i], rp[i + 1]
        if e > s:
            out[s:e] = np.abs(val[s:e]).max()
    return out


def check_fp64(S, ref, tol=1e-12):
    rp, col, val = gpu_csr(S)
    assert np.array_equal(rp, ref.row_ptr), "row_ptr differs from the oracle"
    assert np.array_equal(col, ref.col), "column indices differ from the oracle"
    floor = 1e-3 * rowmax(rp, ref.val)
    err = np.abs(val - ref.val) / np.maximum(np.abs(ref.val), floor)
    assert err.max() <= tol, f"max floored relative error {err.max():.3e}"
    return rp, col, val


def check_bulk(S, ref, tol=1e-5):
    rp, col, val = gpu_csr(S)
    assert np.array_equal(rp, ref.row_ptr) and np.array_equal(col, ref.col)
    fro = np.linalg.norm(val - ref.val) / np.linalg.norm(ref.val)
    assert fro <= tol, f"relative Frobenius error {fro:.3e}"
    return rp, col, val


def symmetric_bitwise(rp, col, val):
    import scipy.sparse as sp
    A = sp.csr_matrix((val, col, rp), shape=(len(rp) - 1, len(rp) - 1))
    return (A != A.T).nnz == 0


CASES = {
    # cfg 1: constant kernel, nocaps, 7-point rules, structured h = 0.05 on [-0.1, 1.1]^2
    "cfg1_constant_nocaps": (meshes.cfg1_mesh, dict(kernel="constant", delta=0.1, ball="nocaps")),
    # cfg 2 shape at small size: fractional s = 0.5, approxcaps, 16-point rules, jittered Delaunay
    "cfg2_small_fractional": (lambda: meshes.jittered_delaunay(-0.1, 1.1, 30, 0.03, seed=2207039212),
                              dict(kernel="fractional", s=0.5, delta=0.1, ball="approxcaps",
                                   quad_outer=16, quad_inner=16)),
    # cfg 3 shape at small size: peridynamics, delta = 4h, structured
    "cfg3_small_peridynamic": (lambda: meshes.structured(-0.2, 1.2, 20),
                               dict(kernel="peridynamic", delta=0.28, ball="nocaps")),
    # general fractional order through exp2/log2, 16-point outer / 7-point inner
    "fractional_s075_mixed_rules": (lambda: meshes.jittered_delaunay(-0.15, 1.15, 18, 0.05, seed=4),
                                    dict(kernel="fractional", s=0.75, delta=0.15, ball="nocaps",
                                         quad_outer=16, quad_inner=7)),
    # constant kernel with approxcaps on a structured grid: many exact distance ties
    "constant_approxcaps_ties": (lambda: meshes.structured(-0.2, 1.2, 28),
                                 dict(kernel="constant", delta=0.2, ball="approxcaps")),
    # infinity ball, delta = 2h on a structured grid: the square's sides run along mesh lines
    "infinity_constant_ties": (lambda: meshes.structured(-0.2, 1.2, 28),
                               dict(kernel="constant", delta=0.1, ball="infinity")),
    # infinity ball, fractional kernel, 16-point rules, jittered Delaunay
    "infinity_fractional_jittered": (lambda: meshes.jittered_delaunay(-0.15, 1.15, 18, 0.05, seed=6),
                                     dict(kernel="fractional", s=0.5, delta=0.15, ball="infinity",
                                          quad_outer=16, quad_inner=16)),
    # infinity ball, peridynamics, delta = 3h
    "infinity_peridynamic": (lambda: meshes.structured(-0.2, 1.2, 20),
                             dict(kernel="peridynamic", delta=0.21, ball="infinity")),
    # user-defined radial kernel from a table (a Gaussian bump on 33 nodes), approxcaps
    "tabulated_gaussian": (lambda: meshes.jittered_delaunay(-0.2, 1.2, 20, 0.05, seed=31),
                           dict(kernel="tabulated", delta=0.2, ball="approxcaps", kconst=50.0,
                                kernel_table=np.exp(-3.0 * np.linspace(0.0, 1.0, 33) ** 2))),
    # user-defined kernel on the infinity ball (held beyond delta), 16-point inner rule, ties
    "tabulated_infinity": (lambda: meshes.structured(-0.2, 1.2, 28),
                           dict(kernel="tabulated", delta=0.1, ball="infinity", quad_inner=16,
                                kernel_table=np.array([2.0, 1.5, 0.5, 0.25, 0.1]))),
}


@pytest.fixture(scope="module")
def refs():
    cache = {}

    def get(name):
        if name not in cache:
            mk, kw = CASES[name]
            m = mk()
            ndof = 2 if kw["kernel"] == "peridynamic" else 1
            rng = np.random.default_rng(1)
            f = rng.standard_normal(m.M * ndof)
            cache[name] = (m, kw, f, oracle.assemble(m, f_nodal=f, **kw))
        return cache[name]
    return get


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_matches_oracle(refs, name):
    m, kw, f, ref = refs(name)
    ndof = 2 if kw["kernel"] == "peridynamic" else 1
    mesh = Mesh.from_synth(m, ndof)
    S = assemble(mesh, precision="fp64", f_nodal=f, **kw)
    rp, col, val = check_fp64(S, ref)
    assert symmetric_bitwise(rp, col, val)
    F = S.rhs().cpu().numpy()
    assert np.max(np.abs(F - ref.F)) <= 1e-12 * np.max(np.abs(ref.F))
    info = S.info()
    assert info["npairs"] == ref.counts["pairs"]
    assert info["pairs_identical"] == ref.counts["pairs_identical"]
    assert info["pairs_edge"] == ref.counts["pairs_edge"]
    assert info["pairs_vertex"] == ref.counts["pairs_vertex"]
    # the interaction graph itself
    k, l = mesh.pairs()
    got = set(zip(k.cpu().numpy().tolist(), l.cpu().numpy().tolist()))
    want = set(map(tuple, ref.pairs.tolist()))
    assert got == want
    assert np.array_equal(S.dirichlet().cpu().numpy(), ref.dirichlet)


@pytest.mark.parametrize("name", list(CASES))
def test_fp32_bulk_matches_oracle(refs, name):
    m, kw, f, ref = refs(name)
    ndof = 2 if kw["kernel"] == "peridynamic" else 1
    mesh = Mesh.from_synth(m, ndof)
    S = assemble(mesh, precision="fp32_bulk", f_nodal=f, **kw)
    rp, col, val = check_bulk(S, ref)
    assert symmetric_bitwise(rp, col, val)


def test_deterministic_and_cached(refs):
    m, kw, f, ref = refs("cfg2_small_fractional")
    mesh = Mesh.from_synth(m)
    a = assemble(mesh, precision="fp32_bulk", **kw)
    b = assemble(mesh, precision="fp32_bulk", **kw)
    assert b.info()["cached"] == 1 and a.info()["cached"] == 0
    va, vb = a.csr()[2].cpu().numpy(), b.csr()[2].cpu().numpy()
    assert np.array_equal(va.view(np.uint64), vb.view(np.uint64))
    c = assemble(Mesh.from_synth(m), precision="fp64", **kw)
    d = assemble(Mesh.from_synth(m), precision="fp64", **kw)
    assert np.array_equal(c.csr()[2].cpu().numpy().view(np.uint64), d.csr()[2].cpu().numpy().view(np.uint64))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32_bulk", 1e-6)])
def test_null_spaces(precision, tol):
    m = meshes.jittered_delaunay(-0.2, 1.2, 16, 0.1, seed=8)
    for kw in (dict(kernel="constant", delta=0.25, ball="approxcaps"),
               dict(kernel="fractional", s=0.5, delta=0.25, ball="nocaps")):
        S = assemble(Mesh.from_synth(m), precision=precision, **kw)
        A = S.to_torch_sparse()
        scale = S.csr()[2].abs().max().item()
        r = (A @ torch.ones(S.N, dtype=torch.float64, device="cuda")).abs().max().item()
        assert r <= tol * scale * 10
    mp = Mesh.from_synth(m, 2)
    S = assemble(mp, kernel="peridynamic", delta=0.25, precision=precision)
    A = S.to_torch_sparse()
    scale = S.csr()[2].abs().max().item()
    x = torch.as_tensor(m.verts[:, 0], device="cuda")
    y = torch.as_tensor(m.verts[:, 1], device="cuda")
    for mode in (torch.stack([torch.ones_like(x), 0 * x], 1), torch.stack([0 * x, torch.ones_like(x)], 1),
                 torch.stack([-y, x], 1)):
        r = (A @ mode.reshape(-1).contiguous()).abs().max().item()
        assert r <= tol * scale * 10


def test_solve_residual_and_oracle_solution(refs):
    m, kw, f, ref = refs("cfg1_constant_nocaps")
    mesh = Mesh.from_synth(m)
    fval = -4.0 * np.ones(m.M)
    g = m.verts[:, 0] ** 2 + m.verts[:, 1] ** 2
    S = assemble(mesh, precision="fp64", f_nodal=fval, **kw)
    u, info = S.solve(g, tol_rel=1e-10)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-10, info
    ref2 = oracle.assemble(m, f_nodal=fval, **kw)
    u_ref = oracle.solve_dirichlet(ref2, g)
    u = u.cpu().numpy()
    assert np.linalg.norm(u - u_ref) <= 1e-9 * np.linalg.norm(u_ref)
    assert np.array_equal(u[ref2.dirichlet], g[ref2.dirichlet])
    Sb = assemble(mesh, precision="fp32_bulk", f_nodal=fval, **kw)
    ub, infob = Sb.solve(g, tol_rel=1e-10)
    assert infob["rel_residual"] <= 1e-10
    assert np.linalg.norm(ub.cpu().numpy() - u_ref) <= 1e-5 * np.linalg.norm(u_ref)


def test_edge_cases():
    # one triangle: only the (0, 0) pair
    m = meshes.Mesh(np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]]), np.array([[0, 2, 1]], dtype=np.int32),
                    np.array([1], dtype=np.int8), 1.0)
    ref = oracle.assemble(m, kernel="constant", delta=0.3, ball="approxcaps")
    S = assemble(Mesh.from_synth(m), kernel="constant", delta=0.3, ball="approxcaps")
    check_fp64(S, ref)
    # a horizon far below the mesh size: only touching pairs interact
    m2 = meshes.structured(0.0, 1.0, 9)
    ref = oracle.assemble(m2, kernel="fractional", s=0.25, delta=1e-3)
    S = assemble(Mesh.from_synth(m2), kernel="fractional", s=0.25, delta=1e-3)
    check_fp64(S, ref)
    assert S.info()["pairs_separated"] == 0
    # a horizon covering the whole mesh: every pair interacts
    m3 = meshes.jittered_delaunay(0.0, 1.0, 5, 0.1, seed=3)
    ref = oracle.assemble(m3, kernel="constant", delta=3.0)
    S = assemble(Mesh.from_synth(m3), kernel="constant", delta=3.0)
    check_fp64(S, ref)
    assert S.info()["npairs"] == m3.K * m3.K


def test_error_codes():
    m = meshes.structured(0.0, 1.0, 4)
    mesh = Mesh.from_synth(m)
    with pytest.raises(NlfemError) as e:
        assemble(mesh, kernel="constant", delta=-1.0)
    assert e.value.code == -1
    with pytest.raises(NlfemError) as e:
        assemble(mesh, kernel="peridynamic", delta=0.3)  # the mesh has 1 dof per node
    assert e.value.code == -1
    with pytest.raises(NlfemError) as e:
        assemble(mesh, kernel="fractional", s=1.5, delta=0.3)
    assert e.value.code == -1
    with pytest.raises(NlfemError) as e:
        assemble(mesh, kernel="constant", delta=0.3, mem_budget_bytes=1024)
    assert e.value.code == -4
    bad = np.array([[0, 1, 99]], dtype=np.int32)
    with pytest.raises(NlfemError) as e:
        Mesh(m.verts, bad)
    assert e.value.code == -2
    degenerate = np.array([[0, 1, 2]], dtype=np.int32)  # three collinear grid nodes
    with pytest.raises(NlfemError) as e:
        Mesh(m.verts, degenerate)
    assert e.value.code == -2
    # the library still works after errors
    S = assemble(mesh, kernel="constant", delta=0.3)
    assert S.info()["npairs"] > 0


@pytest.mark.parametrize("kw", [dict(kernel="constant", delta=0.25, ball="approxcaps"),
                                dict(kernel="peridynamic", delta=0.25, ball="nocaps")],
                         ids=lambda k: k["kernel"])
def test_neumann_solve_matches_oracle(kw):
    # pure Neumann-type problem: every element in Omega, so no Dirichlet node; the load is not
    # compatible (nonzero mean), the solve projects it
    base = meshes.jittered_delaunay(0.0, 1.0, 12, 0.1, seed=21)
    m = meshes.Mesh(base.verts, base.elems, np.ones(base.K, dtype=np.int8), base.h)
    ndof = 2 if kw["kernel"] == "peridynamic" else 1
    f = np.stack([1.0 + m.verts[:, 0], m.verts[:, 1] - 0.2], 1)[:, :ndof].reshape(-1)
    ref = oracle.assemble(m, f_nodal=f, **kw)
    assert not ref.dirichlet.any()
    u_ref = oracle.solve_neumann(ref, m.verts)
    S = assemble(Mesh.from_synth(m, ndof), precision="fp64", f_nodal=f, **kw)
    u, info = S.solve_neumann(tol_rel=1e-10)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-10, info
    u = u.cpu().numpy()
    assert np.linalg.norm(u - u_ref) <= 1e-8 * np.linalg.norm(u_ref)
    Sb = assemble(Mesh.from_synth(m, ndof), precision="fp32_bulk", f_nodal=f, **kw)
    ub, infob = Sb.solve_neumann(tol_rel=1e-10)
    assert infob["rel_residual"] <= 1e-10, infob
    assert np.linalg.norm(ub.cpu().numpy() - u_ref) <= 1e-4 * np.linalg.norm(u_ref)


def test_paper_E5_infinity_ball_on_gpu():
    """Sec. 3.3, fixed h = 8.84e-3 (grid spacing a = 0.00625) and delta -> 0, assembled and
    solved on the GPU. The errors here are the modelling error of the exact infinity ball
    (relative symbol deficit 2 k^2 delta^2 / 15 for u = sin(kx) sin(ky)), 1.2 to 1.7 times the
    printed ones, which fall off like an isotropic ball's (k^2 delta^2 / 12): second order
    and the magnitude are pinned, not the printed digits."""
    import json, math, os
    tab = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))
    tab = tab["E5_infinity_fixed_h"]
    ue = lambda x, y: np.sin(4 * math.pi * x) * np.sin(4 * math.pi * y)
    errs = []
    for delta in tab["delta"]:
        m = meshes.paper_square(delta, 0.00625)
        x, y = m.verts[:, 0], m.verts[:, 1]
        S = assemble(Mesh.from_synth(m), kernel="constant", delta=delta, ball="infinity",
                     precision="fp32_bulk", f_nodal=32 * math.pi ** 2 * ue(x, y))
        u, info = S.solve(ue(x, y), tol_rel=1e-10)
        assert info["status"] == 0, info
        errs.append(oracle.l2_error(m, u.cpu().numpy(), ue))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    for r in rates:
        assert 1.8 < r < 2.6, (rates, errs)
    for i, e in enumerate(errs):
        assert 0.5 * tab["l2"][i] < e < 2.0 * tab["l2"][i], (errs, tab["l2"])


@pytest.mark.parametrize("precision", ["fp64", "fp32_bulk"])
def test_label_dependent_kernel_matches_oracle(precision):
    # four materials in the quadrants, a symmetric scale table (Sec. 1: kernels depending on
    # element labels, interface problems)
    m = meshes.jittered_delaunay(-0.2, 1.2, 16, 0.05, seed=23)
    c = m.verts[m.elems].mean(1)
    mat = ((c[:, 0] > 0.5).astype(np.int8) + 2 * (c[:, 1] > 0.5)).astype(np.int8)
    tab = np.array([[1.0, 0.5, 0.3, 0.2], [0.5, 2.0, 0.4, 0.1], [0.3, 0.4, 3.0, 0.6], [0.2, 0.1, 0.6, 0.7]])
    for kw in (dict(kernel="constant", delta=0.2, ball="approxcaps"),
               dict(kernel="fractional", s=0.5, delta=0.2, ball="nocaps"),
               dict(kernel="peridynamic", delta=0.2, ball="infinity")):
        ndof = 2 if kw["kernel"] == "peridynamic" else 1
        ref = oracle.assemble(m, materials=mat, material_scale=tab, **kw)
        mesh = Mesh.from_synth(m, ndof)
        mesh.set_materials(mat)
        S = assemble(mesh, precision=precision, material_scale=tab, **kw)
        if precision == "fp64":
            rp, col, val = check_fp64(S, ref)
        else:
            rp, col, val = check_bulk(S, ref)
        assert symmetric_bitwise(rp, col, val)
    # the table must be symmetric, and labels must exist and fit the table
    with pytest.raises(NlfemError):
        assemble(mesh, precision=precision, material_scale=tab + np.triu(np.ones((4, 4)), 1), **kw)
    with pytest.raises(NlfemError):
        assemble(mesh, precision=precision, material_scale=np.ones((2, 2)), **kw)
    fresh = Mesh.from_synth(m, ndof)
    with pytest.raises(NlfemError):
        assemble(fresh, precision=precision, material_scale=tab, **kw)


@pytest.mark.parametrize("precision", ["fp64", "fp32_bulk"])
def test_dg_matches_oracle(precision):
    # discontinuous P1 ansatz: the GPU mesh copies the vertices per element (node 3k + a), the
    # oracle assembles the same copied mesh; pairs are classified by vertex positions
    m = meshes.jittered_delaunay(-0.2, 1.2, 14, 0.05, seed=35)
    d = meshes.discontinuous(m)
    rng = np.random.default_rng(4)
    for kw in (dict(kernel="constant", delta=0.25, ball="approxcaps"),
               dict(kernel="peridynamic", delta=0.25, ball="nocaps"),
               dict(kernel="tabulated", delta=0.25, ball="infinity", kernel_table=np.array([2.0, 1.0, 0.5])),
               # singular kernels with s <= 1/2: touching pairs in the factored form (Tab. 1)
               dict(kernel="fractional", s=0.5, delta=0.25, ball="approxcaps"),
               dict(kernel="fractional", s=0.25, delta=0.25, ball="nocaps"),
               dict(kernel="constant", delta=0.25, ball="nocaps", close_rule="duffy")):
        ndof = 2 if kw["kernel"] == "peridynamic" else 1
        f = rng.standard_normal(d.M * ndof)
        ref = oracle.assemble(d, f_nodal=f, **kw)
        mesh = Mesh.from_synth(m, ndof, dg=True)
        S = assemble(mesh, precision=precision, f_nodal=f, **kw)
        rp, col, val = check_fp64(S, ref) if precision == "fp64" else check_bulk(S, ref)
        assert symmetric_bitwise(rp, col, val)
        F = S.rhs().cpu().numpy()
        assert np.abs(F - ref.F).max() <= 1e-12 * np.abs(ref.F).max()
        assert np.array_equal(S.dirichlet().cpu().numpy().astype(bool), ref.dirichlet)
    # Tab. 1: no discontinuous ansatz for s > 1/2
    with pytest.raises(NlfemError):
        assemble(Mesh.from_synth(m, 1, dg=True), kernel="fractional", s=0.75, delta=0.25, precision=precision)


def test_dg_singular_rule_variants():
    """The factored singular rule on a DG mesh (k_duffy_split) with other Gauss orders (3, 8), with
    material labels (the pair factor of its records), and inside a batched assembly (the close
    list of a fused batch), against the oracle and against single assemblies."""
    from paper_2207_03921_gb300 import assemble_batch
    m = meshes.jittered_delaunay(-0.2, 1.2, 10, 0.05, seed=36)
    d = meshes.discontinuous(m)
    rng = np.random.default_rng(6)
    f = rng.standard_normal(d.M)
    for n, kw in ((3, dict(kernel="fractional", s=0.3, delta=0.3, ball="nocaps")),
                  (8, dict(kernel="fractional", s=0.5, delta=0.3, ball="approxcaps"))):
        ref = oracle.assemble(d, f_nodal=f, duffy_n=n, **kw)
        S = assemble(Mesh.from_synth(m, 1, dg=True), precision="fp64", f_nodal=f, duffy_gauss=n, **kw)
        rp, col, val = check_fp64(S, ref)
        assert symmetric_bitwise(rp, col, val)
    c = m.verts[m.elems].mean(1)
    mat = ((c[:, 0] > 0.5).astype(np.int8) + 2 * (c[:, 1] > 0.5)).astype(np.int8)
    tab = np.array([[1.0, 0.5, 0.3, 0.2], [0.5, 2.0, 0.4, 0.1], [0.3, 0.4, 3.0, 0.6], [0.2, 0.1, 0.6, 0.7]])
    kw = dict(kernel="fractional", s=0.5, delta=0.3, ball="approxcaps")
    ref = oracle.assemble(d, materials=mat, material_scale=tab, **kw)
    for precision in ("fp64", "fp32_bulk"):
        mesh = Mesh.from_synth(m, 1, dg=True)
        mesh.set_materials(mat)
        S = assemble(mesh, precision=precision, material_scale=tab, **kw)
        rp, col, val = check_fp64(S, ref) if precision == "fp64" else check_bulk(S, ref)
        assert symmetric_bitwise(rp, col, val)
    # batched: a DG item under the singular rule beside a continuous one
    kwb = dict(kw, precision="fp32_bulk")
    m2 = meshes.structured(-0.1, 1.1, 16, name="s16")
    single = [assemble(Mesh.from_synth(m, 1, dg=True), **kwb), assemble(Mesh.from_synth(m2, 1), **kwb)]
    batch = assemble_batch([Mesh.from_synth(m, 1, dg=True), Mesh.from_synth(m2, 1)], [kwb, kwb])
    for S0, S1 in zip(single, batch):
        for a, b in zip(S0.csr(), S1.csr()):
            assert torch.equal(a, b)
    check_bulk(batch[0], oracle.assemble(d, **kw))

def test_paper_E2_fractional_dg_on_gpu():
    """Sec. 3.1's DG table for the truncated fractional kernel (s = 1/2, delta = 0.2, approxcaps),
    assembled (FP32 bulk) and solved on the GPU on the first four grids: second-order rates and
    the printed magnitudes. (The fifth grid's DG pattern holds about 2.6e9 entries.)"""
    import json, math, os
    tab = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))
    tab = tab["E2_fractional_dg"]
    errs = []
    for a in tab["a"][:4]:
        m = meshes.paper_square(0.2, a)
        d = meshes.discontinuous(m)
        S = assemble(Mesh.from_synth(m, 1, dg=True), kernel="fractional", s=0.5, delta=0.2, ball="approxcaps",
                     precision="fp32_bulk", f_nodal=-2.0 * (d.verts[:, 1] + 1.0))
        ue = lambda x, y: x * x * y + y * y
        u, info = S.solve(ue(d.verts[:, 0], d.verts[:, 1]), tol_rel=1e-10)
        assert info["status"] == 0, info
        errs.append(oracle.l2_error(d, u.cpu().numpy(), ue))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    for r in rates:
        assert 1.7 < r < 2.4, (rates, errs)
    for i, e in enumerate(errs):
        assert 0.4 * tab["l2"][i] < e < 2.5 * tab["l2"][i], (errs, tab["l2"])


def test_paper_E4_peridynamic_dg_on_gpu():
    """Sec. 3.2's DG table for bond-based peridynamics (delta = 0.1), assembled and solved on the
    GPU on all five grids: second-order rates and the printed magnitudes."""
    import json, math, os
    tab = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))
    tab = tab["E4_peridynamics_dg"]
    errs = []
    for a in tab["a"]:
        m = meshes.paper_square(0.1, a)
        d = meshes.discontinuous(m)
        x, y = d.verts[:, 0], d.verts[:, 1]
        f = -0.5 * math.pi * np.stack([1.0 + 2.0 * x, y], 1).reshape(-1)
        g = np.stack([y * y, x * x * y], 1).reshape(-1)
        S = assemble(Mesh.from_synth(m, 2, dg=True), kernel="peridynamic", delta=0.1, ball="approxcaps",
                     precision="fp32_bulk", f_nodal=f)
        u, info = S.solve(g, tol_rel=1e-10)
        assert info["status"] == 0, info
        ue = lambda x, y: np.stack([y * y, x * x * y])
        errs.append(oracle.l2_error(d, u.cpu().numpy(), ue, ndof=2))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    for r in rates:
        assert 1.7 < r < 2.4, (rates, errs)
    for i, e in enumerate(errs):
        assert 0.4 * tab["l2"][i] < e < 2.5 * tab["l2"][i], (errs, tab["l2"])
