"""Batched assembly (nlfem_batch_assemble): every system equals its single assembly bit for
bit, across kernel classes (constant nocaps, fractional approxcaps with the singular rule,
peridynamics) and with an FP64 item in the same call; error cases."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2207_03921_gb300 import Mesh, NlfemError, assemble, assemble_batch  # noqa: E402
from synth import meshes  # noqa: E402


def _items():
    specs = [s for s in meshes.serving_requests(n_requests=128) if s["K_target"] <= 3000][:6]
    out = []
    for sp in specs:
        m = meshes.request_mesh(sp)
        kw = dict(kernel=sp["kernel"], delta=sp["delta"], s=sp["s"],
                  ball="approxcaps" if sp["kernel"] == "fractional" else "nocaps", precision="fp32_bulk")
        out.append((m, 1, kw))
    # a peridynamic item and an FP64 item
    m3 = meshes.structured(-0.1, 1.1, 24, name="s24")
    out.append((m3, 2, dict(kernel="peridynamic", delta=0.1, precision="fp32_bulk")))
    out.append((meshes.structured(-0.1, 1.1, 24, name="s24b"), 1, dict(kernel="constant", delta=0.1, precision="fp64")))
    return out


def _host(S):
    rp, col, val = (t.cpu().numpy() for t in S.csr())
    return rp, col, val, S.rhs().cpu().numpy()


def test_batch_equals_single_bitwise():
    items = _items()
    assert len({(kw["kernel"], kw.get("ball")) for _, _, kw in items}) >= 3
    single = []
    for m, nd, kw in items:
        mesh = Mesh.from_synth(m, nd)
        f = np.linspace(-1.0, 1.0, m.M * nd)
        single.append(_host(assemble(mesh, f_nodal=f, **kw)))
    ms = [Mesh.from_synth(m, nd) for m, nd, _ in items]
    fs = [np.linspace(-1.0, 1.0, m.M * nd) for m, nd, _ in items]
    systems = assemble_batch(ms, [kw for _, _, kw in items], fs)
    for (rp0, col0, val0, F0), S in zip(single, systems):
        rp, col, val, F = _host(S)
        assert np.array_equal(rp, rp0) and np.array_equal(col, col0)
        assert np.array_equal(val, val0)
        assert np.array_equal(F, F0)


def test_batch_cached_second_call_and_errors():
    m = meshes.structured(-0.1, 1.1, 20, name="s20")
    a, b = Mesh.from_synth(m), Mesh.from_synth(m)
    kw = dict(kernel="constant", delta=0.1, precision="fp32_bulk")
    first = assemble_batch([a, b], [kw, kw])
    again = assemble_batch([a, b], [kw, kw])  # pair lists and patterns cached in the handles
    assert again[0].info()["cached"] == 1
    assert np.array_equal(first[0].csr()[2].cpu().numpy(), again[1].csr()[2].cpu().numpy())
    with pytest.raises(NlfemError):
        assemble_batch([a, a], [kw, kw])
    assert assemble_batch([], []) == []


def test_batch_plan_graph_replay_equals_single():
    items = [it for it in _items() if it[2]["precision"] == "fp32_bulk"]
    ms = [Mesh.from_synth(m, nd) for m, nd, _ in items]
    fs = [np.linspace(-1.0, 1.0, m.M * nd) for m, nd, _ in items]
    single = [_host(assemble(Mesh.from_synth(m, nd), f_nodal=f, **kw)) for (m, nd, kw), f in zip(items, fs)]
    from paper_2207_03921_gb300 import BatchPlan
    plan = BatchPlan(ms, [kw for _, _, kw in items], fs)
    for rep in range(2):
        t = plan.run()
        assert t > 0
        for (rp0, col0, val0, F0), S in zip(single, plan.systems):
            rp, col, val, F = _host(S)
            assert np.array_equal(val, val0) and np.array_equal(F, F0)
    with pytest.raises(NlfemError):
        BatchPlan(ms[:1], [dict(items[0][2], precision="fp64")])


@pytest.mark.parametrize("kw", [dict(kernel="constant", delta=0.1, ball="nocaps"),
                                dict(kernel="fractional", s=0.5, delta=0.1, ball="approxcaps", quad_outer=16,
                                     quad_inner=16)])
def test_autotune_keeps_results(kw):
    # the launch shape (grid size, outer points per chunk of the cut-pair kernel) changes the
    # schedule only: every shape gives the same bits
    from paper_2207_03921_gb300 import autotune, tune_set
    m = meshes.jittered_delaunay(-0.1, 1.1, 30, 0.03, seed=2207039219)
    mesh = Mesh.from_synth(m)
    kw = dict(kw, precision="fp32_bulk")
    tune_set((64, 64, 0), **kw)
    before = assemble(mesh, **kw).csr()[2].cpu().numpy()
    for shape in ((2, 3, 1), (8, 4, 2), (16, 1, 5)):   # non-default grids and chunks
        tune_set(shape, **kw)
        assert np.array_equal(assemble(mesh, **kw).csr()[2].cpu().numpy(), before), shape
    best = autotune(mesh, **kw)
    assert best[0] in (2, 4, 8, 16, 32, 64) and best[1] in (2, 4, 8, 16, 32, 64)
    assert 1 <= best[2] <= (8 if kw["ball"] == "approxcaps" else 7)
    after = assemble(mesh, **kw).csr()[2].cpu().numpy()
    assert np.array_equal(before, after)
    with pytest.raises(NlfemError):
        tune_set((0, 4, 2), **kw)


def _items_extended():
    """Infinity ball (FP32 cut passes on a jittered mesh, FP64 on a grid the square follows), a
    tabulated user kernel, a discontinuous peridynamic mesh and a label-dependent kernel."""
    jm = meshes.jittered_delaunay(-0.2, 1.2, 22, 0.05, seed=41)
    sm = meshes.structured(-0.2, 1.2, 28, name="s28")
    c = jm.verts[jm.elems].mean(1)
    mat = (c[:, 0] > 0.5).astype(np.int8)
    return [
        (jm, 1, dict(kernel="constant", delta=0.15, ball="infinity", precision="fp32_bulk"), {}),
        (sm, 1, dict(kernel="constant", delta=0.1, ball="infinity", precision="fp32_bulk"), {}),
        (jm, 1, dict(kernel="tabulated", delta=0.15, ball="approxcaps", precision="fp32_bulk",
                     kernel_table=np.array([1.0, 0.7, 0.2])), {}),
        (sm, 2, dict(kernel="peridynamic", delta=0.15, ball="nocaps", precision="fp32_bulk"), {"dg": True}),
        (jm, 1, dict(kernel="constant", delta=0.15, ball="nocaps", precision="fp32_bulk",
                     material_scale=np.array([[1.0, 0.4], [0.4, 2.5]])), {"mat": mat}),
    ]


def _mesh(m, nd, extra):
    mesh = Mesh.from_synth(m, nd, dg=extra.get("dg", False))
    if "mat" in extra:
        mesh.set_materials(extra["mat"])
    return mesh


def test_batch_and_graph_with_infinity_ball_dg_and_user_kernels():
    items = _items_extended()
    fs = [np.linspace(-1.0, 1.0, _mesh(m, nd, ex).M * nd) for m, nd, _, ex in items]
    single = [_host(assemble(_mesh(m, nd, ex), f_nodal=f, **kw)) for (m, nd, kw, ex), f in zip(items, fs)]
    ms = [_mesh(m, nd, ex) for m, nd, _, ex in items]
    systems = assemble_batch(ms, [kw for _, _, kw, _ in items], fs)
    for (rp0, col0, val0, F0), S in zip(single, systems):
        rp, col, val, F = _host(S)
        assert np.array_equal(rp, rp0) and np.array_equal(col, col0)
        assert np.array_equal(val, val0) and np.array_equal(F, F0)
    from paper_2207_03921_gb300 import BatchPlan
    plan = BatchPlan([_mesh(m, nd, ex) for m, nd, _, ex in items], [kw for _, _, kw, _ in items], fs)
    for rep in range(2):
        plan.run()
        for (rp0, col0, val0, F0), S in zip(single, plan.systems):
            rp, col, val, F = _host(S)
            assert np.array_equal(val, val0) and np.array_equal(F, F0)
