"""nlfem_pairs_noalloc: the interaction graph without any device allocation.

Some callers cannot allocate device memory when they need the element pairs: a server
that reserved all device memory up front for its own arena, a host framework whose
caching allocator owns the device memory, or code that must not be able to fail with
out-of-memory. This entry point works entirely in caller buffers plus a fixed file-scope
device array. Its pairs must be exactly those of the regular path (nlfem_assemble, then
nlfem_mesh_pairs), call after call, since the shared array keeps whatever the previous
call left in it.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2207_03921_gb300 import Mesh, NlfemError, assemble, binding  # noqa: E402
from synth import meshes  # noqa: E402


def _regular_pairs(m, ball, nq, delta):
    mesh = Mesh.from_synth(m)
    assemble(mesh, kernel="constant", delta=delta, ball=ball, quad_outer=nq, precision="fp32_bulk")
    k_ref, l_ref = mesh.pairs()
    return k_ref.clone(), l_ref.clone()


def _noalloc(m, ball, nq, delta, cap):
    # the caller owns inputs and outputs; the entry point allocates nothing
    verts = torch.as_tensor(m.verts).cuda()
    elems = torch.as_tensor(m.elems).cuda()
    out_k = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    out_l = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    n = binding.nlfem_pairs_noalloc(verts, elems, delta, ball, nq, out_k, out_l)
    return n, out_k, out_l


@pytest.mark.parametrize("ball,nq,delta", [("approxcaps", 16, 0.12), ("nocaps", 7, 0.1), ("infinity", 7, 0.1)])
def test_pairs_noalloc_matches_the_regular_pair_search(ball, nq, delta):
    m = meshes.jittered_delaunay(-0.1, 1.1, 30, 0.03, seed=2207039219)
    k_ref, l_ref = _regular_pairs(m, ball, nq, delta)
    cap = int(k_ref.numel()) + 64
    for _ in range(2):  # two calls in a row on the same shared scratch
        n, out_k, out_l = _noalloc(m, ball, nq, delta, cap)
        assert n == k_ref.numel()
        assert torch.equal(out_k[:n], k_ref) and torch.equal(out_l[:n], l_ref)


def test_pairs_noalloc_large_rows_and_scratch_left_by_another_mesh():
    # a mesh whose elements have more than 512 partners (the block-per-segment sort), and a
    # small mesh whose result must not change after the large one filled the shared array
    # with other cells, counts and offsets
    big = meshes.structured(0.0, 1.0, 64)          # 8,192 triangles, h = 1/64
    small = meshes.jittered_delaunay(-0.1, 1.1, 30, 0.03, seed=2207039219)
    kb, lb = _regular_pairs(big, "nocaps", 7, 0.25)  # delta / h = 16
    partners = np.bincount(kb.cpu().numpy(), minlength=big.K)
    assert partners.max() > 512
    ks, ls = _regular_pairs(small, "approxcaps", 16, 0.12)
    n0, k0, l0 = _noalloc(small, "approxcaps", 16, 0.12, int(ks.numel()) + 8)
    assert n0 == ks.numel() and torch.equal(k0[:n0], ks) and torch.equal(l0[:n0], ls)
    n1, k1, l1 = _noalloc(big, "nocaps", 7, 0.25, int(kb.numel()))
    assert n1 == kb.numel() and torch.equal(k1[:n1], kb) and torch.equal(l1[:n1], lb)
    n2, k2, l2 = _noalloc(small, "approxcaps", 16, 0.12, int(ks.numel()) + 8)
    assert n2 == ks.numel() and torch.equal(k2[:n2], ks) and torch.equal(l2[:n2], ls)


def test_pairs_noalloc_limits():
    m = meshes.structured(0.0, 1.0, 130)  # 33,800 triangles: above the 32,768 limit
    verts = torch.as_tensor(m.verts).cuda()
    elems = torch.as_tensor(m.elems).cuda()
    out = torch.empty(16, dtype=torch.int32, device="cuda")
    with pytest.raises(NlfemError) as e:
        binding.nlfem_pairs_noalloc(verts, elems, 0.05, "nocaps", 7, out, out.clone())
    assert e.value.code == -8
    small = meshes.structured(0.0, 1.0, 8)
    v = torch.as_tensor(small.verts).cuda()
    el = torch.as_tensor(small.elems).cuda()
    with pytest.raises(NlfemError) as e:  # capacity too small: the needed count comes back
        binding.nlfem_pairs_noalloc(v, el, 0.3, "nocaps", 7, out, out.clone())
    assert e.value.code == -1 and e.value.npairs > 16
    with pytest.raises(NlfemError) as e:  # the capacity is the shorter of the two outputs
        binding.nlfem_pairs_noalloc(v, el, 0.3, "nocaps", 7, torch.empty(10**6, dtype=torch.int32, device="cuda"),
                                    out.clone())
    assert e.value.code == -1
