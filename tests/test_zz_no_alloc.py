"""nlfem_pairs_noalloc: the interaction graph without any device allocation.

Some callers cannot allocate device memory when they need the element pairs: code
inside a CUDA graph capture, a server that reserved all device memory up front for its
own arena, or code that must not be able to fail with out-of-memory. This entry point
works entirely in caller buffers plus a fixed file-scope device array. Its pairs must be
exactly those of the regular path (nlfem_assemble, then nlfem_mesh_pairs), call after
call, since the shared array keeps whatever the previous call left in it.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2207_03921_gb300 import Mesh, NlfemError, assemble, binding  # noqa: E402
from synth import meshes  # noqa: E402


@pytest.mark.parametrize("ball,nq,delta", [("approxcaps", 16, 0.12), ("nocaps", 7, 0.1), ("infinity", 7, 0.1)])
def test_pairs_noalloc_matches_the_regular_pair_search(ball, nq, delta):
    m = meshes.jittered_delaunay(-0.1, 1.1, 30, 0.03, seed=2207039219)
    mesh = Mesh.from_synth(m)
    assemble(mesh, kernel="constant", delta=delta, ball=ball, quad_outer=nq)
    k_ref, l_ref = mesh.pairs()
    # the caller owns inputs and outputs; the entry point allocates nothing
    verts = torch.as_tensor(m.verts).cuda()
    elems = torch.as_tensor(m.elems).cuda()
    cap = int(k_ref.numel()) + 64
    out_k = torch.empty(cap, dtype=torch.int32, device="cuda")
    out_l = torch.empty(cap, dtype=torch.int32, device="cuda")
    for _ in range(2):  # two calls in a row on the same shared scratch
        out_k.fill_(-1)
        out_l.fill_(-1)
        n = binding.nlfem_pairs_noalloc(verts, elems, delta, ball, nq, out_k, out_l)
        assert n == k_ref.numel()
        assert torch.equal(out_k[:n], k_ref) and torch.equal(out_l[:n], l_ref)


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
