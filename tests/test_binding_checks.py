"""Host-side argument checks of the binding (no GPU): wrong dtypes, shapes, strides or
devices are refused before any pointer reaches the C library."""
import pytest

torch = pytest.importorskip("torch")

from paper_2207_03921_gb300 import binding  # noqa: E402


def _args():
    verts = torch.zeros(10, 2, dtype=torch.float64)
    elems = torch.zeros(4, 3, dtype=torch.int32)
    out_k = torch.zeros(64, dtype=torch.int32)
    out_l = torch.zeros(64, dtype=torch.int32)
    return verts, elems, out_k, out_l


@pytest.mark.parametrize("which,bad,msg", [
    (0, torch.zeros(10, 2, dtype=torch.float32), "verts must be a float64"),
    (0, torch.zeros(10, 3, dtype=torch.float64), "verts must be a float64"),
    (1, torch.zeros(4, 3, dtype=torch.int64), "elems must be an int32"),
    (1, torch.zeros(12, dtype=torch.int32), "elems must be an int32"),
    (2, torch.zeros(64, dtype=torch.int64), "out_k must be"),
    (3, torch.zeros(8, 8, dtype=torch.int32), "out_l must be"),
    (0, torch.zeros(2, 10, dtype=torch.float64).t(), "verts must be contiguous"),
    (3, torch.zeros(128, dtype=torch.int32)[::2], "out_l must be contiguous"),
])
def test_pairs_noalloc_refuses_bad_tensors(which, bad, msg):
    a = list(_args())
    a[which] = bad
    with pytest.raises(ValueError, match=msg):
        binding.nlfem_pairs_noalloc(a[0], a[1], 0.1, "nocaps", 7, a[2], a[3])


def test_pairs_noalloc_refuses_host_tensors():
    verts, elems, out_k, out_l = _args()
    with pytest.raises(ValueError, match="CUDA tensor"):
        binding.nlfem_pairs_noalloc(verts, elems, 0.1, "nocaps", 7, out_k, out_l)


def test_pairs_noalloc_capacity_is_the_shorter_output():
    _, _, out_k, out_l = _args()
    assert binding._noalloc_capacity(out_k, out_l[:10]) == 10
    assert binding._noalloc_capacity(out_k[:7], out_l) == 7
