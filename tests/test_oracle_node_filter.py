"""The oracle's node filter (node_keep) used by the full-size row tests: the rows of the
flagged nodes equal those of the full assembly bit for bit, and pairs that cannot write into
them are dropped. Pinned against the unfiltered oracle on small meshes (CPU)."""
import numpy as np
import pytest

import oracle
from synth import meshes


def _row(S, i, ndof):
    out = {}
    for d in range(ndof):
        r = i * ndof + d
        s, e = S.row_ptr[r], S.row_ptr[r + 1]
        out[d] = (S.col[s:e].copy(), S.val[s:e].copy())
    return out


@pytest.mark.parametrize("kw", [
    dict(kernel="fractional", s=0.5, delta=0.3, ball="approxcaps", quad_outer=7, quad_inner=16),
    dict(kernel="peridynamic", delta=0.25, ball="nocaps"),
    dict(kernel="constant", delta=0.2, ball="infinity"),
])
def test_node_filter_keeps_the_rows_of_flagged_nodes(kw):
    m = meshes.jittered_delaunay(-0.25, 1.25, 9, 0.03, seed=5)
    ndof = 2 if kw["kernel"] == "peridynamic" else 1
    full = oracle.assemble(m, **kw)
    rng = np.random.default_rng(3)
    picks = rng.choice(m.M, size=4, replace=False)
    keep = np.zeros(m.M, dtype=bool)
    keep[picks] = True
    part = oracle.assemble(m, node_keep=keep, **kw)
    assert 0 < part.counts["pairs"] < full.counts["pairs"]
    # every kept pair touches a flagged node; every full pair touching one is kept
    T = m.elems
    touch = keep[T[full.pairs[:, 0]]].any(1) | keep[T[full.pairs[:, 1]]].any(1)
    assert part.counts["pairs"] == int(touch.sum())
    for i in picks:
        a, b = _row(full, i, ndof), _row(part, i, ndof)
        for d in range(ndof):
            assert np.array_equal(a[d][0], b[d][0])
            assert np.array_equal(a[d][1], b[d][1])  # same pairs summed in the same order
