"""Serving loop on the GPU: each result is the same alone and in the mix (bitwise: the FP32
bulk sums are integer fixed point and each request's work is independent of the others; in
the mix the requests admitted together are assembled as one batch),
requests overlap, every solve reaches the 1e-10 FP64 relative residual, and a short Poisson
stream completes with p50 <= p99."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2207_03921_gb300.serving import Server, make_request  # noqa: E402
from synth import meshes  # noqa: E402


def _requests(n, kmax, at_once):
    specs = [s for s in meshes.serving_requests(n_requests=256) if s["K_target"] <= kmax][:n]
    reqs = []
    for s in specs:
        r = make_request(s, meshes.request_mesh(s))
        if at_once:
            r.arrival = 0.0
        reqs.append(r)
    return reqs


def test_same_result_alone_and_in_the_mix():
    reqs = _requests(8, 4000, at_once=True)
    kinds = {(r.kernel, r.s) for r in reqs}
    assert len(kinds) >= 2  # constant and fractional requests mixed
    alone = Server(slots=1, keep_values=True, cache_meshes=False).run(reqs, realtime=False)
    mix = Server(slots=4, keep_values=True, cache_meshes=False).run(reqs, realtime=False)
    assert mix.max_inflight > 1
    assert not any(r.batched for r in alone.results) and sum(r.batched for r in mix.results) >= 2
    for a, b in zip(alone.results, mix.results):
        assert a.error is None and b.error is None, (a.error, b.error)
        assert a.rel_residual <= 1e-10 and b.rel_residual <= 1e-10
        assert np.array_equal(a.val, b.val)
        assert np.array_equal(a.u, b.u)


def test_short_poisson_stream():
    reqs = _requests(24, 8000, at_once=False)
    srv = Server(budget_bytes=8 << 30, slots=4)
    st = srv.run(reqs, realtime=True)
    srv.close()
    s = st.summary()
    assert s["completed"] == len(reqs), [r.error for r in st.results if r.error]
    assert s["p99_ms"] >= s["p50_ms"] > 0
    assert st.max_used_bytes <= 8 << 30
    assert all(r.rel_residual <= 1e-10 for r in st.results)
