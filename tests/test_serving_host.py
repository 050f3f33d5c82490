"""Scheduling of the serving loop on the host (no GPU): admission by the device-memory
budget, slots, arrival order, rejection of requests larger than the budget, failures."""
import threading
import time

import numpy as np

from paper_2207_03921_gb300.serving import Request, Server, estimate_bytes, estimate_pairs


def _req(i, arrival, nbytes):
    v = np.zeros((3, 2))
    e = np.zeros((1, 3), dtype=np.int32)
    lab = np.ones(1, dtype=np.int8)
    return Request(id=i, arrival=arrival, verts=v, elems=e, labels=lab, delta=0.1, est_bytes=nbytes)


def test_admission_respects_budget_and_slots():
    inflight = []
    peak = {"n": 0, "bytes": 0}
    lock = threading.Lock()

    def fake(req, res, slot):
        with lock:
            inflight.append(req)
            peak["n"] = max(peak["n"], len(inflight))
            peak["bytes"] = max(peak["bytes"], sum(r.est_bytes for r in inflight))
        time.sleep(0.003 + 0.001 * (req.id % 3))
        res.pairs = 10
        with lock:
            inflight.remove(req)

    sizes = [30, 50, 20, 70, 10, 40, 60, 25, 35, 45, 15, 55]
    reqs = [_req(i, 0.0005 * i, b) for i, b in enumerate(sizes)] + [_req(99, 0.001, 1000)]
    st = Server(budget_bytes=100, slots=3, execute=fake).run(reqs, realtime=True)
    res = {r.id: r for r in st.results}
    assert res[99].error and "admission" in res[99].error
    ok = [r for r in st.results if r.id != 99]
    assert all(r.error is None for r in ok)
    assert peak["n"] <= 3 and peak["bytes"] <= 100
    assert st.max_inflight >= 2  # requests overlap
    # admitted in arrival order, never before arrival
    adm = [res[i].admitted for i in range(len(sizes))]
    assert all(a <= b + 1e-9 for a, b in zip(adm, adm[1:]))
    assert all(res[i].admitted >= reqs[i].arrival - 1e-9 for i in range(len(sizes)))
    s = st.summary()
    assert s["completed"] == len(sizes) and s["failed"] == 1 and s["p99_ms"] >= s["p50_ms"] > 0


def test_failed_request_does_not_stop_the_loop():
    def fake(req, res, slot):
        if req.id == 2:
            raise RuntimeError("CG did not converge")
        res.pairs = 1

    reqs = [_req(i, 0.0, 10) for i in range(5)]
    st = Server(budget_bytes=100, slots=2, execute=fake).run(reqs, realtime=False)
    errs = {r.id: r.error for r in st.results}
    assert errs[2] and "CG" in errs[2]
    assert all(errs[i] is None for i in (0, 1, 3, 4))


def test_estimates_grow_with_delta_and_size():
    a = estimate_pairs(10000, 1.44, 0.05)
    b = estimate_pairs(10000, 1.44, 0.1)
    c = estimate_pairs(40000, 1.44, 0.1)
    assert a < b < c
    # a structured mesh of 600^2 cells with delta = 0.01: about 2.1e8 pairs measured
    p = estimate_pairs(720000, 1.02 ** 2, 0.01)
    assert 1.5e8 < p < 3.5e8
    assert estimate_bytes(361201, 720000, 1.02 ** 2, 0.01) > 2e10


def _tri_req(i, arrival, nbytes):
    v = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    e = np.array([[0, 1, 2]], dtype=np.int32)
    return Request(id=i, arrival=arrival, verts=v, elems=e, labels=np.ones(1, dtype=np.int8), delta=0.1,
                   est_bytes=nbytes)


def test_requests_admitted_together_are_assembled_as_one_batch():
    groups, singles = [], []
    lock = threading.Lock()

    def single(req, res, slot):
        with lock:
            singles.append(req.id)
        res.pairs = 1

    def batch(reqs, ress, slots):
        assert len(set(slots)) == len(slots) == len(reqs) > 1
        with lock:
            groups.append([r.id for r in reqs])

        def cont(res):
            time.sleep(0.002)
            res.pairs = 1
        return [lambda res=res: cont(res) for res in ress]

    # a burst of 4 at t = 0 fills the 4 slots in one pass; the later arrivals come one at a time
    reqs = [_tri_req(i, 0.0, 10) for i in range(4)] + [_tri_req(4 + i, 0.05 + 0.02 * i, 10) for i in range(3)]
    st = Server(budget_bytes=1000, slots=4, execute=single, execute_batch=batch).run(reqs, realtime=True)
    assert all(r.error is None and r.pairs == 1 for r in st.results)
    assert groups and sorted(groups[0]) == [0, 1, 2, 3]
    assert sorted(sum(groups, []) + singles) == list(range(7))
    assert st.max_inflight == 4


def test_a_failed_batch_fails_its_requests_only():
    def single(req, res, slot):
        res.pairs = 1

    def batch(reqs, ress, slots):
        if 0 in [r.id for r in reqs]:
            raise RuntimeError("batched assembly failed")
        return [lambda: None for _ in reqs]

    reqs = [_tri_req(i, 0.0, 10) for i in range(3)] + [_tri_req(3, 0.05, 10)]
    st = Server(budget_bytes=1000, slots=3, execute=single, execute_batch=batch).run(reqs, realtime=True)
    errs = {r.id: r.error for r in st.results}
    assert all(errs[i] and "batched assembly failed" in errs[i] for i in range(3))
    assert errs[3] is None


def test_batching_off_runs_every_request_alone():
    seen = []

    def single(req, res, slot):
        seen.append(req.id)

    def batch(reqs, ress, slots):
        raise AssertionError("batching is off")

    reqs = [_tri_req(i, 0.0, 10) for i in range(4)]
    st = Server(budget_bytes=1000, slots=4, execute=single, execute_batch=batch, batch=False).run(reqs,
                                                                                                   realtime=False)
    assert sorted(seen) == [0, 1, 2, 3] and all(r.error is None for r in st.results)
