"""Serving loop: assemble-and-solve requests of uneven size as they arrive.

Requests (mesh, delta, kernel) arrive as a Poisson stream. The scheduler admits a request
when a slot is free and its estimated device memory fits the budget; each admitted
request runs on a stream of its own, driven by its own host thread, so the kernels of
several requests overlap on the GPU while new requests keep being admitted as slots and
memory free up (continuous batching, not a queue alone). A request uploads its mesh,
assembles A and F (nlfem_assemble, pair search and pattern included), solves the
nonlocal Dirichlet problem with FP64 residual refinement (nlfem_solve) and copies u
back; its latency is completion minus arrival. Small requests admitted in the same
scheduling pass are assembled together by nlfem_batch_assemble, which fuses the bulk
quadrature of all of them into one launch per kernel class; each then solves on its own
slot's stream and thread.

Meshes with their pair lists and CSR patterns stay on the device in an LRU cache under
the same budget, so a repeated (mesh, delta, ball) skips the pair search and pattern.
All device work goes through the C ABI; this module only schedules.
"""
from __future__ import annotations

import functools
import hashlib
import math
import threading
import time
from collections import OrderedDict, deque
from dataclasses import dataclass, field

import numpy as np

# bytes per ordered pair held during and after a cold FP32-bulk assembly: pair list and class
# (9), transposed index (4), work lists (4) and the whole pairs' elements (8), kl ranks (18),
# ll records (24), search temporaries (about 60)
BYTES_PER_PAIR = 128
# bytes per CSR entry: column (4), value (8), transposed position (8), node pattern (4),
# fixed-point sums (8 per upper entry)
BYTES_PER_NNZ = 28
# requests with fewer estimated ordered pairs than this are assembled in batches: a larger one
# fills the GPU by itself, and alone it keeps its cold path (pair search, pattern) overlapped
# with the other slots' work
BATCH_MAX_PAIRS = 4_000_000


def estimate_pairs(K: int, area: float, delta: float) -> float:
    """Ordered interacting pairs of a quasi-uniform mesh: K * pi (delta + 2 r)^2 / |E|."""
    e_area = area / max(K, 1)
    r = math.sqrt(2.0 * e_area)  # about the element diameter
    return K * math.pi * (delta + r) ** 2 / e_area


def estimate_bytes(M: int, K: int, area: float, delta: float, ndof: int = 1) -> int:
    """Device bytes of one cold assembly plus solve (upper estimate used for admission)."""
    pairs = estimate_pairs(K, area, delta)
    e_area = area / max(K, 1)
    r = math.sqrt(2.0 * e_area)
    nnz = M * math.pi * (delta + 2 * r) ** 2 / (e_area / 2.0) * ndof * ndof
    vectors = 16 * M * ndof * 8
    return int(pairs * BYTES_PER_PAIR + nnz * BYTES_PER_NNZ + vectors + 64 * K + (64 << 20))


@dataclass
class Request:
    id: int
    arrival: float                 # seconds after the start of the stream
    verts: np.ndarray              # [M, 2] float64
    elems: np.ndarray              # [K, 3] int32
    labels: np.ndarray             # [K] int8, 1 = Omega
    delta: float
    kernel: str = "constant"
    s: float = 0.5
    ball: str = "nocaps"
    precision: str = "fp32_bulk"
    quad_outer: int = 7
    quad_inner: int = 7
    est_bytes: int = 0

    def key(self) -> str:
        h = hashlib.sha1()
        h.update(self.verts.tobytes())
        h.update(self.elems.tobytes())
        h.update(self.labels.tobytes())
        return h.hexdigest()


@dataclass
class Result:
    id: int
    arrival: float
    admitted: float = 0.0
    done: float = 0.0
    u: np.ndarray | None = None
    val: np.ndarray | None = None
    pairs: int = 0
    iterations: int = 0
    rel_residual: float = float("nan")
    error: str | None = None
    cached_mesh: bool = False
    batched: bool = False     # assembled in a batch with other requests (nlfem_batch_assemble)
    t_mesh: float = 0.0       # upload and mesh preparation (s)
    t_assemble: float = 0.0   # nlfem_assemble (pair search and pattern unless cached)
    t_solve: float = 0.0      # nlfem_solve and the copy of u to the host

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def make_request(spec: dict, mesh) -> Request:
    """Request of the serving stream (synth.meshes.serving_requests) on its mesh."""
    kernel = spec["kernel"]
    return Request(id=spec["id"], arrival=spec["arrival"], verts=mesh.verts, elems=mesh.elems,
                   labels=mesh.elem_label, delta=spec["delta"], kernel=kernel, s=spec["s"],
                   ball="approxcaps" if kernel == "fractional" else "nocaps")


class MemoryBudget:
    """Device-memory admission: reserve an estimate, settle to the bytes actually held."""

    def __init__(self, budget: int):
        self.budget = int(budget)
        self.used = 0
        self.cv = threading.Condition()

    def fits(self, n: int) -> bool:
        return self.used + n <= self.budget

    def reserve(self, n: int):
        self.used += n

    def release(self, n: int):
        with self.cv:
            self.used -= n
            self.cv.notify_all()


class MeshCache:
    """Device-resident meshes (with their pair lists and patterns), LRU under the budget."""

    def __init__(self, budget: MemoryBudget, capacity: int = 64):
        self.items: OrderedDict[tuple, tuple] = OrderedDict()   # key -> (mesh, bytes, users)
        self.budget = budget
        self.capacity = capacity
        self.lock = threading.Lock()

    def get(self, key):
        """The cached mesh (marked in use), or None; a mesh in use by another request is not
        shared (its pair cache may be rebuilt for other parameters)."""
        with self.lock:
            it = self.items.get(key)
            if it is None or it[2] > 0:
                return None
            mesh, nbytes, users = it
            self.items[key] = (mesh, nbytes, users + 1)
            self.items.move_to_end(key)
            return mesh

    def put(self, key, mesh, nbytes) -> bool:
        """Keep a mesh after its request if its bytes fit the budget (evicting idle meshes,
        oldest first); returns False if it was not kept."""
        with self.budget.cv:
            freed = self.evict_for(nbytes)
            self.budget.used -= freed
            if not self.budget.fits(nbytes):
                return False
            self.budget.used += nbytes
            with self.lock:
                self.items[key] = (mesh, nbytes, 0)
                self.items.move_to_end(key)
            return True

    def done(self, key):
        with self.lock:
            it = self.items.get(key)
            if it is not None:
                self.items[key] = (it[0], it[1], it[2] - 1)

    def evict_for(self, need: int) -> int:
        """Drop idle meshes (oldest first) until need bytes fit; returns bytes freed."""
        freed = 0
        with self.lock:
            for key in list(self.items):
                if self.budget.used + need - freed <= self.budget.budget and len(self.items) <= self.capacity:
                    break
                mesh, nbytes, users = self.items[key]
                if users == 0:
                    del self.items[key]
                    freed += nbytes
        return freed


@dataclass
class Stats:
    results: list = field(default_factory=list)
    wall: float = 0.0
    max_inflight: int = 0
    max_used_bytes: int = 0

    def summary(self) -> dict:
        ok = [r for r in self.results if r.error is None]
        lat = np.array([r.latency for r in ok]) * 1e3
        pairs = sum(r.pairs for r in ok)
        return {"requests": len(self.results), "completed": len(ok),
                "failed": len(self.results) - len(ok),
                "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
                "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
                "mean_ms": float(lat.mean()) if len(lat) else None,
                "wall_s": self.wall, "requests_per_s": len(ok) / self.wall if self.wall else None,
                "pairs_per_s": pairs / self.wall if self.wall else None,
                "max_inflight": self.max_inflight, "max_device_bytes_reserved": self.max_used_bytes,
                "batched": sum(r.batched for r in ok),
                "mean_mesh_ms": float(np.mean([r.t_mesh for r in ok]) * 1e3) if ok else None,
                "mean_assemble_ms": float(np.mean([r.t_assemble for r in ok]) * 1e3) if ok else None,
                "mean_solve_ms": float(np.mean([r.t_solve for r in ok]) * 1e3) if ok else None,
                "mean_cg_iterations": float(np.mean([r.iterations for r in ok])) if ok else None,
                "max_cg_iterations": int(max(r.iterations for r in ok)) if ok else None}


class Server:
    """Continuous-batching request loop over the C ABI (one stream and host thread per slot).

    budget_bytes: device-memory admission budget; slots: requests in flight at most;
    keep_results: copy u (and optionally the CSR values) back to the host for checking.
    execute: the per-request work (default: upload, assemble, solve); replaceable for
    host-only tests of the scheduling. batch: assemble the small requests admitted in one
    scheduling pass together (nlfem_batch_assemble); execute_batch(reqs, results, slots)
    does it and returns one callable per request that finishes it (default: upload,
    batched assembly, then per request solve), replaceable like execute.
    """

    def __init__(self, budget_bytes: int = 40 << 30, slots: int = 8, keep_values: bool = False,
                 execute=None, cache_meshes: bool = True, clock=time.perf_counter, batch: bool = True,
                 execute_batch=None):
        self.budget = MemoryBudget(budget_bytes)
        self.slots = slots
        self.keep_values = keep_values
        self.execute = execute or self._execute
        if execute_batch is None and execute is None:
            execute_batch = self._execute_batch
        self.execute_batch = execute_batch if batch else None
        self.cache = MeshCache(self.budget) if cache_meshes and execute is None else None
        self.clock = clock
        self._streams = None

    def close(self):
        """Drop the cached meshes (their device memory is freed)."""
        if self.cache is not None:
            with self.cache.lock:
                self.cache.items.clear()

    # ---- per-request device work -------------------------------------------------------
    def _prepare(self, req: Request, res: Result, stream):
        """Mesh handle (cached or uploaded), load f and Dirichlet data g on the device."""
        import torch
        from .api import Mesh
        key = (req.key(), 1)
        mesh = self.cache.get(key) if self.cache else None
        res.cached_mesh = mesh is not None
        if mesh is None:
            mesh = Mesh(req.verts, req.elems, req.labels, 1, stream=stream)
        x, y = req.verts[:, 0], req.verts[:, 1]
        f = torch.full((len(x),), -4.0, dtype=torch.float64, device="cuda")
        g = torch.as_tensor(x * x + y * y, dtype=torch.float64).cuda()
        return key, mesh, f, g

    @staticmethod
    def _params(req: Request) -> dict:
        return dict(kernel=req.kernel, delta=req.delta, s=req.s, ball=req.ball, quad_outer=req.quad_outer,
                    quad_inner=req.quad_inner, precision=req.precision)

    def _solve_finish(self, req: Request, res: Result, slot: int, key, mesh, g, S):
        """Solve on the slot's stream, copy u back, hand the mesh to the cache."""
        import torch
        stream = self._streams[slot]
        clk = time.perf_counter
        with torch.cuda.stream(stream):
            info = S.info()
            t = clk()
            u, sinfo = S.solve(g, tol_rel=1e-10, stream=stream)
            res.u = u.cpu().numpy()
            res.t_solve = clk() - t
            if self.keep_values:
                res.val = S.csr_views()[2].cpu().numpy()
            res.pairs = int(info["npairs"])
            res.iterations = int(sinfo["iterations"])
            res.rel_residual = float(sinfo["rel_residual"])
            held = mesh.device_bytes()
            del S
            stream.synchronize()
            if self.cache is not None and not res.cached_mesh:
                if not self.cache.put(key, mesh, held):
                    del mesh
            elif self.cache is not None:
                self.cache.done(key)
            return held

    def _execute(self, req: Request, res: Result, slot: int):
        import torch
        from .api import assemble
        stream = self._streams[slot]
        clk = time.perf_counter
        with torch.cuda.stream(stream):
            t = clk()
            key, mesh, f, g = self._prepare(req, res, stream)
            stream.synchronize()
            res.t_mesh = clk() - t
            t = clk()
            S = assemble(mesh, f_nodal=f, stream=stream, **self._params(req))
            stream.synchronize()
            res.t_assemble = clk() - t
        return self._solve_finish(req, res, slot, key, mesh, g, S)

    def _execute_batch(self, reqs: list, ress: list, slots: list) -> list:
        import torch
        from .api import assemble_batch
        stream = self._streams[slots[0]]
        clk = time.perf_counter
        with torch.cuda.stream(stream):
            t = clk()
            preps = [self._prepare(req, res, stream) for req, res in zip(reqs, ress)]
            stream.synchronize()
            t_mesh = (clk() - t) / len(reqs)
            t = clk()
            systems = assemble_batch([p[1] for p in preps], [self._params(r) for r in reqs], [p[2] for p in preps],
                                     stream=stream)
            stream.synchronize()
            t_asm = clk() - t
        conts = []
        for req, res, slot, (key, mesh, _, g), S in zip(reqs, ress, slots, preps, systems):
            res.t_mesh, res.t_assemble, res.batched = t_mesh, t_asm, True
            conts.append(functools.partial(self._solve_finish, req, res, slot, key, mesh, g, S))
        return conts

    # ---- the loop -------------------------------------------------------------------------
    def run(self, requests: list[Request], realtime: bool = True) -> Stats:
        """Serve the requests in arrival order; realtime = wait for each arrival time."""
        if self.execute == self._execute:
            import torch
            self._streams = [torch.cuda.Stream() for _ in range(self.slots)]
        for r in requests:
            if not r.est_bytes:
                lo, hi = r.verts.min(0), r.verts.max(0)
                area = float((hi[0] - lo[0]) * (hi[1] - lo[1]))
                r.est_bytes = estimate_bytes(len(r.verts), len(r.elems), area, r.delta)
        stats = Stats()
        pending: deque = deque()
        results = {r.id: Result(r.id, r.arrival) for r in requests}
        free_slots = list(range(self.slots))
        inflight = {}
        cv = self.budget.cv
        order = sorted(requests, key=lambda r: r.arrival)
        t0 = self.clock()
        nxt = 0

        def finish(req, slot, err=None):
            res = results[req.id]
            if err is not None:
                res.error = err
            res.done = self.clock() - t0
            with cv:
                self.budget.used -= req.est_bytes
                free_slots.append(slot)
                del inflight[req.id]
                cv.notify_all()

        def worker(req, slot):
            try:
                self.execute(req, results[req.id], slot)
            except Exception as e:  # a failed request is reported, the loop goes on
                finish(req, slot, f"{type(e).__name__}: {e}")
                return
            finish(req, slot)

        def run_one(req, slot, cont):
            try:
                cont()
            except Exception as e:
                finish(req, slot, f"{type(e).__name__}: {e}")
                return
            finish(req, slot)

        def batch_worker(reqs, slots):
            try:
                conts = self.execute_batch(reqs, [results[r.id] for r in reqs], slots)
            except Exception as e:  # the whole batch failed: each request reports it
                for r, sl in zip(reqs, slots):
                    finish(r, sl, f"{type(e).__name__}: {e}")
                return
            ths = [threading.Thread(target=run_one, args=a, daemon=True) for a in zip(reqs[1:], slots[1:], conts[1:])]
            for th in ths:
                th.start()
            run_one(reqs[0], slots[0], conts[0])
            for th in ths:
                th.join()

        def batchable(req):
            if self.execute_batch is None:
                return False
            lo, hi = req.verts.min(0), req.verts.max(0)
            area = float((hi[0] - lo[0]) * (hi[1] - lo[1]))
            return estimate_pairs(len(req.elems), area, req.delta) < BATCH_MAX_PAIRS

        with cv:
            while nxt < len(order) or pending or inflight:
                now = self.clock() - t0
                while nxt < len(order) and (not realtime or order[nxt].arrival <= now):
                    pending.append(order[nxt])
                    nxt += 1
                # admit in arrival order while a slot is free and the estimate fits; the small
                # requests admitted in this pass form one batch
                group = []
                while pending and free_slots:
                    req = pending[0]
                    if req.est_bytes > self.budget.budget:
                        pending.popleft()
                        results[req.id].error = (f"admission: needs about {req.est_bytes} device bytes, "
                                                 f"budget {self.budget.budget}")
                        results[req.id].done = self.clock() - t0
                        continue
                    if not self.budget.fits(req.est_bytes) and self.cache is not None:
                        self.budget.used -= self.cache.evict_for(req.est_bytes)
                    if not self.budget.fits(req.est_bytes):
                        break
                    pending.popleft()
                    self.budget.reserve(req.est_bytes)
                    slot = free_slots.pop()
                    results[req.id].admitted = self.clock() - t0
                    if batchable(req):
                        group.append((req, slot))
                        continue
                    th = threading.Thread(target=worker, args=(req, slot), daemon=True)
                    inflight[req.id] = th
                    th.start()
                if len(group) == 1:
                    req, slot = group[0]
                    th = threading.Thread(target=worker, args=(req, slot), daemon=True)
                    inflight[req.id] = th
                    th.start()
                elif group:
                    reqs, slots = [g[0] for g in group], [g[1] for g in group]
                    th = threading.Thread(target=batch_worker, args=(reqs, slots), daemon=True)
                    for r in reqs:
                        inflight[r.id] = th
                    th.start()
                stats.max_inflight = max(stats.max_inflight, len(inflight))
                stats.max_used_bytes = max(stats.max_used_bytes, self.budget.used)
                if nxt < len(order) and realtime:
                    wait = max(0.0, order[nxt].arrival - (self.clock() - t0))
                    cv.wait(timeout=min(wait, 0.05) if wait > 0 else 0.0005)
                elif inflight or pending:
                    cv.wait(timeout=0.05)
        stats.wall = self.clock() - t0
        stats.results = [results[r.id] for r in requests]
        return stats
