"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only builds meshes and nodal data. It holds none of the assembly
arithmetic, so both the CUDA path and the CPU oracle may take their inputs from
it without sharing any part of the method.

Meshes follow the paper's experiments (Sec. 3): a square base domain
[lo, hi]^2 split into right triangles, or a jittered Delaunay triangulation of
the same grid. Elements are labelled Omega when their centroid lies in the open
box ``omega`` and Omega_D otherwise (Sec. 2.2, the assumption that Omega and
Omega_D are exactly covered by elements).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Mesh:
    verts: np.ndarray          # float64 [M, 2]
    elems: np.ndarray          # int32 [K, 3], counter-clockwise
    elem_label: np.ndarray     # int8 [K]; 1 = Omega, 0 = Omega_D
    h: float                   # grid spacing the mesh was built from
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def M(self) -> int:
        return int(self.verts.shape[0])

    @property
    def K(self) -> int:
        return int(self.elems.shape[0])

    def dirichlet_nodes(self) -> np.ndarray:
        """Bool [M]: node is a vertex of some Omega_D element (Sec. 2.2)."""
        d = np.zeros(self.M, dtype=bool)
        d[self.elems[self.elem_label == 0].ravel()] = True
        return d


def _grid_coords(lo: float, hi: float, n: int) -> np.ndarray:
    # i/n interpolation keeps both ends exact; interior grid lines that should
    # sit on 0 or 1 are snapped so that Omega's boundary is a set of mesh edges.
    t = np.arange(n + 1, dtype=np.float64) / n
    x = lo + (hi - lo) * t
    x[0], x[-1] = lo, hi
    for v in (0.0, 1.0, 0.5):
        close = np.abs(x - v) < 1e-12 * max(1.0, abs(hi - lo))
        x[close] = v
    return x


def _labels(verts, elems, omega):
    c = verts[elems].mean(axis=1)
    (a0, b0), (a1, b1) = omega
    inside = (c[:, 0] > a0) & (c[:, 0] < b0) & (c[:, 1] > a1) & (c[:, 1] < b1)
    return inside.astype(np.int8)


def _ccw(verts, elems):
    p = verts[elems]
    det = (p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1]) - \
          (p[:, 1, 1] - p[:, 0, 1]) * (p[:, 2, 0] - p[:, 0, 0])
    e = elems.copy()
    neg = det < 0
    e[neg, 1], e[neg, 2] = elems[neg, 2], elems[neg, 1]
    return e


def structured(lo: float, hi: float, n: int, omega=((0.0, 1.0), (0.0, 1.0)),
               name: str = "") -> Mesh:
    """(n+1)^2 grid nodes on [lo,hi]^2, each cell split by its "/" diagonal."""
    x = _grid_coords(lo, hi, n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    verts = np.stack([X.ravel(), Y.ravel()], axis=1)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    v00 = (j * (n + 1) + i).ravel()
    v10 = v00 + 1
    v01 = v00 + (n + 1)
    v11 = v01 + 1
    lower = np.stack([v00, v10, v11], axis=1)
    upper = np.stack([v00, v11, v01], axis=1)
    elems = np.empty((2 * n * n, 3), dtype=np.int32)
    elems[0::2] = lower
    elems[1::2] = upper
    h = (hi - lo) / n
    return Mesh(verts, elems, _labels(verts, elems, omega), h, name or f"structured{n}",
                {"lo": lo, "hi": hi, "n": n, "omega": omega})


def jittered_delaunay(lo: float, hi: float, n: int, jitter: float, seed: int,
                      omega=((0.0, 1.0), (0.0, 1.0)), name: str = "") -> Mesh:
    """Grid nodes moved uniformly by up to ``jitter * h`` per coordinate, then
    Delaunay-triangulated. Nodes on the base-domain boundary and on the lines
    x, y in {0, 1} keep the coordinate across that line fixed, so the
    Omega / Omega_D interface stays a set of mesh edges."""
    from scipy.spatial import Delaunay

    x = _grid_coords(lo, hi, n)
    h = (hi - lo) / n
    X, Y = np.meshgrid(x, x, indexing="xy")
    rng = np.random.Generator(np.random.PCG64(seed))
    jx = rng.uniform(-jitter * h, jitter * h, size=X.shape)
    jy = rng.uniform(-jitter * h, jitter * h, size=Y.shape)
    fixed = np.array([lo, hi, 0.0, 1.0])
    on_x = np.isin(X, fixed)
    on_y = np.isin(Y, fixed)
    jx[on_x] = 0.0
    jy[on_y] = 0.0
    verts = np.stack([(X + jx).ravel(), (Y + jy).ravel()], axis=1)
    tri = Delaunay(verts)
    elems = _ccw(verts, tri.simplices.astype(np.int32))
    # Drop slivers Delaunay can leave on exactly collinear boundary nodes.
    p = verts[elems]
    det = (p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1]) - \
          (p[:, 1, 1] - p[:, 0, 1]) * (p[:, 2, 0] - p[:, 0, 0])
    elems = elems[det > 1e-12 * h * h]
    return Mesh(verts, np.ascontiguousarray(elems, dtype=np.int32),
                _labels(verts, elems, omega), h, name or f"jittered{n}",
                {"lo": lo, "hi": hi, "n": n, "seed": seed, "jitter": jitter, "omega": omega})


# --- workloads shaped like the paper's (Sec. 3) and the benchmark configurations ----------

MESH_SEED_BASE = 2207039210


def cfg1_mesh() -> Mesh:
    """[-0.1, 1.1]^2, h = 0.05, structured: 1152 triangles."""
    return structured(-0.1, 1.1, 24, name="cfg1_structured_h0.05")


def cfg2_mesh(n: int = 120) -> Mesh:
    """[-0.1, 1.1]^2 jittered Delaunay, h = 0.01 (n = 120), 3% jitter."""
    return jittered_delaunay(-0.1, 1.1, n, 0.03, MESH_SEED_BASE + 2, name=f"cfg2_jittered{n}")


def cfg3_mesh(n: int = 208) -> Mesh:
    """[-0.02, 1.02]^2, h = 0.005 (n = 208), structured: 86,528 triangles."""
    return structured(-0.02, 1.02, n, name=f"cfg3_structured{n}")


def cfg5_mesh(n: int = 510) -> Mesh:
    """[-0.01, 1.01]^2, h = 0.002 (n = 510), structured: 520,200 triangles."""
    return structured(-0.01, 1.01, n, name=f"cfg5_structured{n}")


def cfg720k_mesh(n: int = 600) -> Mesh:
    """[-0.01, 1.01]^2 with 600 x 600 cells: exactly 720,000 triangles."""
    return structured(-0.01, 1.01, n, name=f"structured{n}_720k")


def paper_square(delta: float, a: float) -> Mesh:
    """Sec. 3 domain: Omega = (0, 0.5)^2 inside [-delta, 0.5 + delta]^2 with grid spacing a."""
    n = int(round((0.5 + 2 * delta) / a))
    return structured(-delta, 0.5 + delta, n, omega=((0.0, 0.5), (0.0, 0.5)),
                      name=f"paper_square_d{delta}_a{a}")


def discontinuous(mesh: Mesh) -> Mesh:
    """The same triangles with their own copies of the vertices (the P1-DG ansatz of Sec. 2.2:
    J = 3K nodes, node 3k + a = vertex a of element k as given in mesh.elems)."""
    K = mesh.K
    verts = np.ascontiguousarray(mesh.verts[mesh.elems].reshape(3 * K, 2))
    elems = np.arange(3 * K, dtype=np.int32).reshape(K, 3)
    return Mesh(verts, elems, mesh.elem_label.copy(), mesh.h, name=mesh.name + "_dg", meta=dict(mesh.meta))


def nodal(mesh: Mesh, fn) -> np.ndarray:
    """Evaluate fn(x, y) at the nodes; returns float64 [M] or [M, n]."""
    v = fn(mesh.verts[:, 0], mesh.verts[:, 1])
    return np.ascontiguousarray(np.asarray(v, dtype=np.float64).T if np.ndim(v) > 1 else v)


def serving_requests(n_requests: int = 512, rate: float = 200.0, seed: int = 2207039214,
                     kmin: int = 500, kmax: int = 50000):
    """Poisson arrival stream of (mesh, delta, kernel) requests.

    Mesh sizes are log-uniform in [kmin, kmax] triangles; delta is drawn from
    {0.05, 0.1, 0.2}; the kernel is constant or fractional with s in {0.25, 0.75}.
    Returns a list of dicts with arrival time (s) and request parameters; meshes
    are built lazily by :func:`request_mesh`.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, size=n_requests)
    t = np.cumsum(gaps) - gaps[0]
    logk = rng.uniform(math.log(kmin), math.log(kmax), size=n_requests)
    deltas = rng.choice([0.05, 0.1, 0.2], size=n_requests)
    kinds = rng.integers(0, 3, size=n_requests)
    mseeds = rng.integers(0, 2**31 - 1, size=n_requests)
    out = []
    for r in range(n_requests):
        kernel, s = [("constant", -1.0), ("fractional", 0.25), ("fractional", 0.75)][int(kinds[r])]
        out.append({"id": r, "arrival": float(t[r]), "K_target": int(math.exp(logk[r])),
                    "delta": float(deltas[r]), "kernel": kernel, "s": s,
                    "mesh_seed": int(mseeds[r])})
    return out


def request_mesh(req) -> Mesh:
    """Jittered Delaunay mesh of [-delta, 1 + delta]^2 with about K_target triangles."""
    d = req["delta"]
    side = 1.0 + 2 * d
    n = max(4, int(round(math.sqrt(req["K_target"] / 2.0))))
    h = side / n
    # Keep 0 and 1 on grid lines: choose n so that delta / h is an integer.
    m = max(1, int(round(d / h)))
    h = d / m
    n = int(round(side / h))
    return jittered_delaunay(-d, 1.0 + d, n, 0.03, req["mesh_seed"], name=f"req{req['id']}")
