"""ctypes wrapper around the FP64 C oracle (test infrastructure only).

Builds ``oracle/_build/liborc.so`` from ``nlfem_oracle.c`` with gcc on first use
(-O2 -ffp-contract=off, OpenMP over outer elements), and exposes:

- :func:`assemble`: full A_h^# over all nodes of the base domain plus the load
  vector (Sec. 2.2 eq. biFormApprox, Sec. 3 kernels), as CSR;
- :func:`pairs`: the interaction graph found by Alg. 2 (or brute force);
- :func:`pair_block`: the local block of one ordered pair (Alg. 1);
- :func:`clip`: E_l cut by a ball approximation (Defs. 2.1 / 2.2);
- :func:`solve_dirichlet`: the column split of eq. inhomogeneousDirichletData
  and a direct sparse solve;
- :func:`l2_error`: L2(Omega) error with the 7-point rule.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

from . import rules as R

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "nlfem_oracle.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liborc.so")

KERNELS = {"constant": 0, "fractional": 1, "peridynamic": 2, "tabulated": 3}
BALLS = {"nocaps": 0, "approxcaps": 1, "infinity": 2}
CLOSE_RULES = {"auto": 0, "duffy": 1, "nozerodiv": 2, "standard": 3}

_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return os.environ.get("NLFEM_ORACLE_LIB") or LIB


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, FP64, no FMA contraction). With NLFEM_ORACLE_LIB
    set, that prebuilt library is used instead (the tests that check the pins against copies of
    the oracle with planted mistakes)."""
    if os.environ.get("NLFEM_ORACLE_LIB"):
        return os.environ["NLFEM_ORACLE_LIB"]
    os.makedirs(BUILD, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        compile_source(SRC, tmp)
        os.replace(tmp, LIB)
    return LIB


def compile_source(src: str, out: str) -> None:
    """gcc of one oracle source file into a shared library (the flags of the oracle's build)."""
    cmd = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", out, src, "-lm"]
    subprocess.check_call(cmd)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int)
            lp = C.POINTER(C.c_longlong)
            cp = C.POINTER(C.c_byte)
            lib.orc_assemble.restype = C.c_void_p
            lib.orc_assemble.argtypes = [C.c_int, dp, C.c_int, ip, cp, C.c_int, C.c_double, C.c_double,
                                         C.c_double, C.c_int, C.c_int, dp, C.c_int, dp, C.c_int, C.c_int,
                                         dp, dp, C.c_int, dp, C.c_int, C.c_int, C.c_int, ip, cp, C.c_int, dp,
                                         C.c_int, dp, cp]
            lib.orc_sys_sizes.argtypes = [C.c_void_p, lp]
            lib.orc_sys_copy.argtypes = [C.c_void_p, lp, ip, dp, dp, ip, cp, cp, lp]
            lib.orc_sys_free.argtypes = [C.c_void_p]
            lib.orc_pairs.restype = C.c_void_p
            lib.orc_pairs.argtypes = [C.c_int, dp, C.c_int, ip, C.c_int, C.c_double, C.c_double, C.c_int,
                                      C.c_int, dp, C.c_int, C.c_int, C.c_int, lp]
            lib.orc_free.argtypes = [C.c_void_p]
            lib.orc_pair_block.restype = C.c_int
            lib.orc_pair_block.argtypes = [C.c_int, dp, C.c_int, ip, C.c_int, C.c_double, C.c_double,
                                           C.c_double, C.c_int, C.c_int, dp, C.c_int, dp, C.c_int,
                                           C.c_int, dp, dp, C.c_int, C.c_int, C.c_int, ip, dp]
            lib.orc_clip.restype = C.c_int
            lib.orc_clip.argtypes = [dp, C.c_double, C.c_double, C.c_double, C.c_int, dp, ip]
            _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t))


@dataclass
class OracleSystem:
    N: int
    ndof: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    F: np.ndarray
    pairs: np.ndarray
    pclass: np.ndarray
    dirichlet: np.ndarray
    counts: dict

    def dense(self) -> np.ndarray:
        A = np.zeros((self.N, self.N))
        for i in range(self.N):
            s, e = self.row_ptr[i], self.row_ptr[i + 1]
            A[i, self.col[s:e]] = self.val[s:e]
        return A

    def scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.row_ptr), shape=(self.N, self.N))


def _kernel_args(kernel, delta, s, kconst, ball, quad_outer, quad_inner, close_rule, duffy_n):
    qo = np.ascontiguousarray(R.rule(quad_outer))
    qi = np.ascontiguousarray(R.rule(quad_inner))
    gx, gw = R.gauss01(duffy_n)
    gx = np.ascontiguousarray(gx)
    gw = np.ascontiguousarray(gw)
    if kernel == "fractional" and not (0.0 < s < 1.0) and close_rule == "auto" and s > 0:
        raise ValueError("fractional kernel needs s in (0, 1)")
    return (KERNELS[kernel], float(delta), float(s), float("nan") if kconst is None else float(kconst),
            BALLS[ball], qo, qi, CLOSE_RULES[close_rule], gx, gw)


def assemble(mesh, kernel: str = "constant", delta: float = 0.1, s: float = -1.0, kconst=None,
             ball: str = "nocaps", quad_outer: int = 7, quad_inner: int = 7, close_rule: str = "auto",
             duffy_n: int = 5, f_nodal=None, pairs_mode: str = "bfs", threads: int = 0,
             elem_subset=None, materials=None, material_scale=None, kernel_table=None,
             node_keep=None) -> OracleSystem:
    """FP64 assembly of A_h^# and F. materials [K] (0..n-1) with the symmetric n x n table
    material_scale make the kernel label dependent: Psi on E_k x E_l times
    material_scale[materials[k], materials[l]] (Sec. 1, interface problems). kernel="tabulated"
    takes the user kernel c g(|z|) from kernel_table (g at r_i = i delta / (n - 1), linear in
    between, held beyond delta; c = kconst, default 1). node_keep [M] (bool): keep only the
    pairs with a flagged node among the vertices of E_k or E_l; the rows of the flagged nodes
    are then those of the full assembly (every pair writing into them is kept)."""
    lib = _load()
    ndof = 2 if kernel == "peridynamic" else 1
    (kid, delta, s, kc, bid, qo, qi, cid, gx, gw) = _kernel_args(
        kernel, delta, s, kconst, ball, quad_outer, quad_inner, close_rule, duffy_n)
    X = np.ascontiguousarray(mesh.verts, dtype=np.float64)
    T = np.ascontiguousarray(mesh.elems, dtype=np.int32)
    lab = np.ascontiguousarray(mesh.elem_label, dtype=np.int8)
    f = None
    if f_nodal is not None:
        f = np.ascontiguousarray(np.asarray(f_nodal, dtype=np.float64).reshape(mesh.M * ndof))
    tab = None
    if kernel == "tabulated":
        tab = np.ascontiguousarray(kernel_table, dtype=np.float64).reshape(-1)
        assert 2 <= len(tab) <= 1024
    mat = msc = None
    nmat = 0
    if materials is not None:
        mat = np.ascontiguousarray(materials, dtype=np.int8)
        msc = np.ascontiguousarray(material_scale, dtype=np.float64)
        nmat = int(msc.shape[0])
        assert msc.shape == (nmat, nmat) and mat.shape == (mesh.K,) and 0 <= mat.min() and mat.max() < nmat
    keep = None
    if node_keep is not None:
        keep = np.ascontiguousarray(np.asarray(node_keep).reshape(-1).astype(np.int8))
        assert keep.shape == (mesh.M,)
    sub = None
    nsub = 0
    if elem_subset is not None:
        sub = np.ascontiguousarray(elem_subset, dtype=np.int32)
        nsub = len(sub)
    h = lib.orc_assemble(mesh.M, _p(X, C.c_double), mesh.K, _p(T, C.c_int), _p(lab, C.c_byte), kid, delta, s,
                         kc, bid, len(qo), _p(qo, C.c_double), len(qi), _p(qi, C.c_double), cid, len(gx),
                         _p(gx, C.c_double), _p(gw, C.c_double), ndof,
                         _p(f, C.c_double) if f is not None else None,
                         0 if pairs_mode == "bfs" else 1, int(threads), nsub,
                         _p(sub, C.c_int) if sub is not None else None,
                         _p(mat, C.c_byte) if mat is not None else None, nmat,
                         _p(msc, C.c_double) if msc is not None else None,
                         len(tab) if tab is not None else 0, _p(tab, C.c_double) if tab is not None else None,
                         _p(keep, C.c_byte) if keep is not None else None)
    sz = np.zeros(3, dtype=np.int64)
    lib.orc_sys_sizes(h, _p(sz, C.c_longlong))
    N, nnz, npairs = (int(v) for v in sz)
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    col = np.zeros(max(nnz, 1), dtype=np.int32)
    val = np.zeros(max(nnz, 1), dtype=np.float64)
    F = np.zeros(max(N, 1), dtype=np.float64)
    pr = np.zeros((max(npairs, 1), 2), dtype=np.int32)
    pc = np.zeros(max(npairs, 1), dtype=np.int8)
    dr = np.zeros(max(mesh.M, 1), dtype=np.int8)
    cnt = np.zeros(10, dtype=np.int64)
    lib.orc_sys_copy(h, _p(row_ptr, C.c_longlong), _p(col, C.c_int), _p(val, C.c_double), _p(F, C.c_double),
                     _p(pr, C.c_int), _p(pc, C.c_byte), _p(dr, C.c_byte), _p(cnt, C.c_longlong))
    lib.orc_sys_free(h)
    names = ["evals", "cut_points", "full_points", "subtris", "duffy_points", "pairs", "pairs_identical",
             "pairs_edge", "pairs_vertex", "pairs_separated"]
    return OracleSystem(N, ndof, row_ptr, col[:nnz], val[:nnz], F[:N], pr[:npairs], pc[:npairs],
                        dr[:mesh.M].astype(bool), dict(zip(names, (int(c) for c in cnt))))


def pairs(mesh, kernel="constant", delta=0.1, s=-1.0, ball="nocaps", quad_outer=7, close_rule="auto",
          mode="bfs", threads=0) -> np.ndarray:
    """Ordered interacting pairs (k, l), grouped by k in traversal order."""
    lib = _load()
    qo = np.ascontiguousarray(R.rule(quad_outer))
    X = np.ascontiguousarray(mesh.verts, dtype=np.float64)
    T = np.ascontiguousarray(mesh.elems, dtype=np.int32)
    n = C.c_longlong(0)
    ptr = lib.orc_pairs(mesh.M, _p(X, C.c_double), mesh.K, _p(T, C.c_int), KERNELS[kernel], float(delta),
                        float(s), BALLS[ball], len(qo), _p(qo, C.c_double), CLOSE_RULES[close_rule],
                        0 if mode == "bfs" else 1, int(threads), C.byref(n))
    arr = np.ctypeslib.as_array(C.cast(ptr, C.POINTER(C.c_int)), shape=(max(n.value, 1) * 2,)).copy()
    lib.orc_free(ptr)
    return arr[:2 * n.value].reshape(-1, 2)


def pair_block(mesh, k: int, l: int, kernel="constant", delta=0.1, s=-1.0, kconst=None, ball="nocaps",
               quad_outer=7, quad_inner=7, close_rule="auto", duffy_n=5):
    """Local block of the ordered pair (E_k, E_l) on its union vertices.

    Returns (nodes [U], block [U*ndof, U*ndof], interacts)."""
    lib = _load()
    ndof = 2 if kernel == "peridynamic" else 1
    (kid, delta, s, kc, bid, qo, qi, cid, gx, gw) = _kernel_args(
        kernel, delta, s, kconst, ball, quad_outer, quad_inner, close_rule, duffy_n)
    X = np.ascontiguousarray(mesh.verts, dtype=np.float64)
    T = np.ascontiguousarray(mesh.elems, dtype=np.int32)
    node = np.zeros(6, dtype=np.int32)
    blk = np.zeros(144, dtype=np.float64)
    r = lib.orc_pair_block(mesh.M, _p(X, C.c_double), mesh.K, _p(T, C.c_int), kid, delta, s, kc, bid,
                           len(qo), _p(qo, C.c_double), len(qi), _p(qi, C.c_double), cid, len(gx),
                           _p(gx, C.c_double), _p(gw, C.c_double), ndof, int(k), int(l),
                           _p(node, C.c_int), _p(blk, C.c_double))
    U = abs(r)
    n = U * ndof
    return node[:U].copy(), blk[:n * n].reshape(n, n).copy(), r > 0


def clip(V, c, delta: float, caps: bool = False, ball=None):
    """E_l (3x2 vertices) cut by the ball around c: nocaps / approxcaps (caps) or, with
    ball="infinity", the infinity norm ball. Returns (points [n,2], full)."""
    lib = _load()
    V = np.ascontiguousarray(np.asarray(V, dtype=np.float64).reshape(6))
    out = np.zeros(32, dtype=np.float64)
    full = C.c_int(0)
    b = BALLS[ball] if ball is not None else int(bool(caps))
    n = lib.orc_clip(_p(V, C.c_double), float(c[0]), float(c[1]), float(delta), b,
                     _p(out, C.c_double), C.byref(full))
    return out[:2 * n].reshape(n, 2).copy(), bool(full.value)


def solve_dirichlet(system: OracleSystem, g_nodal) -> np.ndarray:
    """Solve A_FF u_F = F_F - A_FD g (eq. inhomogeneousDirichletData) by a direct sparse solve."""
    import scipy.sparse.linalg as spla
    ndof = system.ndof
    dmask = np.repeat(system.dirichlet, ndof)
    free = np.flatnonzero(~dmask)
    dof_d = np.flatnonzero(dmask)
    g = np.asarray(g_nodal, dtype=np.float64).reshape(-1)
    A = system.scipy().tocsc()
    b = system.F[free] - A[free][:, dof_d] @ g[dof_d]
    u = g.copy()
    if len(free):
        u[free] = spla.spsolve(A[free][:, free].tocsc(), b)
    return u


def null_space(verts, ndof: int) -> np.ndarray:
    """Columns spanning the null space of the full (Neumann-type) matrix: the constants for a
    scalar kernel, the rigid motions (two translations, the rotation (-y, x)) for the vector
    peridynamic kernel (Sec. 2, symmetrised form, Remark on asymmetry due to quadrature)."""
    X = np.asarray(verts, dtype=np.float64)
    M = X.shape[0]
    if ndof == 1:
        return np.ones((M, 1))
    Z = np.zeros((M, 2, 3))
    Z[:, 0, 0] = 1.0
    Z[:, 1, 1] = 1.0
    Z[:, 0, 2] = -X[:, 1]
    Z[:, 1, 2] = X[:, 0]
    return Z.reshape(2 * M, 3)


def solve_neumann(system: OracleSystem, verts) -> np.ndarray:
    """Pure Neumann-type problem on the full matrix: the minimum-norm u with A u = F - P F,
    P the orthogonal projector onto the null space N of A. Solved as the bordered system
    [[A, Z], [Z^T, 0]] [u; lam] = [F; 0] with Z spanning N (dense, small meshes only)."""
    Z = null_space(verts, system.ndof)
    A = system.dense()
    n, m = Z.shape
    K = np.zeros((n + m, n + m))
    K[:n, :n] = A
    K[:n, n:] = Z
    K[n:, :n] = Z.T
    rhs = np.concatenate([system.F, np.zeros(m)])
    return np.linalg.solve(K, rhs)[:n]


def l2_error(mesh, u_h, u_exact, ndof: int = 1) -> float:
    """||u_h - u||_{L2(Omega)} with the 7-point rule on the Omega elements."""
    q = R.rule7()
    E = mesh.elems[mesh.elem_label == 1]
    P = mesh.verts[E]                                   # [K, 3, 2]
    det = np.abs((P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1]) -
                 (P[:, 1, 1] - P[:, 0, 1]) * (P[:, 2, 0] - P[:, 0, 0]))
    uh = np.asarray(u_h).reshape(mesh.M, ndof)
    err = 0.0
    for l0, l1, l2, w in q:
        x = l0 * P[:, 0] + l1 * P[:, 1] + l2 * P[:, 2]
        uq = l0 * uh[E[:, 0]] + l1 * uh[E[:, 1]] + l2 * uh[E[:, 2]]
        ue = np.asarray(u_exact(x[:, 0], x[:, 1]), dtype=np.float64)
        ue = ue.T.reshape(-1, ndof) if ue.ndim > 1 else ue.reshape(-1, 1)
        err += np.sum(w * det * np.sum((uq.reshape(-1, ndof) - ue) ** 2, axis=1))
    return math.sqrt(err)
