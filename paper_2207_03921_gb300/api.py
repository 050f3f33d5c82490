"""Python front end: meshes, assembly and solve as torch tensors on the GPU.

Thin wrappers over the C ABI in :mod:`binding`; torch provides device memory and
streams. Matrices come back as CSR tensors (row_ptr int64, col int32, val float64)
over all dofs of the base domain; :meth:`System.csr` copies them out of the library,
:meth:`System.csr_views` returns zero-copy views valid while the System lives.
"""
from __future__ import annotations

import numpy as np

from . import binding as B


class _DevView:
    """__cuda_array_interface__ over a library-owned device buffer (keeps the owner alive)."""

    def __init__(self, ptr, n, typestr, owner):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr, "data": (int(ptr or 0), False),
                                         "version": 3, "strides": None}
        self._owner = owner


def _torch():
    import torch
    return torch


def _as_dev(x, dtype):
    """Host/device array -> contiguous torch CUDA tensor of dtype."""
    torch = _torch()
    if isinstance(x, torch.Tensor):
        return x.to(device="cuda", dtype=dtype).contiguous()
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype).cuda()


class Mesh:
    """A triangle mesh of the base domain uploaded to the GPU (nlfem_mesh_create)."""

    def __init__(self, verts, elems, elem_label=None, ndof_per_node=1, stream=None, dg=False):
        """dg=True: discontinuous P1 ansatz, node 3k + a = vertex a of element k
        (nlfem_mesh_create_dg); the mesh then has 3K nodes."""
        torch = _torch()
        self.verts = _as_dev(verts, torch.float64)
        self.elems = _as_dev(elems, torch.int32)
        self.elem_label = None if elem_label is None else _as_dev(elem_label, torch.int8)
        self.K = int(self.elems.shape[0])
        self.M = 3 * self.K if dg else int(self.verts.shape[0])
        self.ndof = int(ndof_per_node)
        self.dg = bool(dg)
        self.handle = B.nlfem_mesh_create(self.verts, self.elems, self.elem_label, self.ndof, stream, dg=dg)

    @classmethod
    def from_synth(cls, m, ndof_per_node=1, stream=None, dg=False):
        return cls(m.verts, m.elems, m.elem_label, ndof_per_node, stream, dg=dg)

    def pairs(self):
        """(k, l) int32 tensors of the cached interaction graph (copies)."""
        torch = _torch()
        kp, lp, n = B.nlfem_mesh_pairs(self.handle)
        k = torch.as_tensor(_DevView(kp, n, "<i4", self), device="cuda").clone()
        l = torch.as_tensor(_DevView(lp, n, "<i4", self), device="cuda").clone()
        return k, l

    def device_bytes(self) -> int:
        return B.nlfem_mesh_device_bytes(self.handle)

    def set_materials(self, material, stream=None) -> None:
        """Material labels [K] (0..15) of a label-dependent kernel (nlfem_mesh_set_materials)."""
        torch = _torch()
        self.material = None if material is None else _as_dev(material, torch.int8)
        B.nlfem_mesh_set_materials(self.handle, self.material, stream)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            B.nlfem_mesh_destroy(h)
            self.handle = None


class System:
    """An assembled stiffness matrix and load vector (nlfem_assemble)."""

    def __init__(self, mesh: Mesh, handle, owner=None):
        self.mesh = mesh
        self.handle = handle
        self._owner = owner  # a BatchPlan that owns the handle, or None
        rp, col, val, n, nnz = B.nlfem_system_csr(handle)
        self.N, self.nnz = n, nnz
        self._ptrs = (rp, col, val)

    def csr_views(self):
        torch = _torch()
        rp, col, val = self._ptrs
        return (torch.as_tensor(_DevView(rp, self.N + 1, "<i8", self), device="cuda"),
                torch.as_tensor(_DevView(col, self.nnz, "<i4", self), device="cuda"),
                torch.as_tensor(_DevView(val, self.nnz, "<f8", self), device="cuda"))

    def csr(self):
        return tuple(t.clone() for t in self.csr_views())

    def rhs(self):
        torch = _torch()
        return torch.as_tensor(_DevView(B.nlfem_system_rhs(self.handle), self.N, "<f8", self), device="cuda").clone()

    def dirichlet(self):
        torch = _torch()
        return torch.as_tensor(_DevView(B.nlfem_system_dirichlet(self.handle), self.mesh.M, "|i1", self),
                               device="cuda").clone().bool()

    def info(self) -> dict:
        return B.nlfem_system_info(self.handle)

    def census(self) -> dict:
        return B.nlfem_system_census(self.handle)

    def to_torch_sparse(self):
        torch = _torch()
        rp, col, val = self.csr()
        return torch.sparse_csr_tensor(rp, col.long(), val, size=(self.N, self.N))

    def solve(self, g_nodal=None, tol_rel=1e-10, max_iter=20000, stream=None):
        """u with A_FF u_F = F_F - A_FD g and u = g at Dirichlet dofs (nlfem_solve)."""
        torch = _torch()
        u = torch.empty(self.N, dtype=torch.float64, device="cuda")
        g = None if g_nodal is None else _as_dev(g_nodal, torch.float64).reshape(-1)
        info = B.nlfem_solve(self.handle, g, tol_rel, max_iter, u, stream)
        return u, info

    def solve_neumann(self, tol_rel=1e-10, max_iter=20000, stream=None):
        """u orthogonal to the null space N of A with P A u = P F (nlfem_solve_neumann)."""
        torch = _torch()
        u = torch.empty(self.N, dtype=torch.float64, device="cuda")
        info = B.nlfem_solve_neumann(self.handle, tol_rel, max_iter, u, stream)
        return u, info

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and getattr(self, "_owner", None) is None:
            B.nlfem_system_destroy(h)
        self.handle = None


def assemble(mesh: Mesh, kernel="constant", delta=0.1, s=0.5, kconst=None, ball="nocaps", quad_outer=7,
             quad_inner=7, duffy_gauss=5, close_rule="auto", precision="fp64", f_nodal=None,
             mem_budget_bytes=0, stream=None, material_scale=None, kernel_table=None,
             singular_precision="fp64", geometry_precision="fp32") -> System:
    """Assemble A_h^# and F on the GPU (nlfem_assemble). material_scale: symmetric table of a
    label-dependent kernel over the labels of Mesh.set_materials; kernel_table: the values of
    g for kernel="tabulated"; singular_precision ("fp64" | "fp32") and geometry_precision
    ("fp32" | "fp64"): arithmetic of the singular rule and of the cut geometry when
    precision="fp32_bulk"."""
    torch = _torch()
    p = B.make_params(kernel, delta, s, kconst, ball, quad_outer, quad_inner, duffy_gauss, close_rule,
                      precision, mem_budget_bytes, material_scale, kernel_table, singular_precision,
                      geometry_precision)
    f = None if f_nodal is None else _as_dev(f_nodal, torch.float64).reshape(-1)
    h = B.nlfem_assemble(mesh.handle, p, f, stream)
    return System(mesh, h)


def assemble_batch(meshes, params, f_nodal=None, stream=None) -> list:
    """Assemble several systems with fused bulk launches (nlfem_batch_assemble).

    meshes: distinct Mesh objects; params: one dict of assemble() keyword arguments per mesh
    (kernel, delta, s, ball, quad_outer, quad_inner, precision, ...); f_nodal: None or a list
    of nodal load arrays (or None). Every System equals the one assemble() gives.
    """
    torch = _torch()
    ps = _params_list(params)
    fs = None
    if f_nodal is not None:
        fs = [None if f is None else _as_dev(f, torch.float64).reshape(-1) for f in f_nodal]
    hs = B.nlfem_batch_assemble([m.handle for m in meshes], ps, fs, stream)
    return [System(m, h) for m, h in zip(meshes, hs)]


def _params_list(params):
    ps = []
    for p in params:
        q = dict(kernel="constant", delta=0.1, s=0.5, kconst=None, ball="nocaps", quad_outer=7, quad_inner=7,
                 duffy_gauss=5, close_rule="auto", precision="fp64", mem_budget_bytes=0, material_scale=None,
                 kernel_table=None, singular_precision="fp64", geometry_precision="fp32")
        q.update(p)
        ps.append(B.make_params(q["kernel"], q["delta"], q["s"], q["kconst"], q["ball"], q["quad_outer"],
                                q["quad_inner"], q["duffy_gauss"], q["close_rule"], q["precision"],
                                q["mem_budget_bytes"], q["material_scale"], q["kernel_table"],
                                q["singular_precision"], q["geometry_precision"]))
    return ps


class BatchPlan:
    """Systems of several meshes kept on the GPU and re-assembled by one CUDA graph replay
    (nlfem_batch_create / nlfem_batch_run). FP32 bulk only."""

    def __init__(self, meshes, params, f_nodal=None, stream=None):
        torch = _torch()
        self.meshes = list(meshes)
        fs = None
        if f_nodal is not None:
            fs = [None if f is None else _as_dev(f, torch.float64).reshape(-1) for f in f_nodal]
        self.handle = B.nlfem_batch_create([m.handle for m in self.meshes], _params_list(params), fs, stream)
        self.systems = [System(m, B.nlfem_batch_system(self.handle, i), owner=self)
                        for i, m in enumerate(self.meshes)]

    def run(self, stream=None) -> float:
        """Re-assemble every system in place; returns the device time of the replay in ms."""
        return B.nlfem_batch_run(self.handle, stream)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            for s in getattr(self, "systems", []):
                s.handle = None
            B.nlfem_batch_destroy(h)
            self.handle = None


def autotune(mesh: Mesh, stream=None, **params) -> tuple:
    """Pick the FP32-bulk launch shape for this kernel class on mesh (nlfem_autotune); returns
    (blocks per SM of the whole-pair kernel, of the cut-pair kernel, its outer points per chunk)."""
    q = dict(precision="fp32_bulk")
    q.update(params)
    return B.nlfem_autotune(mesh.handle, _params_list([q])[0], stream)


def tune_set(shape, **params) -> None:
    """Set the FP32-bulk launch shape (whole bps, cut bps, outer points per chunk) of the kernel
    class of params without timing (nlfem_tune_set)."""
    q = dict(precision="fp32_bulk")
    q.update(params)
    B.nlfem_tune_set(_params_list([q])[0], shape)

