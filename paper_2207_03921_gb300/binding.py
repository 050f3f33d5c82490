"""ctypes binding of libnlfem.so (include/nlfem.h).

The functions below carry the C names and only marshal arguments: torch tensors or
numpy arrays in, device pointers and CUDA stream handles out. Every computation runs
in the CUDA library; if the shared library cannot be loaded, import fails loudly.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import re
import threading

import importlib

_build = importlib.import_module(__package__ + ".build")

_lib = None
_lock = threading.Lock()

NLFEM_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "BAD_MESH", -3: "OOM", -4: "BUDGET", -5: "CUDA", -6: "NOT_CONVERGED",
          -7: "TIMEOUT", -8: "UNSUPPORTED"}
KERNELS = {"constant": 0, "fractional": 1, "peridynamic": 2, "tabulated": 3}
BALLS = {"nocaps": 0, "approxcaps": 1, "infinity": 2}
CLOSE_RULES = {"auto": 0, "duffy": 1, "nozerodiv": 2, "standard": 3}
PRECISIONS = {"fp64": 0, "fp32_bulk": 1}
SINGULAR_PRECISIONS = {"fp64": 0, "fp32": 1}
GEOMETRY_PRECISIONS = {"fp32": 0, "fp64": 1}


class NlfemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"nlfem error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


class nlfem_params(C.Structure):
    _fields_ = [("kernel", C.c_int), ("delta", C.c_double), ("s", C.c_double), ("kconst", C.c_double),
                ("ball", C.c_int), ("quad_outer", C.c_int), ("quad_inner", C.c_int), ("duffy_gauss", C.c_int),
                ("close_rule", C.c_int), ("precision", C.c_int), ("mem_budget_bytes", C.c_int64),
                ("n_materials", C.c_int), ("material_scale", C.c_void_p),
                ("table_size", C.c_int), ("kernel_table", C.c_void_p),
                ("singular_precision", C.c_int), ("geometry_precision", C.c_int)]


class nlfem_assembly_info(C.Structure):
    _fields_ = [("npairs", C.c_int64), ("pairs_identical", C.c_int64), ("pairs_edge", C.c_int64),
                ("pairs_vertex", C.c_int64), ("pairs_separated", C.c_int64), ("nnz", C.c_int64),
                ("device_bytes", C.c_int64), ("ms_pairs", C.c_double), ("ms_pattern", C.c_double),
                ("ms_quadrature", C.c_double), ("ms_reduce", C.c_double), ("cached", C.c_int),
                ("ms_whole", C.c_double), ("ms_cut", C.c_double), ("ms_close", C.c_double),
                ("pairs_whole", C.c_int64), ("n_upper", C.c_int64), ("n_contrib", C.c_int64),
                ("ms_sums", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class nlfem_solve_info(C.Structure):
    _fields_ = [("iterations", C.c_int), ("refinements", C.c_int), ("rel_residual", C.c_double)]


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libnlfem.so (building it first if it is missing and nvcc is available)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_build.LIB):
            if not build_if_missing:
                raise RuntimeError(f"libnlfem.so not built at {_build.LIB}")
            _build.build()
        lib = C.CDLL(_build.LIB)
        vp, i64, ip, dp = C.c_void_p, C.c_int64, C.c_int, C.c_double
        lib.nlfem_last_error.restype = C.c_char_p
        lib.nlfem_version.restype = C.c_char_p
        lib.nlfem_mesh_create.argtypes = [vp, i64, vp, i64, vp, ip, vp, C.POINTER(vp)]
        lib.nlfem_mesh_create_dg.argtypes = [vp, i64, vp, i64, vp, ip, vp, C.POINTER(vp)]
        lib.nlfem_mesh_destroy.argtypes = [vp]
        lib.nlfem_mesh_destroy.restype = None
        lib.nlfem_params_default.argtypes = [C.POINTER(nlfem_params), ip]
        lib.nlfem_params_default.restype = None
        lib.nlfem_assemble.argtypes = [vp, C.POINTER(nlfem_params), vp, vp, C.POINTER(vp)]
        lib.nlfem_system_csr.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(i64),
                                         C.POINTER(i64)]
        lib.nlfem_system_rhs.argtypes = [vp, C.POINTER(vp)]
        lib.nlfem_system_dirichlet.argtypes = [vp, C.POINTER(vp)]
        lib.nlfem_system_info.argtypes = [vp, C.POINTER(nlfem_assembly_info)]
        lib.nlfem_mesh_pairs.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(i64)]
        lib.nlfem_solve.argtypes = [vp, vp, dp, ip, vp, C.POINTER(nlfem_solve_info), vp]
        lib.nlfem_solve_neumann.argtypes = [vp, dp, ip, vp, C.POINTER(nlfem_solve_info), vp]
        lib.nlfem_mesh_set_materials.argtypes = [vp, vp, vp]
        lib.nlfem_system_census.argtypes = [vp, C.POINTER(C.c_int64), vp]
        lib.nlfem_system_destroy.argtypes = [vp]
        lib.nlfem_system_destroy.restype = None
        lib.nlfem_mesh_device_bytes.argtypes = [vp]
        lib.nlfem_mesh_device_bytes.restype = i64
        lib.nlfem_trim_memory.argtypes = [vp]
        lib.nlfem_batch_assemble.argtypes = [C.POINTER(vp), C.POINTER(nlfem_params), C.POINTER(vp), ip, vp,
                                             C.POINTER(vp)]
        lib.nlfem_batch_create.argtypes = [C.POINTER(vp), C.POINTER(nlfem_params), C.POINTER(vp), ip, vp,
                                           C.POINTER(vp)]
        lib.nlfem_batch_run.argtypes = [vp, vp, C.POINTER(C.c_double)]
        lib.nlfem_batch_system.argtypes = [vp, ip, C.POINTER(vp)]
        lib.nlfem_batch_destroy.argtypes = [vp]
        lib.nlfem_batch_destroy.restype = None
        lib.nlfem_autotune.argtypes = [vp, C.POINTER(nlfem_params), vp, C.POINTER(C.c_int32)]
        lib.nlfem_tune_set.argtypes = [C.POINTER(nlfem_params), C.POINTER(C.c_int32)]
        lib.nlfem_pairs_noalloc.argtypes = [vp, i64, vp, i64, dp, ip, ip, vp, vp, i64, C.POINTER(i64), vp]
        _lib = lib
    return _lib


def header_symbols() -> list[str]:
    """Names of the functions declared in include/nlfem.h."""
    hdr = os.path.join(os.path.dirname(_build.HERE), "include", "nlfem.h")
    txt = open(hdr).read()
    return sorted(set(re.findall(r"\b(nlfem_[a-z_]+)\s*\(", txt)))


def _check(code):
    if code != NLFEM_OK:
        raise NlfemError(code, load().nlfem_last_error().decode())


def _ptr(x):
    """Device or host pointer of a torch tensor / numpy array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


# ---- the C ABI, one Python function per C function ----------------------------------------

def nlfem_mesh_create(verts, elems, elem_label=None, ndof_per_node=1, stream=None, dg=False):
    lib = load()
    h = C.c_void_p()
    M = int(verts.shape[0])
    K = int(elems.shape[0])
    fn = lib.nlfem_mesh_create_dg if dg else lib.nlfem_mesh_create
    _check(fn(_ptr(verts), M, _ptr(elems), K, _ptr(elem_label), int(ndof_per_node), _stream(stream), C.byref(h)))
    return h


def nlfem_mesh_destroy(mesh):
    load().nlfem_mesh_destroy(mesh)


def nlfem_params_default(kernel: int) -> nlfem_params:
    p = nlfem_params()
    load().nlfem_params_default(C.byref(p), int(kernel))
    return p


def nlfem_assemble(mesh, params: nlfem_params, f_nodal=None, stream=None):
    h = C.c_void_p()
    _check(load().nlfem_assemble(mesh, C.byref(params), _ptr(f_nodal), _stream(stream), C.byref(h)))
    return h


def nlfem_batch_assemble(meshes, params, f_nodal=None, stream=None):
    """n systems with fused bulk launches; f_nodal: None or a list of (None | tensor)."""
    n = len(meshes)
    vp = C.c_void_p
    mh = (vp * n)(*[m.value if isinstance(m, C.c_void_p) else m for m in meshes])
    pa = (nlfem_params * n)(*params)
    fp = None
    if f_nodal is not None:
        fp = (vp * n)(*[_ptr(f) for f in f_nodal])
    out = (vp * n)()
    _check(load().nlfem_batch_assemble(mh, pa, fp, n, _stream(stream), out))
    return [C.c_void_p(h) for h in out]


def nlfem_batch_create(meshes, params, f_nodal=None, stream=None):
    n = len(meshes)
    vp = C.c_void_p
    mh = (vp * n)(*[m.value if isinstance(m, C.c_void_p) else m for m in meshes])
    pa = (nlfem_params * n)(*params)
    fp = None if f_nodal is None else (vp * n)(*[_ptr(f) for f in f_nodal])
    h = C.c_void_p()
    _check(load().nlfem_batch_create(mh, pa, fp, n, _stream(stream), C.byref(h)))
    return h


def nlfem_autotune(mesh, params: nlfem_params, stream=None) -> tuple:
    """(blocks per SM of the whole-pair kernel, of the cut-pair kernel, its outer points per chunk)."""
    best = (C.c_int32 * 3)()
    _check(load().nlfem_autotune(mesh, C.byref(params), _stream(stream), best))
    return int(best[0]), int(best[1]), int(best[2])


def nlfem_tune_set(params: nlfem_params, shape) -> None:
    """Set the launch shape (whole bps, cut bps, outer points per chunk) of a kernel class."""
    arr = (C.c_int32 * 3)(*[int(v) for v in shape])
    _check(load().nlfem_tune_set(C.byref(params), arr))


def nlfem_batch_run(batch, stream=None) -> float:
    ms = C.c_double(0.0)
    _check(load().nlfem_batch_run(batch, _stream(stream), C.byref(ms)))
    return ms.value


def nlfem_batch_system(batch, i: int):
    h = C.c_void_p()
    _check(load().nlfem_batch_system(batch, int(i), C.byref(h)))
    return h


def nlfem_batch_destroy(batch):
    load().nlfem_batch_destroy(batch)


def nlfem_system_csr(sys):
    rp, col, val = C.c_void_p(), C.c_void_p(), C.c_void_p()
    n, nnz = C.c_int64(), C.c_int64()
    _check(load().nlfem_system_csr(sys, C.byref(rp), C.byref(col), C.byref(val), C.byref(n), C.byref(nnz)))
    return rp.value, col.value, val.value, n.value, nnz.value


def nlfem_system_rhs(sys):
    F = C.c_void_p()
    _check(load().nlfem_system_rhs(sys, C.byref(F)))
    return F.value


def nlfem_system_dirichlet(sys):
    d = C.c_void_p()
    _check(load().nlfem_system_dirichlet(sys, C.byref(d)))
    return d.value


def nlfem_system_info(sys) -> dict:
    info = nlfem_assembly_info()
    _check(load().nlfem_system_info(sys, C.byref(info)))
    return info.as_dict()


def nlfem_mesh_pairs(mesh):
    k, l, n = C.c_void_p(), C.c_void_p(), C.c_int64()
    _check(load().nlfem_mesh_pairs(mesh, C.byref(k), C.byref(l), C.byref(n)))
    return k.value, l.value, n.value


def nlfem_solve(sys, g_nodal, tol_rel, max_iter, u_out, stream=None) -> dict:
    info = nlfem_solve_info()
    code = load().nlfem_solve(sys, _ptr(g_nodal), float(tol_rel), int(max_iter), _ptr(u_out),
                              C.byref(info), _stream(stream))
    out = {"iterations": info.iterations, "refinements": info.refinements, "rel_residual": info.rel_residual,
           "status": code}
    if code not in (NLFEM_OK, -6):
        _check(code)
    return out


def nlfem_solve_neumann(sys, tol_rel, max_iter, u_out, stream=None) -> dict:
    info = nlfem_solve_info()
    code = load().nlfem_solve_neumann(sys, float(tol_rel), int(max_iter), _ptr(u_out), C.byref(info),
                                      _stream(stream))
    out = {"iterations": info.iterations, "refinements": info.refinements, "rel_residual": info.rel_residual,
           "status": code}
    if code not in (NLFEM_OK, -6):
        _check(code)
    return out


CENSUS = ["evals", "full_points", "cut_points", "subtris", "duffy_points", "trunc_pairs", "singular_pairs",
          "empty_points", "outer_points", "evals_whole", "evals_cut", "outer_points_cut", "cut_points_cut",
          "nonempty_points_cut", "subtri_evals_cut", "evals_canonical"]


def nlfem_system_census(sys, stream=None) -> dict:
    c = (C.c_int64 * 16)()
    _check(load().nlfem_system_census(sys, c, _stream(stream)))
    return dict(zip(CENSUS, (int(v) for v in c)))


def nlfem_system_destroy(sys):
    load().nlfem_system_destroy(sys)


def nlfem_mesh_device_bytes(mesh) -> int:
    return int(load().nlfem_mesh_device_bytes(mesh))


def nlfem_trim_memory(stream=None) -> None:
    """Return the unused blocks of the device memory pool the library allocates from."""
    _check(load().nlfem_trim_memory(_stream(stream)))


def _check_noalloc_args(verts, elems, out_k, out_l):
    """Argument checks of nlfem_pairs_noalloc, before anything reaches the C library: the
    kernels read verts as 2 M doubles and elems as 3 K ints, and write up to capacity
    entries of out_k and out_l, so a wrong dtype, shape, stride or device is refused here."""
    import torch
    for name, t in (("verts", verts), ("elems", elems), ("out_k", out_k), ("out_l", out_l)):
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"{name} must be a torch tensor")
    if verts.dtype != torch.float64 or verts.dim() != 2 or verts.shape[1] != 2:
        raise ValueError("verts must be a float64 tensor of shape [M, 2]")
    if elems.dtype != torch.int32 or elems.dim() != 2 or elems.shape[1] != 3:
        raise ValueError("elems must be an int32 tensor of shape [K, 3]")
    for name, t in (("out_k", out_k), ("out_l", out_l)):
        if t.dtype != torch.int32 or t.dim() != 1:
            raise ValueError(f"{name} must be a one-dimensional int32 tensor")
    for name, t in (("verts", verts), ("elems", elems), ("out_k", out_k), ("out_l", out_l)):
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    for name, t in (("verts", verts), ("elems", elems), ("out_k", out_k), ("out_l", out_l)):
        if not t.is_cuda or t.device.index != torch.cuda.current_device():
            raise ValueError(f"{name} must be a CUDA tensor on the current device")
    return _noalloc_capacity(out_k, out_l)


def _noalloc_capacity(out_k, out_l) -> int:
    """Pairs the two output buffers can both hold: the shorter of the two."""
    return min(int(out_k.numel()), int(out_l.numel()))


def nlfem_pairs_noalloc(verts, elems, delta, ball, quad_outer, out_k, out_l, stream=None) -> int:
    """Interaction graph of a small mesh into caller-owned device buffers, without any
    device allocation. verts [M, 2] float64, elems [K, 3] int32, out_k / out_l int32 (contiguous
    CUDA tensors on the current device; the capacity is the shorter of the two). Returns the
    number of ordered pairs written (sorted by (k, l)). The call synchronises the stream."""
    capacity = _check_noalloc_args(verts, elems, out_k, out_l)
    n = C.c_int64(0)
    code = load().nlfem_pairs_noalloc(_ptr(verts), int(verts.shape[0]), _ptr(elems), int(elems.shape[0]),
                                      float(delta), BALLS[ball] if isinstance(ball, str) else int(ball),
                                      int(quad_outer), _ptr(out_k), _ptr(out_l), capacity,
                                      C.byref(n), _stream(stream))
    if code != NLFEM_OK:
        err = NlfemError(code, load().nlfem_last_error().decode())
        err.npairs = n.value
        raise err
    return n.value


def nlfem_mesh_create_dg(verts, elems, elem_label=None, ndof_per_node=1, stream=None):
    return nlfem_mesh_create(verts, elems, elem_label, ndof_per_node, stream, dg=True)


def nlfem_mesh_set_materials(mesh, material, stream=None) -> None:
    _check(load().nlfem_mesh_set_materials(mesh, _ptr(material), _stream(stream)))


def nlfem_last_error() -> str:
    return load().nlfem_last_error().decode()


def nlfem_version() -> str:
    return load().nlfem_version().decode()


def make_params(kernel="constant", delta=0.1, s=0.5, kconst=None, ball="nocaps", quad_outer=7, quad_inner=7,
                duffy_gauss=5, close_rule="auto", precision="fp64", mem_budget_bytes=0,
                material_scale=None, kernel_table=None, singular_precision="fp64",
                geometry_precision="fp32") -> nlfem_params:
    """nlfem_params; material_scale: symmetric n x n table of a label-dependent kernel;
    kernel_table: values of g for kernel="tabulated" (the returned struct keeps both arrays
    alive for the calls it is passed to); singular_precision ("fp64" | "fp32") and
    geometry_precision ("fp32" | "fp64"): arithmetic of the singular rule and of the cut
    geometry in the FP32-bulk path."""
    p = nlfem_params()
    p.kernel = KERNELS[kernel]
    p.delta = float(delta)
    p.s = float(s)
    p.kconst = math.nan if kconst is None else float(kconst)
    p.ball = BALLS[ball]
    p.quad_outer = int(quad_outer)
    p.quad_inner = int(quad_inner)
    p.duffy_gauss = int(duffy_gauss)
    p.close_rule = CLOSE_RULES[close_rule]
    p.precision = PRECISIONS[precision]
    p.mem_budget_bytes = int(mem_budget_bytes)
    p.singular_precision = SINGULAR_PRECISIONS[singular_precision]
    p.geometry_precision = GEOMETRY_PRECISIONS[geometry_precision]
    p.n_materials = 0
    p.material_scale = None
    if material_scale is not None:
        import numpy as np
        tab = np.ascontiguousarray(material_scale, dtype=np.float64)
        assert tab.ndim == 2 and tab.shape[0] == tab.shape[1]
        p._keep = tab
        p.n_materials = int(tab.shape[0])
        p.material_scale = tab.ctypes.data
    p.table_size = 0
    p.kernel_table = None
    if kernel_table is not None:
        import numpy as np
        kt = np.ascontiguousarray(kernel_table, dtype=np.float64).reshape(-1)
        p._keep_table = kt
        p.table_size = int(kt.size)
        p.kernel_table = kt.ctypes.data
    return p
