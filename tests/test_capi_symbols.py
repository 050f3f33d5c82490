"""The C ABI library builds, loads and exports every function include/nlfem.h declares (CPU)."""
import ctypes
import os
import re

from paper_2207_03921_gb300 import binding


def test_library_loads_and_exports_header_symbols():
    lib = binding.load()
    syms = binding.header_symbols()
    assert len(syms) >= 12
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing
    assert binding.nlfem_version().startswith("nlfem")


def test_header_documents_every_function():
    hdr = open(os.path.join(os.path.dirname(binding.lib_path()), "..", "..", "include", "nlfem.h")).read()
    assert "extern \"C\"" in hdr
    for s in binding.header_symbols():
        assert re.search(r"\b" + s + r"\s*\(", hdr)


def test_params_default_without_gpu():
    # a pure host call: fills the defaults of Sec. 3.1
    p = binding.nlfem_params_default(1)
    assert p.kernel == 1 and p.quad_outer == 7 and p.quad_inner == 7 and p.duffy_gauss == 5
    assert p.delta > 0 and p.ball == 0


def test_python_binding_names_match_c_abi():
    for s in binding.header_symbols():
        assert hasattr(binding, s), s


def test_library_is_in_tree_and_not_a_cpu_fallback():
    path = binding.lib_path()
    assert os.path.dirname(os.path.dirname(path)).endswith("paper_2207_03921_gb300")
    lib = ctypes.CDLL(path)
    assert hasattr(lib, "nlfem_assemble")


def test_null_handles_fail_with_invalid_arg_and_a_thread_local_message():
    # host-side argument checks: no CUDA call is made before them
    import threading
    lib = binding.load()
    info = binding.nlfem_assembly_info()
    assert lib.nlfem_system_info(None, ctypes.byref(info)) == -1 and binding.ERRORS[-1] == "INVALID_ARG"
    msg = binding.nlfem_last_error()
    assert "NULL" in msg
    seen = []
    t = threading.Thread(target=lambda: seen.append(binding.nlfem_last_error()))
    t.start()
    t.join()
    assert seen == [""]                      # the message belongs to the failing thread
    assert binding.nlfem_last_error() == msg
    # destroying a NULL handle is a no-op
    lib.nlfem_mesh_destroy(None)
    lib.nlfem_system_destroy(None)
    lib.nlfem_batch_destroy(None)
    assert lib.nlfem_mesh_device_bytes(None) == 0
