"""The C-ABI library loads and exports every entry point include/fipt.h
declares; host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "fipt.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:fipt_status|const char\*|uint64_t)\s+(fipt_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def L():
    from paper_2304_05669_gb300 import _native
    return _native.lib()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("fipt_scene_create", "fipt_bake", "fipt_render_fwd", "fipt_render_bwd",
                 "fipt_tri_error", "fipt_trace_closest", "fipt_camera_queries"):
        assert must in names


def test_library_exports_every_declared_symbol(L):
    missing = [n for n in declared_symbols() if not hasattr(L, n)]
    assert missing == []


def test_python_signatures_cover_the_header():
    from paper_2304_05669_gb300 import _native
    assert set(declared_symbols()) <= set(_native.SIGNATURES)


def test_host_side_argument_checks(L):
    from paper_2304_05669_gb300 import _native
    n = ctypes.c_size_t()
    assert L.fipt_scene_workspace_size(100, 36, ctypes.byref(n)) == 0
    assert n.value > 36 * (64 + 48 + 32)
    assert L.fipt_scene_workspace_size(-1, 36, ctypes.byref(n)) == 1
    assert L.fipt_bake(None, None, 0, None, None, None, None, None) == 1
    assert b"NULL" in L.fipt_last_error()
    p = _native.BakeParams()
    p.K = 0
    assert L.fipt_bake(ctypes.c_void_p(1), None, 10, ctypes.byref(p), None, None, None, None) == 1
    assert L.fipt_tri_error_workspace_size(10, 5, ctypes.byref(n)) == 0
    assert L.fipt_render_workspace_size(1000, ctypes.byref(n)) == 0
    assert L.fipt_compact_workspace_size(1000, ctypes.byref(n)) == 0
    assert L.fipt_status_string(3) == b"workspace too small"
    assert L.fipt_version().startswith(b"fipt-gb300")


def test_refine_workspace_and_render_pass_checks(L):
    """Host arithmetic of the refinement's workspace (184 B of path state per
    sample, at most 2^24 samples per chunk, whole points) and the argument
    checks of the one-pass render, none of which touches a device."""
    from paper_2304_05669_gb300 import _native
    n = ctypes.c_size_t()
    p = _native.BakeParams()
    p.K, p.spp_diffuse, p.spp_specular = 6, 32, 32           # 224 samples per point
    assert L.fipt_bake_refine_workspace_size(1000, ctypes.byref(p), 8, ctypes.byref(n)) == 0
    assert 1000 * 224 * 184 <= n.value <= 1000 * 224 * 184 + 64 * 1024
    small = n.value
    assert L.fipt_bake_refine_workspace_size(1 << 20, ctypes.byref(p), 8, ctypes.byref(n)) == 0
    per_chunk = (1 << 24) // 224
    assert per_chunk * 224 * 184 <= n.value <= per_chunk * 224 * 184 + 64 * 1024 and n.value > small
    assert L.fipt_bake_refine_workspace_size(0, ctypes.byref(p), 8, ctypes.byref(n)) == 0 and n.value == 0
    p.spp_diffuse = 1 << 24                                    # one point over a chunk
    assert L.fipt_bake_refine_workspace_size(1, ctypes.byref(p), 8, ctypes.byref(n)) == 1
    p.spp_diffuse = 32
    assert L.fipt_bake_refine_workspace_size(1, ctypes.byref(p), 4096, ctypes.byref(n)) == 1
    grid = (ctypes.c_float * 1)(0.5)                           # K = 1: a lerp needs two nodes
    assert L.fipt_render_fwd_grad(None, None, None, 10, 1, grid, None, None, None, None, None, None, None,
                                  None, None, None, None, 0, None) == 1
    assert L.fipt_render_grad_scale(0, None, None, None, None, None) == 0
    assert L.fipt_render_grad_scale(5, None, None, None, None, None) == 1


def test_query_record_is_40_bytes():
    # x, n, wo (9 floats) + tri (int32), the layout the bindings pack
    class Q(ctypes.Structure):
        _fields_ = [("x", ctypes.c_float * 3), ("n", ctypes.c_float * 3),
                    ("wo", ctypes.c_float * 3), ("tri", ctypes.c_int32)]
    assert ctypes.sizeof(Q) == 40


def _toolchain():
    import shutil
    from paper_2304_05669_gb300 import build, _native
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    lib = _native.library_path()
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(build._nvcc())), "lib64")
    return gcc, lib, cuda_lib


def test_header_is_standalone_c_and_cxx(tmp_path):
    """include/fipt.h compiles alone as C11 and as C++17, warnings as errors."""
    import subprocess
    gcc, _lib, _cuda = _toolchain()
    src = tmp_path / "h.c"
    src.write_text('#include "fipt.h"\nint main(void) { return (int)sizeof(fipt_query) - 40; }\n')
    inc = os.path.join(ROOT, "include")
    subprocess.run([gcc, "-std=c11", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", inc, "-fsyntax-only",
                    str(src)], check=True)
    subprocess.run([gcc, "-x", "c++", "-std=c++17", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", inc,
                    "-fsyntax-only", str(src)], check=True)


def test_c_client_links_and_host_calls_answer(tmp_path):
    """tests/c/abi_host.c, a C11 client, links against the library and checks
    the host-side calls (version, status strings, workspace queries,
    argument errors, the admission arena) without a GPU."""
    import subprocess
    gcc, lib, cuda_lib = _toolchain()
    exe = tmp_path / "abi_host"
    libdir = os.path.dirname(lib)
    subprocess.run([gcc, "-std=c11", "-Wall", "-Wextra", "-pedantic", "-Werror",
                    "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c", "abi_host.c"),
                    "-L", libdir, "-l", "fipt", "-Wl,-rpath," + libdir, "-L", cuda_lib,
                    "-Wl,-rpath-link," + cuda_lib, "-o", str(exe)], check=True)
    env = dict(os.environ)
    env["LD_LIBRARY_PATH"] = cuda_lib + os.pathsep + env.get("LD_LIBRARY_PATH", "")
    out = subprocess.run([str(exe)], env=env, capture_output=True, text=True)
    assert out.returncode == 0, out.stderr
    assert "abi host checks ok" in out.stdout
