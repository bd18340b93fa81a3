"""Host-side checks of the C ABI (no GPU): the library loads, exports every
symbol that include/gjp.h declares, and validates geometry arguments on the
host without touching CUDA."""
import ctypes
import os
import re

import numpy as np
import pytest

import synth
from paper_1609_00958_gb300 import _capi, Geometry, GjpError

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1609_00958_gb300 import build
    build.build()
    return _capi.load()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "gjp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gjp_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_abi():
    assert declared_symbols() == sorted(_capi.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    raw = ctypes.CDLL(_capi.LIB_PATH)
    for name in declared_symbols():
        assert hasattr(raw, name), name


def test_status_strings(lib):
    assert _capi.gjp_status_string(0) == "GJP_OK"
    assert _capi.gjp_status_string(1) == "GJP_ERR_INVALID_ARG"
    assert _capi.gjp_status_string(99) == "GJP_ERR_UNKNOWN"


def _geom(n_views=3):
    return synth.circular(n_views, 16, 12, 100.0, 200.0, 1.5)


def test_geometry_create_info_destroy(lib):
    cg = _geom()
    g = Geometry.from_cone(cg)
    st, nvw, nu, nv = _capi.gjp_geometry_info(g.handle)
    assert (st, nvw, nu, nv) == (0, 3, 16, 12)
    g.close()
    g.close()  # idempotent
    _capi.gjp_geometry_destroy(None)  # NULL-safe


@pytest.mark.parametrize("bad", ["nan_src", "zero_u", "parallel_uv", "src_on_panel", "n0", "nu0"])
def test_geometry_rejects_invalid(lib, bad):
    cg = _geom()
    src, org, du, dv = cg.src.copy(), cg.det_origin.copy(), cg.det_u.copy(), cg.det_v.copy()
    n, nu, nv = cg.n_views, cg.nu, cg.nv
    if bad == "nan_src":
        src[1, 0] = np.nan
    elif bad == "zero_u":
        du[2] = 0.0
    elif bad == "parallel_uv":
        dv[0] = 2.0 * du[0]
    elif bad == "src_on_panel":
        src[0] = org[0] + 3.0 * du[0] + 5.0 * dv[0]
    elif bad == "n0":
        n = 0
        src, org, du, dv = [a[:0] for a in (src, org, du, dv)]
    elif bad == "nu0":
        nu = 0
    st, h = _capi.gjp_geometry_create(n, nu, nv, src, org, du, dv)
    assert st == _capi.GJP_ERR_INVALID_ARG and h is None


def test_null_arguments_rejected_without_cuda(lib):
    cg = _geom()
    g = Geometry.from_cone(cg)
    # NULL volume / projection pointers are rejected before any CUDA call
    assert _capi.gjp_forward(0, 0, 8, 8, 8, (1, 1, 1), None, g.handle, 0, 0) == _capi.GJP_ERR_INVALID_ARG
    assert _capi.gjp_adjoint(0, g.handle, 8, 8, 8, (1, 1, 1), None, 0, 0, 0) == _capi.GJP_ERR_INVALID_ARG
    assert _capi.gjp_forward(16, 7, 8, 8, 8, (1, 1, 1), None, g.handle, 16, 0) == _capi.GJP_ERR_INVALID_ARG
    assert _capi.gjp_forward(16, 0, 0, 8, 8, (1, 1, 1), None, g.handle, 16, 0) == _capi.GJP_ERR_INVALID_ARG
    assert _capi.gjp_forward(16, 0, 8, 8, 8, (1, -1, 1), None, g.handle, 16, 0) == _capi.GJP_ERR_INVALID_ARG
    assert _capi.gjp_forward(16, 0, 8, 8, 8, (1, 1, 1), None, None, 16, 0) == _capi.GJP_ERR_INVALID_ARG


def test_source_inside_volume_rejected_without_cuda(lib):
    cg = _geom()
    g = Geometry.from_cone(cg)
    # a 300^3 unit grid contains the sources at radius 100
    assert _capi.gjp_forward(16, 0, 300, 300, 300, (1, 1, 1), None, g.handle, 16, 0) == \
        _capi.GJP_ERR_INVALID_ARG


def test_python_layer_refuses_cpu_tensors(lib):
    import torch
    import paper_1609_00958_gb300 as gjp
    g = Geometry.from_cone(_geom())
    with pytest.raises(ValueError):
        gjp.forward(torch.zeros(4, 4, 4), g)
    with pytest.raises(GjpError):
        Geometry(np.zeros((2, 3)), np.zeros((2, 3)), np.zeros((2, 3)), np.zeros((2, 3)), 4, 4)


def test_problem_struct_layout_matches_header(tmp_path):
    """The ctypes mirror of gjp_problem has the C layout: every field offset
    and the size, as the C compiler lays out include/gjp.h."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = [f[0] for f in _capi.GjpProblem._fields_]
    src = tmp_path / "layout.c"
    src.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"gjp.h\"\nint main(void){\n"
                   + "".join(f'printf("%zu\\n", offsetof(gjp_problem, {f}));\n' for f in fields)
                   + 'printf("%zu\\n", sizeof(gjp_problem));\nreturn 0;}\n')
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = [getattr(_capi.GjpProblem, f).offset for f in fields] + [ctypes.sizeof(_capi.GjpProblem)]
    assert got == want


def test_batch_create_rejects_bad_arguments_without_a_gpu(lib):
    st, h = _capi.gjp_batch_create([])
    assert st == _capi.GJP_ERR_INVALID_ARG and h is None
    r = _capi.GjpProblem()            # NULL volume / geometry / projections
    st, h = _capi.gjp_batch_create([r])
    assert st == _capi.GJP_ERR_INVALID_ARG and h is None
    assert _capi.gjp_batch_forward(None, 0) == _capi.GJP_ERR_INVALID_ARG
    assert _capi.gjp_batch_autotune(None, 0, 1) == _capi.GJP_ERR_INVALID_ARG
    assert _capi.gjp_batch_get_tuning(None, 0)[0] == _capi.GJP_ERR_INVALID_ARG
    assert _capi.gjp_batch_launch_count(None)[0] == _capi.GJP_ERR_INVALID_ARG
    _capi.gjp_batch_destroy(None)


def test_forward_path_validation_without_cuda(lib):
    """GJP_PATH_PAIRS is a forward family only; unknown families are
    rejected before any CUDA call; trimming the (empty) workspace pools is
    host-only."""
    g = Geometry.from_cone(_geom())
    assert _capi.gjp_forward_ex(16, 0, 8, 8, 8, (1, 1, 1), None, g.handle, 16, 99, 0) == _capi.GJP_ERR_INVALID_ARG
    assert _capi.gjp_adjoint_ex(16, g.handle, 8, 8, 8, (1, 1, 1), None, 16, 0, _capi.GJP_PATH_PAIRS, 0) == \
        _capi.GJP_ERR_INVALID_ARG
    assert _capi.gjp_forward_ex(0, 0, 8, 8, 8, (1, 1, 1), None, g.handle, 16, _capi.GJP_PATH_PAIRS, 0) == \
        _capi.GJP_ERR_INVALID_ARG
    assert _capi.gjp_trim_workspace() == _capi.GJP_OK


def test_debug_fail_allocations_arguments(lib):
    """The out-of-memory injection hook is host-only: it takes a count and
    rejects a negative one (its effect is tested on the GPU)."""
    assert _capi.gjp_debug_fail_allocations(-1) == _capi.GJP_ERR_INVALID_ARG
    assert _capi.gjp_debug_fail_allocations(3) == _capi.GJP_OK
    assert _capi.gjp_debug_fail_allocations(0) == _capi.GJP_OK
