"""The C ABI library builds for sm_103a, loads, and exports every function include/ declares.
No compute calls (no GPU needed)."""
import os
import re
import subprocess

import pytest

from conftest import ROOT


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            text = open(os.path.join(inc, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            for m in re.finditer(r"^\s*(?:int|const char\*|int64_t|void)\s+(lob_\w+)\s*\(", text, flags=re.M):
                names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def built_lib():
    from paper_1609_01689_gb300 import _build
    return _build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("lob_create", "lob_spmm", "lob_solve", "lob_destroy", "lob_strerror", "lob_gram", "lob_lincomb",
              "lob_precond_apply", "lob_rayleigh_ritz", "lob_export_tiles", "lob_matrix_info_get", "lob_spmm_batch",
              "lob_server_create", "lob_server_submit", "lob_server_progress", "lob_server_poll",
              "lob_server_destroy"):
        assert f in names


def test_library_exports_every_declared_symbol(built_lib):
    out = subprocess.run(["nm", "-D", "--defined-only", built_lib], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = declared_functions() - exported
    assert not missing, missing


def test_library_loads_and_reports_errors(built_lib):
    import paper_1609_01689_gb300 as lob
    lib = lob.build()
    assert lob.strerror(lob.LOB_ERR_ARG) == "invalid argument"
    assert lob.strerror(lob.LOB_ERR_NOCONV).startswith("iteration limit")
    # argument checks happen before any device work
    assert lib.lob_spmm(None, 0, None, None, 8, None) == lob.LOB_ERR_ARG
    assert lib.lob_gram(0, 1, None, 1, 1, None, 1, None, 0, None) == lob.LOB_ERR_ARG
    assert lib.lob_destroy(None) == lob.LOB_OK
    assert lib.lob_spmm_batch(1, None, None, None, None, None, None, None) == lob.LOB_ERR_ARG
    assert lib.lob_spmm_batch(0, None, None, None, None, None, None, None) == lob.LOB_OK
    assert lib.lob_server_create(None, None) == lob.LOB_ERR_ARG
    assert lib.lob_server_submit(None, None, None) == lob.LOB_ERR_ARG
    assert lib.lob_server_progress(None, 0, None) == lob.LOB_ERR_ARG
    assert lib.lob_server_poll(None, 1, None) == lob.LOB_ERR_ARG
    assert lib.lob_server_destroy(None) == lob.LOB_ERR_ARG
    assert lib.lob_batch_create(0, None, None, None) == lob.LOB_ERR_ARG
    assert lib.lob_batch_solve(None, None, None, None, None, None, None) == lob.LOB_ERR_ARG
    assert lib.lob_batch_destroy(None) == lob.LOB_OK
    assert lib.lob_vcreate(None, None, 0, 0, None, None) == lob.LOB_ERR_ARG
    assert lib.lob_vspmm(None, None, None, 1, None) == lob.LOB_ERR_ARG
    assert lib.lob_vdestroy(None) == lob.LOB_OK


def test_synth_device_library_builds():
    import synth
    assert os.path.exists(synth.build_device())


def test_binding_struct_layouts_match_the_header(built_lib):
    """Every ctypes mirror of an ABI struct has the size the C compiler gives the header's struct."""
    import ctypes

    import paper_1609_01689_gb300 as lob
    lib = lob.build()
    lib.lob_struct_size.restype = ctypes.c_int64
    lib.lob_struct_size.argtypes = [ctypes.c_char_p]
    pairs = {"lob_coo": lob.Coo, "lob_create_opts": lob.CreateOpts, "lob_matrix_info": lob.MatrixInfo,
             "lob_solve_opts": lob.SolveOpts, "lob_stats": lob.Stats, "lob_lanczos_stats": lob.LanczosStats,
             "lob_server_opts": lob.ServerOpts, "lob_request": lob.Request, "lob_result": lob.Result,
             "lob_server_stats": lob.ServerStats, "lob_batch_opts": lob.BatchOpts,
             "lob_batch_stats": lob.BatchStats, "lob_vmatrix_info": lob.VMatrixInfo}
    for name, cls in pairs.items():
        assert lib.lob_struct_size(name.encode()) == ctypes.sizeof(cls), name
    assert lib.lob_struct_size(b"no_such_struct") == 0
    assert lib.lob_struct_size(None) == 0
