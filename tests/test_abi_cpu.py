"""CPU checks of the C-ABI library: it builds for sm_103a, loads, and exports
every entry point include/*.h declares.  No compute call is made."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


CPU_HEADER = "idm_cpu.h"   # declared by libidm_cpu.so, the separate CPU backend


def header_functions(cpu=False):
    """Functions declared by the CUDA library's headers (cpu=False) or by the
    CPU backend's header (cpu=True)."""
    src = ""
    for name in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if name.endswith(".h") and (name == CPU_HEADER) == cpu:
            src += open(os.path.join(ROOT, "include", name)).read() + "\n"
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+char\s*\*|int|size_t)\s*\**\s*(idm_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2412_16750_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = header_functions()
    for must in ("idm_ctx_create", "idm_ctx_destroy", "idm_forward", "idm_backward", "idm_loss_grad", "idm_fit",
                 "idm_layout", "idm_status", "idm_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in header_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(libpath):
    from paper_2412_16750_gb300 import lib
    assert set(lib.exported_symbols()) == set(header_functions())
    lib.load(libpath)


def test_query_without_device(libpath):
    from paper_2412_16750_gb300 import lib
    lib.load(libpath)
    assert lib.idm_max_lane_supported() == 2048


def test_null_context_is_rejected(libpath):
    from paper_2412_16750_gb300 import lib
    L = lib.load(libpath)
    assert L.idm_ctx_create(None, 0) == lib.IDM_ERR_ARG
    assert L.idm_ctx_destroy(None) == lib.IDM_OK
    assert L.idm_set_tuning(None, 0, 0, 16, 8) == lib.IDM_ERR_ARG
    assert L.idm_set_fit_mode(None, lib.IDM_FIT_AUTO) == lib.IDM_ERR_ARG
    assert L.idm_last_fit_form(None) == 0


def test_cpu_backend_exports_its_header():
    from paper_2412_16750_gb300 import build, cpu
    path = build.build_cpu()
    lib = ctypes.CDLL(path)
    names = header_functions(cpu=True)
    assert names and all(hasattr(lib, n) for n in names)
    assert set(cpu.exported_symbols()) == set(names)
    # the CUDA library carries no CPU path
    assert not any(hasattr(ctypes.CDLL(build.LIB), n) for n in names)


def test_missing_library_fails_loudly(tmp_path):
    from paper_2412_16750_gb300 import lib
    saved = lib._lib
    try:
        lib._lib = None
        with pytest.raises(RuntimeError, match="no CPU"):
            lib.load(str(tmp_path / "nope.so"))
    finally:
        lib._lib = saved


def test_param_row_pointers_without_views():
    """make_params builds the six row pointers from the base pointer and the
    row stride; they equal the rows' own data pointers, also for a (6, N)
    slice of a wider tensor, and a tensor whose rows are not contiguous falls
    back to the rows' pointers."""
    import torch
    from paper_2412_16750_gb300 import lib

    def rows(s):
        return [getattr(s, f[0]) for f in s._fields_]

    t = torch.zeros(6, 1000)
    assert rows(lib.make_params(t)) == [t[q].data_ptr() for q in range(6)]
    wide = torch.zeros(6, 1500)
    sl = wide[:, 100:1100]
    assert rows(lib.make_params(sl)) == [sl[q].data_ptr() for q in range(6)]
    tr = torch.zeros(1000, 6).t()  # rows with stride 6
    assert rows(lib.make_params(tr)) == [tr[q].data_ptr() for q in range(6)]
