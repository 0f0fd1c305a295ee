"""CPU-side checks of the CUDA library: it builds, loads, and exports every
symbol include/*.h declares; argument errors come back as statuses.  No call
here touches a GPU."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:sf_status|void|const char\s*\*)\s*(\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_1009_5169_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for n in ("sf_lattice_create", "wilson_apply_block", "solve_block", "fermion_force", "plaquette_action",
              "sf_lattice_destroy", "sf_last_error", "sf_batch_create", "sf_batch_solve"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_invalid_arguments_return_status_without_gpu(libpath):
    from paper_1009_5169_gb300 import binding as sf
    lib = sf.lib()
    h = ctypes.c_void_p()
    # odd L is rejected before any CUDA call
    rc = lib.sf_lattice_create(ctypes.byref(h), 5, 4, 0.5, 0.13, 4.52, None, 0, None)
    assert rc == sf.SF_EINVAL
    assert b"even" in lib.sf_last_error()
    rc = lib.solve_block(None, 1, 5, None, None, None, 1e-10, 100, None)
    assert rc == sf.SF_EINVAL


def test_oracle_is_not_imported_by_the_package():
    pkg = os.path.join(ROOT, "paper_1009_5169_gb300")
    for f in glob.glob(os.path.join(pkg, "**", "*.py"), recursive=True) + \
            glob.glob(os.path.join(pkg, "csrc", "*")):
        text = open(f).read()
        assert "import oracle" not in text and "from oracle" not in text, f
        assert "sf_oracle" not in text, f
