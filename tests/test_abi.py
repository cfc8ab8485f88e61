"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/ledds.h declares (no GPU needed: nothing here calls into CUDA)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "ledds.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ledds_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("ledds_create", "ledds_step", "ledds_set_particles", "ledds_read_fields",
                     "ledds_read_forces", "ledds_set_wall_velocity", "ledds_set_forcing"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2512_04997_gb300 import build
    if not os.path.exists("/usr/local/cuda/bin/nvcc") and not os.path.exists(build.LIB):
        pytest.skip("nvcc not available to build the library")
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    # a call that touches no device: version and error strings
    lib.ledds_strerror.restype = ctypes.c_char_p
    assert lib.ledds_version() >= 1
    assert lib.ledds_strerror(-1) == b"invalid argument"


def test_binding_names_match_header():
    from paper_2512_04997_gb300 import ledds
    assert set(ledds._SIGS) == set(_declared())


def test_invalid_arguments_rejected_without_gpu():
    """Argument checks run on the host before any CUDA call."""
    from paper_2512_04997_gb300 import ledds
    L = ledds.lib()
    p = ledds.make_params(tau=0.5)   # tau must exceed 1/2
    d = ledds.make_dims(8, 8, 8)
    n = ctypes.c_size_t(0)
    assert L.ledds_workspace_size(ctypes.byref(d), ctypes.byref(p), ctypes.byref(n)) == -1
    p = ledds.make_params()
    assert L.ledds_workspace_size(ctypes.byref(d), ctypes.byref(p), ctypes.byref(n)) == 0
    assert n.value >= 2 * 19 * 512 * 4
    d2 = ledds.make_dims(0, 0, 0, max_particles=10)   # DEM-only needs a grid spacing
    assert L.ledds_workspace_size(ctypes.byref(d2), ctypes.byref(p), ctypes.byref(n)) == -1
