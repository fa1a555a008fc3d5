"""The C-ABI library builds, loads and exports every symbol include/lcbp.h declares.

CPU-only: no compute call is made (there is no GPU here); only pure host
entry points (status strings, workspace sizing) are called.
"""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in sorted(os.listdir(os.path.join(ROOT, "include")))
           if h.endswith(".h")]


@pytest.fixture(scope="module")
def libpath():
    from paper_0901_3293_gb300 import build
    return build.build()


def declared_symbols():
    names = []
    for h in HEADERS:
        text = open(h).read()
        names += re.findall(r"LCBP_API\s+[\w\s\*]+?\b(lcbp_\w+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_symbols()
    for must in ("lcbp_create", "lcbp_step", "lcbp_read_q", "lcbp_read_u", "lcbp_free_energy",
                 "lcbp_init_q", "lcbp_set_ldg", "lcbp_set_flow", "lcbp_totals"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header(libpath):
    from paper_0901_3293_gb300 import lcbp
    lcbp.lib()
    missing = [n for n in declared_symbols() if n not in lcbp._SIGNATURES]
    assert not missing, missing


def test_host_only_entry_points(libpath):
    from paper_0901_3293_gb300 import lcbp
    L = lcbp.lib()
    assert L.lcbp_version() == 1
    assert L.lcbp_strerror(lcbp.EINVAL).startswith(b"LCBP_EINVAL")
    assert L.lcbp_workspace_bytes(0, 4, 4, lcbp.F32) == 0
    assert L.lcbp_workspace_bytes(4, 4, 4, 7) == 0
    small = L.lcbp_workspace_bytes(8, 8, 8, lcbp.F32)
    big = L.lcbp_workspace_bytes(8, 8, 8, lcbp.F64)
    # 67 state/scratch values per site at least
    assert small >= 67 * 512 * 4 and big >= 67 * 512 * 8


def test_no_cpu_fallback_in_product_package():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_0901_3293_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in text and "from oracle" not in text, fn


def test_write_pgm_roundtrip(tmp_path):
    import numpy as np
    from paper_0901_3293_gb300 import lcbp
    img = np.linspace(0, 0.5, 12, dtype=np.float32).reshape(3, 4)
    path = str(tmp_path / "t.pgm")
    lcbp.write_pgm(img, path)
    data = open(path, "rb").read()
    assert data.startswith(b"P5\n4 3\n255\n")
    px = np.frombuffer(data[len(b"P5\n4 3\n255\n"):], dtype=np.uint8).reshape(3, 4)
    assert px[0, 0] == 0 and px[-1, -1] == 255
