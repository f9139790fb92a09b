"""CPU checks of the boundary: the CUDA library builds, loads, and exports
every entry point that include/*.h declares (no compute calls without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(apsp_\w+)\s*\(", text, flags=re.M):
            if "typedef" in text[text.rfind("\n", 0, m.start()) + 1:m.start() + 1]:
                continue
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2412_15122_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("apsp_init", "apsp_add_node", "apsp_remove_node", "apsp_update_edge", "apsp_query",
                     "apsp_destroy", "apsp_copy_D", "apsp_last_stats"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert missing == []


def test_version_and_status_strings(lib):
    lib.apsp_version.restype = ctypes.c_char_p
    lib.apsp_status_string.restype = ctypes.c_char_p
    assert lib.apsp_version().decode().count(".") == 2
    assert lib.apsp_status_string(0) == b"ok"
    assert lib.apsp_status_string(4) == b"no free slot"


def test_binding_names_match_the_c_entry_points():
    from paper_2412_15122_gb300 import apsp
    for n in declared_functions():
        if n in ("apsp_set_allocator",):
            continue
        assert hasattr(apsp, n), n


def test_init_rejects_bad_arguments_without_touching_the_device(lib):
    h = ctypes.c_void_p()
    # capacity < n and capacity above the maximum are argument errors
    assert lib.apsp_init(ctypes.byref(h), None, 4, 2, 0, 0, None, None) in (1, 6)
    assert lib.apsp_init(None, None, 0, 1, 0, 0, None, None) == 1
