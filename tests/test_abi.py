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


def _header_constants():
    """#define values and enumerator values of include/apsp.h."""
    text = open(os.path.join(ROOT, "include", "apsp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    vals = {}
    for m in re.finditer(r"#define\s+(APSP_\w+)\s+(0x[0-9A-Fa-f]+|\d+)", text):
        vals[m.group(1)] = int(m.group(2), 0)
    for body in re.findall(r"enum\s*\{(.*?)\}", text, flags=re.S):
        for m in re.finditer(r"(APSP_\w+)\s*=\s*(\d+)u?", body):
            vals[m.group(1)] = int(m.group(2))
    return vals


def test_binding_constants_match_the_header():
    from paper_2412_15122_gb300 import apsp
    h = _header_constants()
    assert h["APSP_INF_I32"] == apsp.APSP_INF_I32
    assert h["APSP_MAX_CAPACITY"] == apsp.APSP_MAX_CAPACITY
    assert h["APSP_MODEL_NPARAM"] == apsp.MODEL_NPARAM and h["APSP_MODEL_NTRAIN"] == apsp.MODEL_NTRAIN
    assert (h["APSP_I32"], h["APSP_F32"]) == (apsp.APSP_I32, apsp.APSP_F32)
    assert (h["APSP_UNDIRECTED"], h["APSP_D_GIVEN"], h["APSP_DEVICE_INPUT"], h["APSP_MINIMAX"]) == \
        (apsp.APSP_UNDIRECTED, apsp.APSP_D_GIVEN, apsp.APSP_DEVICE_INPUT, apsp.APSP_MINIMAX)
    for code, name in apsp.STATUS.items():
        assert h[name] == code, name
    assert [h["APSP_DISPATCH_DELTA"], h["APSP_DISPATCH_ALWAYS_WARM"], h["APSP_DISPATCH_ALWAYS_COLD"],
            h["APSP_DISPATCH_MODEL"]] == [apsp.DISPATCH[k] for k in ("delta", "warm", "cold", "model")]
    assert [h["APSP_LIST_COROLLARY3"], h["APSP_LIST_DIRECT_EDGE"], h["APSP_LIST_ALGORITHM12"]] == \
        [apsp.LIST_MODES[k] for k in ("corollary3", "direct_edge", "algorithm12")]
    assert [h["APSP_BATCH_ADD"], h["APSP_BATCH_REMOVE"], h["APSP_BATCH_EDGE"], h["APSP_BATCH_QUERY"]] == \
        [apsp.BATCH_OPS[k] for k in ("add", "remove", "edge", "query")]


def test_struct_layouts_match_the_header(tmp_path):
    # sizes and field offsets of the C structs, as a C compiler lays them out
    # from include/apsp.h, equal those of the ctypes mirrors in the binding
    import shutil
    import subprocess
    from paper_2412_15122_gb300 import apsp
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    structs = {"apsp_stats": apsp.apsp_stats, "apsp_info": apsp.apsp_info, "apsp_batch_item": apsp.apsp_batch_item,
               "apsp_request": apsp.apsp_request, "apsp_request_result": apsp.apsp_request_result,
               "apsp_serve_config": apsp.apsp_serve_config, "apsp_profile_entry": apsp.apsp_profile_entry,
               "apsp_batch_info": apsp.apsp_batch_info}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "apsp.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'printf("{name}.{field} %zu\\n", offsetof({name}, {field}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    r = subprocess.run([gcc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert int(got[f"{name}.{field}"]) == getattr(cls, field).offset, f"{name}.{field}"


def test_binding_fails_loudly_without_the_library(monkeypatch):
    # no silent fallback: a missing CUDA library is an error, not a CPU path
    from paper_2412_15122_gb300 import apsp
    monkeypatch.setattr(apsp, "_lib", None)
    monkeypatch.setattr(apsp, "LIB_PATH", os.path.join(ROOT, "no_such_dir", "libapsp_gb300.so"))
    with pytest.raises(RuntimeError, match="not built"):
        apsp.lib()
