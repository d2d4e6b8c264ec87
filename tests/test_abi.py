"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function that include/cdr.h declares (no compute call: there may be no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cdr.h")


def _header_text():
    with open(HEADER) as f:
        s = f.read()
    s = re.sub(r"/\*.*?\*/", " ", s, flags=re.S)
    return re.sub(r"//[^\n]*", " ", s)


def declared_functions():
    return sorted(set(re.findall(r"\b(cdr_\w+)\s*\(", _header_text())))


def declared_enum(name):
    m = re.search(r"\b%s\s*=\s*(-?\d+)" % name, _header_text())
    return int(m.group(1))


@pytest.fixture(scope="module")
def built_lib():
    from paper_1903_03406_gb300 import build
    try:
        path = build.build()
    except FileNotFoundError:
        pytest.skip("nvcc not available")
    return path


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("cdr_create", "cdr_refine", "cdr_round", "cdr_export", "cdr_destroy",
                 "cdr_delaunay_box", "cdr_eval_predicates"):
        assert must in names


def test_library_exports_every_declared_function(built_lib):
    L = ctypes.CDLL(built_lib)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, "declared in cdr.h but not exported: %s" % missing


def test_host_only_calls_and_status_codes(built_lib):
    L = ctypes.CDLL(built_lib)
    L.cdr_status_string.restype = ctypes.c_char_p
    L.cdr_status_string.argtypes = [ctypes.c_int]
    assert L.cdr_device_arch() == 103
    codes = ("CDR_OK", "CDR_ROUND_LIMIT", "CDR_ERR_INVALID_INPUT", "CDR_ERR_OOM", "CDR_ERR_CUDA",
             "CDR_ERR_ITER_LIMIT", "CDR_ERR_INTERNAL", "CDR_ERR_TOO_LARGE")
    texts = set()
    for c in codes:
        t = L.cdr_status_string(declared_enum(c)).decode()
        assert t and t != "unknown status", c
        texts.add(t)
    assert len(texts) == len(codes)
    # argument checks happen on the host, before any device work
    assert L.cdr_create(None, None, None, None, None) == declared_enum("CDR_ERR_INVALID_INPUT")


def test_binding_constants_match_header():
    from paper_1903_03406_gb300 import cdr
    m = re.search(r"#define\s+CDR_EVAL_NOALLOC_MAX_ITEMS\s+(\d+)", _header_text())
    assert int(m.group(1)) == cdr.EVAL_NOALLOC_MAX_ITEMS
    assert declared_enum("CDR_ERR_TOO_LARGE") == -6


def test_plain_c_caller(built_lib, tmp_path):
    """cdr.h compiles as C99 and a C program links libcdr.so and calls it
    (host-side calls only: no GPU is needed)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    exe = str(tmp_path / "c_abi_host")
    libdir = os.path.dirname(built_lib)
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                    "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c_abi_host.c"), "-L", libdir, "-lcdr",
                    "-Wl,-rpath," + libdir, "-o", exe], check=True)
    p = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert p.returncode == 0, p.stdout + p.stderr
    assert p.stdout.strip().endswith("ok")
