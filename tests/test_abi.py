"""The C-ABI library loads without a GPU and exports exactly the functions that
include/rs.h declares (no compute calls: there may be no device here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(rs_\w+)\s*\(", text, flags=re.M))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_2508_01485_gb300 import build
    try:
        return build.build()
    except RuntimeError as e:          # no nvcc on this machine
        pytest.skip(str(e))


def test_header_declares_the_boundary():
    names = declared()
    for core in ("rs_build_graph", "rs_score", "rs_topk", "rs_apply_removals", "rs_get_interaction",
                 "rs_clone_graph", "rs_free_graph", "rs_last_error"):
        assert core in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in sorted(declared()) if not hasattr(L, n)]
    assert not missing, missing


def test_library_exports_nothing_undeclared(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("nm unavailable")
    exported = {line.split()[-1] for line in out.stdout.splitlines() if line.split()[-1].startswith("rs_")}
    assert exported == declared()


def test_binding_tuning_struct_matches_the_header():
    """The Python mirror of rs_tuning lists the header's int32 fields in the header's order."""
    text = open(os.path.join(ROOT, "include", "rs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    body = re.search(r"typedef struct \{([^}]*)\} rs_tuning;", text).group(1)
    fields = re.findall(r"int32_t\s+(\w+)\s*;", body)
    assert len(fields) == len([x for x in body.split(";") if x.strip()])
    from paper_2508_01485_gb300 import _lib
    assert tuple(fields) == _lib.TUNING_FIELDS
