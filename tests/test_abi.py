"""The C-ABI library builds, loads without a GPU, and exports every function
declared in include/*.h; the Python binding declares the same names.  No
compute call is made here."""
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
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(qtt_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2501_07778_gb300 import _lib
    lib = ctypes.CDLL(_lib.LIB_PATH)
    declared = _declared_functions()
    assert "qtt_solve" in declared and "qtt_to_full" in declared and "qtt_assemble_stiffness" in declared
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing
    # the binding binds exactly the declared entry points
    assert set(_lib.exported_symbols()) == declared


def test_binding_loads_and_reports_errors_without_gpu():
    import paper_2501_07778_gb300 as q
    lib = q.lib()
    assert lib.qtt_last_error() is not None
    # an argument error is reported before any device work
    rc = lib.qtt_round(None, 1e-3, 0, None)
    assert rc == -1
    assert b"null" in lib.qtt_last_error()


def test_struct_layouts_match_header():
    """Field order of the marshalled structs follows include/qtt.h."""
    from paper_2501_07778_gb300 import _lib
    text = open(os.path.join(ROOT, "include", "qtt.h")).read()
    for struct, fields in [("qtt_solve_opts", _lib.QttSolveOpts._fields_),
                           ("qtt_solve_info", _lib.QttSolveInfo._fields_),
                           ("qtt_problem", _lib.QttProblem._fields_)]:
        body = re.search(r"typedef struct \{([^}]*)\}\s*" + struct + ";", text).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        names = re.findall(r"\b(\w+)\s*[,;]", body)
        assert names == [f for f, _ in fields], (struct, names)
