"""The C-ABI library builds, loads and exports every symbol include/lsrtm.h
declares (no compute calls: these run without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lsrtm.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lsrtm_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("lsrtm_create", "lsrtm_born", "lsrtm_adjoint", "lsrtm_psf",
                     "lsrtm_cg_solve", "lsrtm_destroy", "lsrtm_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2508_10405_gb300 import build
    so = build.build()
    lib = ctypes.CDLL(so)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_export_list_matches_header():
    from paper_2508_10405_gb300 import EXPORTS
    assert sorted(EXPORTS) == _declared()


def test_last_error_callable_without_gpu():
    from paper_2508_10405_gb300 import load_library
    lib = load_library()
    assert lib.lsrtm_last_error() == b""


def test_config_struct_layout_matches_header():
    """The ctypes mirror of lsrtm_config has the header's field order."""
    from paper_2508_10405_gb300.binding import Config
    src = open(HEADER).read()
    body = re.search(r"typedef struct \{(.*?)\} lsrtm_config;", src, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        parts = decl.split(None, 1)[1] if len(decl.split(None, 1)) > 1 else decl
        names += [p.strip() for p in parts.split(",")]
    assert [f[0] for f in Config._fields_] == names
