"""The C-ABI library builds, loads and exports every symbol include/*.h declares
(no compute calls: these run without a GPU)."""
import ctypes
import glob
import os
import re

from paper_1208_2675_gb300 import build as libbuild
from paper_1208_2675_gb300 import sa

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(qap_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ["qap_sa_create", "qap_sa_run", "qap_sa_result", "qap_sa_destroy",
                 "qap_sa_strerror"]:
        assert want in names


def test_library_exports_every_declared_symbol():
    libbuild.build()
    L = ctypes.CDLL(sa.LIB_PATH)
    missing = [n for n in sorted(declared_functions()) if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert declared_functions() <= set(sa.SIGNATURES)


def test_strerror_without_device():
    libbuild.build()
    assert sa.qap_sa_strerror(sa.QAP_E_INVAL) == "invalid argument"
    assert sa.qap_sa_strerror(12345) == "unknown status"
