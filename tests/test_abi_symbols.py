"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every entry point that
include/*.h declares (no compute calls here)."""
import ctypes
import glob
import os
import re

from paper_2410_14117_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"^\s*(?:mg_status|const char\s*\*)\s*(mg_\w+)\s*\(", text,
                                re.M))
    return names


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("mg_create", "mg_destroy", "mg_randomize", "mg_set_actions", "mg_step",
                     "mg_get_state", "mg_reset", "mg_set_state", "mg_get_params", "mg_sync",
                     "mg_last_error", "mg_set_stream"):
        assert required in names


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in sorted(declared_symbols()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    names = declared_symbols() - {"mg_last_error"}
    assert names <= set(_lib.SIGNATURES), names - set(_lib.SIGNATURES)
    L = _lib.load()
    assert L.mg_last_error() == b""


def test_built_for_sm_103a_only():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
