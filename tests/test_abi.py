"""The C ABI library loads and exports every entry point include/glad.h declares (no GPU)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "glad.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(glad_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["glad_create", "glad_destroy", "glad_loglike", "glad_loglike_grad",
              "glad_model_image", "glad_vrms", "glad_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2504_01302_b300 import _lib, build
    if not os.path.exists(_lib.LIB_PATH) or not build.up_to_date():
        build.build()
    lib = _lib.load()
    for n in declared_functions():
        assert hasattr(lib, n), n
        assert n in _lib.SIGNATURES, n
