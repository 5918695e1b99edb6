"""The C-ABI library loads here (no GPU) and exports every declared entry point."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "he_cutmax.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*([a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while")))


def test_header_declares_core_calls():
    names = declared_functions()
    for n in ["he_ctx_create", "he_encrypt", "he_decrypt", "cutmax", "nucleus_sample", "he_keyswitch_raw",
              "he_ntt_device", "he_rotsum"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2509_08383_gb300 import build
    path = build.build_library()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2509_08383_gb300 import he
    monkeypatch.setattr(he, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(he, "_lib", None)
    with pytest.raises(RuntimeError):
        he.lib()
