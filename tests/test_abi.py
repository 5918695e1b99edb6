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


def test_plan_struct_matches_the_header_layout_and_flattens_relax():
    """he_cutmax_plan as the binding packs it: the header's fields in order,
    and `relax` flattened iteration by iteration (k[t] constants each, none
    for a learned iteration, 3/2 for an iteration the plan leaves plain)."""
    import numpy as np
    from paper_2509_08383_gb300 import he
    from paper_2509_08383_gb300 import plan as P
    src = open(HEADER).read()
    body = src[src.index("typedef struct {\n    uint32_t n, packing, T;"):src.index("} he_cutmax_plan;")]
    fields = re.findall(r"([A-Za-z_0-9]+)(?:,|;)", re.sub(r"/\*.*?\*/", "", body, flags=re.S))
    assert [f[0] for f in he.CPlan._fields_] == fields
    pl = P.CutMaxPlan(n=1024, slots=1024, packing="replicate", T=3, p=[3, 3, 3], c=[5.0] * 3, k=[2, 0, 3],
                      kappa=[1.0] * 3, y0=[1.0] * 3, d=2, kappa_f=1.0, lq=[[0, 0, 0], [1.0, 2.0, 3.0], [0, 0, 0]],
                      relax=[[1.9, 1.5], [], None])
    s, keep = he.plan_struct(pl)
    assert np.allclose([s.relax[i] for i in range(5)], [1.9, 1.5, 1.5, 1.5, 1.5])
    assert [s.learned[i] for i in range(9)] == [0, 0, 0, 1.0, 2.0, 3.0, 0, 0, 0]
    s2, _ = he.plan_struct(P.CutMaxPlan(**{**pl.to_dict(), "relax": None}))
    assert not s2.relax
    with pytest.raises(ValueError):
        he.plan_struct(P.CutMaxPlan(**{**pl.to_dict(), "relax": [[1.9], [], None]}))
