"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/trisplat.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "trisplat.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(tri_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_pipeline_and_serving_calls():
    names = declared_functions()
    for want in ("tri_preprocess", "tri_bin_sort", "tri_render_fwd", "tri_render_bwd", "tri_preprocess_bwd",
                 "tri_serve_create", "tri_serve_submit", "tri_serve_poll", "tri_serve_stats"):
        assert want in names
    assert len(names) >= 20


def test_library_exports_every_declared_symbol():
    from paper_2505_19175_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_product_path_fails_loudly_without_the_library(monkeypatch, tmp_path):
    import paper_2505_19175_gb300.native as N
    monkeypatch.setattr(N, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(N, "_lib", None)
    try:
        N.lib()
    except RuntimeError as e:
        assert "native library missing" in str(e)
    else:
        raise AssertionError("loading a missing library did not fail")


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2505_19175_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith(".py"):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, flags=re.M), f
