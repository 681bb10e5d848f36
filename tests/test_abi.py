"""The C-ABI library loads without a GPU and exports every symbol that
include/escher.h declares (no compute call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "escher.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(esc_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2512_21009_gb300 import build as b
    b.build()
    from paper_2512_21009_gb300 import escher
    return escher.load()


def test_header_declares_the_binding_names():
    from paper_2512_21009_gb300 import escher
    assert _declared() == sorted(escher.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_version_string(lib):
    from paper_2512_21009_gb300 import escher
    assert "sm_103a" in escher.esc_version()


def test_library_does_not_link_the_oracle():
    import subprocess
    out = subprocess.run(["nm", "-D", os.path.join(ROOT, "paper_2512_21009_gb300", "libescher.so")],
                         capture_output=True, text=True).stdout
    assert "orc_" not in out


def test_product_sources_do_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2512_21009_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "escher_oracle" not in text, f


def test_missing_library_fails_loudly(tmp_path):
    from paper_2512_21009_gb300 import escher
    saved = escher._lib
    escher._lib = None
    try:
        with pytest.raises(ImportError):
            escher.load(str(tmp_path / "nope.so"))
    finally:
        escher._lib = saved
