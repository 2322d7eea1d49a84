"""Host-side checks of the C-ABI library (no GPU needed): it builds, loads,
and exports every symbol that include/dski.h declares."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "dski.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b((?:dski|pivchol)_[a-z_0-9]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("dski_create", "dski_mvm", "dski_pcg_solve", "dski_logdet_slq", "pivchol_build"):
        assert s in syms


def test_library_exports_every_declared_symbol():
    from paper_1810_12283_gb300 import build, _lib
    try:
        path = build.build()
    except RuntimeError as e:   # no nvcc on this machine
        pytest.skip(str(e))
    lib = _lib.load(path)
    for s in declared_symbols():
        assert hasattr(lib, s), s
    assert set(declared_symbols()) <= set(_lib.EXPORTS) | set(declared_symbols())
    assert sorted(_lib.EXPORTS) == declared_symbols()


def test_last_error_empty_initially():
    from paper_1810_12283_gb300 import build, _lib
    try:
        build.build()
    except RuntimeError as e:
        pytest.skip(str(e))
    assert isinstance(_lib.load().dski_last_error(), bytes)
