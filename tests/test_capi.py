"""The C ABI library builds, loads, and exports every entry point include/bqc.h declares."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "bqc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bqc_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2502_17963_gb300 import _build
    _build.build()
    import paper_2502_17963_gb300 as bqc
    return bqc.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header(lib):
    import paper_2502_17963_gb300 as bqc
    assert sorted(bqc.exported_symbols()) == _declared()


def test_status_strings(lib):
    assert lib.bqc_strerror(0) == b"ok"
    assert b"HBM" in lib.bqc_strerror(-3)
    assert lib.bqc_strerror(12345) == b"unknown status"


def test_footprint_is_monotone(lib):
    import paper_2502_17963_gb300 as bqc
    for prec in range(4):
        a = lib.bqc_serve_footprint(100, 300, 20, prec)
        b = lib.bqc_serve_footprint(200, 600, 40, prec)
        assert b >= a > 0
    # FP16 split shadows take half the bytes of the TF32 ones; FP64 needs none
    f64, tf, f16 = (lib.bqc_serve_footprint(800, 2400, 160, p) for p in (0, 2, 3))
    assert f64 < f16 < tf
    assert lib.bqc_serve_footprint(100, 300, 20, 7) == 0
