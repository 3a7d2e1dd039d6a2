"""The C-ABI library loads and exports every entry point include/mlblup.h
declares (no GPU needed: nothing is called that touches the device)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mlblup.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(mlb_[A-Za-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    import paper_1701_00285_gb300 as pkg
    so = os.path.join(ROOT, "paper_1701_00285_gb300", "libmlblup.so")
    if not os.path.exists(so):
        from paper_1701_00285_gb300.build import build
        build()
    return pkg.lib()


def test_every_declared_symbol_is_exported(lib):
    syms = declared_symbols()
    assert len(syms) >= 20
    for s in syms:
        assert hasattr(lib, s), s


def test_binding_covers_the_header():
    from paper_1701_00285_gb300 import binding
    assert set(declared_symbols()) == set(binding._SIGS)


def test_status_strings_and_default_opts(lib):
    from paper_1701_00285_gb300 import binding
    for s in range(9):
        assert lib.mlb_status_string(s)
    o = binding.Opts()
    lib.mlb_default_opts(o)
    assert o.leaf_size == 64 and o.precond == 1 and o.pcg_rtol == 1e-10 and o.precision == 0
