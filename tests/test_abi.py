"""CPU-side checks of the C ABI: the library builds, loads and exports every declared symbol."""
import os
import re

import pytest

import paper_2511_05958_b300 as mt4g

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(mt4g_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_binding_names():
    assert set(declared_symbols()) == set(mt4g.exported_symbols())


def test_library_exports_every_declared_symbol():
    L = mt4g.load_library()
    for name in declared_symbols():
        assert hasattr(L, name), name


def test_no_cpu_fallback_without_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(Exception):
        mt4g.Engine(0)


def test_critical_value_matches_oracle():
    """Eq. 1 as computed by the library (host code) against the oracle's reading of it."""
    import oracle
    for alpha in (0.1, 0.05, 1e-3, 1e-6):
        for n, m in ((10, 20), (128, 384), (65536, 4096)):
            assert abs(mt4g.critical_value(alpha, n, m) - oracle.critical_value(alpha, n, m)) < 1e-15
    assert mt4g.critical_value(1.5, 3, 3) == -1.0 and mt4g.critical_value(0.05, 0, 3) == -1.0
