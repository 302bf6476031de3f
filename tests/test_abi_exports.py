"""The C-ABI library loads and exports every symbol include/*.h declares.

CPU-only: no call that needs a GPU is made here (only the pure host helpers).
"""
import glob
import os
import re

import pytest

import paper_1708_09746_gb300 as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names += re.findall(r"GF2X_API\s+[\w\s\*]*?\b(gf2x_\w+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1708_09746_gb300 import build
    build.build()
    return G.load()


def test_header_declares_entry_points():
    names = _declared()
    assert "gf2x_mul" in names and "gf2x_plan_execute" in names
    assert len(names) >= 15


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_symbol():
    for name in _declared():
        assert callable(getattr(G, name)), name


def test_host_helpers(lib):
    assert G.gf2x_out_words(0, 5) == 0
    assert G.gf2x_out_words(64, 64) == 2
    assert G.gf2x_out_words(1, 1) == 1
    assert G.gf2x_out_words(1 << 28, 1 << 28) == (1 << 23)
    assert G.gf2x_fft_points(1 << 28, 1 << 28) == 1 << 23
    assert G.gf2x_fft_points(1 << 28, 1 << 16) == 1 << 23
    assert G.gf2x_fft_points(1 << 20, 1 << 20) == 1 << 15
    assert G.gf2x_fft_points(64, 64) == 2
    assert "invalid" in G.gf2x_strerror(-1)
    assert G.gf2x_strerror(12345) == "unknown status"
