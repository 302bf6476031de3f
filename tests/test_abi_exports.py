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


def test_chunking_host_helper(lib):
    # balanced and mildly unequal products run as one transform
    assert G.gf2x_chunking(1 << 28, 1 << 28) == (0, 0, 0)
    assert G.gf2x_chunking(64 * 2048, 64 * 513) == (0, 0, 0)   # 2 chunks only
    # the c1 unequal workload: chunks of 2^10 words, 2^11-point transforms
    assert G.gf2x_chunking(1 << 28, 1 << 16) == (1024, 4096, 2048)
    assert G.gf2x_chunking(1 << 16, 1 << 28) == (1024, 4096, 2048)
    # short operand between 17 and 511 words: chunks of 512 words
    assert G.gf2x_chunking(64 * 5000 + 3, 64 * 20) == (512, 10, 1024)
    # at most 2^15 chunks: the chunk grows with the long operand
    L, C, N = G.gf2x_chunking(1 << 33, 64 * 17)
    assert C <= 1 << 15 and L * C >= (1 << 33) // 64 and L == 1 << 12 and N == 1 << 13
    assert G.gf2x_chunking(0, 5) == (0, 0, 0)
    # a short operand of at most 16 words is multiplied directly (no chunks)
    assert G.gf2x_chunking(64 * 5000 + 3, 1) == (0, 0, 0)
    assert G.gf2x_chunking(1 << 33, 64 * 16) == (0, 0, 0)


def test_product_path_host_helper(lib):
    assert G.gf2x_product_path(1 << 28, 1 << 28) == (0, 1 << 22, 1 << 22)
    assert G.gf2x_product_path(1 << 28, 1 << 16)[0] == 1
    assert G.gf2x_product_path(1 << 28, 64 * 16)[0] == 2
    assert G.gf2x_product_path(64 * 16, 1 << 28)[0] == 2
    assert G.gf2x_product_path(64 * 17, 64 * 17)[0] == 0
    # one word past half the transform: the main product keeps 2^22 + 2^22
    # words (a half-length transform), one word of a is a tail
    assert G.gf2x_product_path((1 << 28) + 64, (1 << 28) + 64) == (3, 1 << 22, (1 << 22) + 1)
    # 17 words past: no split
    n = 64 * ((1 << 14) + 9)
    assert G.gf2x_product_path(n, n)[0] == 0
