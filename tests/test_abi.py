"""The C-ABI library builds, loads without a GPU and exports every function
declared in include/*.h; host-only helpers behave as documented."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(huff_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2010_10039_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_headers_declare_functions():
    assert "huff_encode" in _declared() and "huff_build_codebook" in _declared()


@pytest.mark.parametrize("name", _declared())
def test_symbol_exported(lib, name):
    assert hasattr(lib, name), f"{name} declared but not exported"


def test_codebook_layout_sizes(lib):
    import paper_2010_10039_gb300 as huff
    assert huff.huff_codebook_bytes(1024) == huff.CODEBOOK_HEADER_BYTES + 12 * 1024
    assert huff.huff_max_output_words(100, 7) == (700 + 31) // 32


def test_reduce_factor_rule(lib):
    """Sec. IV-C: floor(log2 beta) + r + 1 = log2(32): beta 1.03 -> 4, 2.73 -> 3,
    4.1 -> 2, 8.3 -> 1 (clamped to [1, 5])."""
    import paper_2010_10039_gb300 as huff
    assert huff.huff_reduce_factor(1.02717, 32) == 4
    assert huff.huff_reduce_factor(2.73, 32) == 3
    assert huff.huff_reduce_factor(3.63, 32) == 3
    assert huff.huff_reduce_factor(4.14, 32) == 2
    assert huff.huff_reduce_factor(5.2, 32) == 2
    assert huff.huff_reduce_factor(8.3, 32) == 1
    assert huff.huff_reduce_factor(0.3, 32) == 5


def test_workspace_grows_with_n(lib):
    import paper_2010_10039_gb300 as huff
    a = huff.huff_workspace_bytes(1 << 20, 1024)
    b = huff.huff_workspace_bytes(1 << 26, 1024)
    assert 256 < a < b
    assert huff.huff_workspace_bytes(1000, 65536) > huff.huff_workspace_bytes(1000, 1024)


def test_default_params(lib):
    import paper_2010_10039_gb300 as huff
    p = huff.huff_default_params()
    assert (p.chunk_log2, p.reduce_log2, p.block_threads, p.merge) == (10, -1, 0, 0)
