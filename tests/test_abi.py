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
    4.1 -> 2, 8.3 -> 1, 17 -> 0 (clamped to [0, 5])."""
    import paper_2010_10039_gb300 as huff
    assert huff.huff_reduce_factor(1.02717, 32) == 4
    assert huff.huff_reduce_factor(2.73, 32) == 3
    assert huff.huff_reduce_factor(3.63, 32) == 3
    assert huff.huff_reduce_factor(4.14, 32) == 2
    assert huff.huff_reduce_factor(5.2, 32) == 2
    assert huff.huff_reduce_factor(8.3, 32) == 1
    assert huff.huff_reduce_factor(17.0, 32) == 0
    assert huff.huff_reduce_factor(40.0, 32) == 0
    assert huff.huff_reduce_factor(0.3, 32) == 5
    assert huff.huff_reduce_factor(1.5, 16) == 3


def test_workspace_grows_with_n(lib):
    import paper_2010_10039_gb300 as huff
    a = huff.huff_workspace_bytes(1 << 20, 1024)
    b = huff.huff_workspace_bytes(1 << 26, 1024)
    assert 256 < a < b
    assert huff.huff_workspace_bytes(1000, 65536) > huff.huff_workspace_bytes(1000, 1024)


def test_default_params(lib):
    import paper_2010_10039_gb300 as huff
    p = huff.huff_default_params()
    assert (p.chunk_log2, p.reduce_log2, p.block_threads, p.merge, p.word_bits, p.layout) == (10, -1, 0, 0, 32, 0)


def test_misaligned_typed_pointers_are_rejected_on_the_host(lib):
    """A u16/u32 symbol pointer that is not element aligned returns
    HUFF_ERR_INVALID_ARG before any device work (no GPU needed)."""
    import paper_2010_10039_gb300 as huff
    L = huff.lib()
    bad16 = 0x100001          # odd: never dereferenced
    assert L.huff_histogram(bad16, 100, huff.HUFF_U16, 1024, 0x200000, 0x300000, None) == 1
    assert L.huff_histogram(0x100002, 100, huff.HUFF_U32, 1024, 0x200000, 0x300000, None) == 1
    p = huff.huff_default_params()
    assert L.huff_encode(bad16, 100, huff.HUFF_U16, 0x400000, 1024, ctypes.byref(p), 0x500000, 100,
                         0x600000, 0x700000, 0x300000, None) == 1


def test_batch_plan_create_rejects_bad_fields_on_the_host(lib):
    import paper_2010_10039_gb300 as huff
    L = huff.lib()
    out = ctypes.c_void_p()
    cfg = huff.huff_batch_cfg()
    L.huff_batch_default_cfg(ctypes.byref(cfg))
    assert (cfg.autotune, cfg.reduce_log2, cfg.max_subtiles, cfg.ctas_per_sm, cfg.encode_form) == (0, -1, 0, 0, 0)
    arr = (huff.huff_field * 1)()
    good = dict(d_sym=0x100000, n=1000, dtype=huff.HUFF_U16, nbins=1024, chunk_log2=10, d_out=0x200000,
                out_capacity_words=1000, d_chunk_bit_offset=0x300000, d_total_bits=0x400000)
    cases = [dict(nbins=0), dict(nbins=70000), dict(dtype=3), dict(dtype=huff.HUFF_U8, nbins=300),
             dict(d_sym=0x100001), dict(d_total_bits=0x400004), dict(chunk_log2=2), dict(chunk_log2=31),
             dict(n=1 << 32), dict(d_out=0)]
    for c in cases:
        f = dict(good)
        f.update(c)
        for k, v in f.items():
            setattr(arr[0], k, v)
        assert L.huff_batch_plan_create(arr, 1, ctypes.byref(cfg), None, ctypes.byref(out)) == 1, c
        assert not out.value
    assert L.huff_batch_plan_create(arr, 0, ctypes.byref(cfg), None, ctypes.byref(out)) == 1
    for k, v in good.items():
        setattr(arr[0], k, v)
    for bad_cfg in (huff.huff_batch_cfg(0, 7, 0, 0), huff.huff_batch_cfg(0, -1, 0, 0, 3)):
        assert L.huff_batch_plan_create(arr, 1, ctypes.byref(bad_cfg), None, ctypes.byref(out)) == 1


def test_binding_structs_match_the_header(tmp_path):
    """Every struct the Python binding declares has the size and field
    offsets the C header gives it (compiled here with gcc), so the binding
    and libhuff.so agree on the records they exchange."""
    import shutil
    import subprocess
    import paper_2010_10039_gb300 as huff
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [huff.huff_params, huff.huff_field, huff.huff_batch_cfg, huff.huff_batch_info,
               huff.huff_serve_cfg, huff.huff_request, huff.huff_result, huff.huff_serve_stats]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "huff.h"', "int main(void) {"]
    for st in structs:
        name = st.__name__
        lines.append(f'    printf("{name} %zu\\n", sizeof({name}));')
        for field, _ in st._fields_:
            lines.append(f'    printf("{name}.{field} %zu\\n", offsetof({name}, {field}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    include = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-std=c11", "-I", include, str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                       text=True).stdout.splitlines())
    for st in structs:
        name = st.__name__
        assert int(got[name]) == ctypes.sizeof(st), name
        for field, _ in st._fields_:
            assert int(got[f"{name}.{field}"]) == getattr(st, field).offset, f"{name}.{field}"
