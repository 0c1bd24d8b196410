"""CPU oracle for the Huffman encoding pipeline (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it and it
never calls the CUDA library: the two share no code.

The arithmetic lives in ``huff_oracle.c`` (serial C, one function per stage
of the paper's pipeline, each citing the passage it restates); this module
only compiles it with the host C compiler and marshals numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "huff_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
MAX_LEN = 64

_lib = None


class OracleError(RuntimeError):
    pass


_ERRORS = {
    -1: "invalid argument",
    -2: "symbol >= nbins",
    -3: "symbol has no codeword",
    -4: "output capacity too small",
    -5: "histogram sum >= 2^32",
    -6: "undecodable stream",
}


def build(force: bool = False) -> str:
    """Compile huff_oracle.c into liboracle.so beside it (gcc, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _bind(lib: ctypes.CDLL) -> ctypes.CDLL:
    """Declares the C signatures on a loaded oracle library (the tests also
    bind builds of deliberately altered copies of the source through this)."""
    vp, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
    lib.oracle_histogram.argtypes = [vp, u64, i32, u32, vp]
    lib.oracle_lengths_two_queue.argtypes = [vp, u32, vp]
    lib.oracle_lengths_heap.argtypes = [vp, u32, vp]
    lib.oracle_canonical.argtypes = [vp, u32, vp, vp, vp, vp, vp, vp]
    lib.oracle_encode.argtypes = [vp, u64, i32, vp, vp, u32, i32, vp, u64, vp, vp]
    lib.oracle_encode_format.argtypes = [vp, u64, i32, vp, vp, u32, i32, i32, i32, vp, u64, vp, vp]
    lib.oracle_decode.argtypes = [vp, u64, u64, vp, vp, vp, vp, u32, i32, vp]
    for f in (lib.oracle_histogram, lib.oracle_lengths_two_queue, lib.oracle_lengths_heap,
              lib.oracle_canonical, lib.oracle_encode, lib.oracle_encode_format, lib.oracle_decode):
        f.restype = i32
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = _bind(ctypes.CDLL(_LIB))
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _check(rc: int) -> int:
    if rc < 0:
        raise OracleError(_ERRORS.get(rc, f"error {rc}"))
    return rc


def _width(sym: np.ndarray) -> int:
    if sym.dtype not in (np.uint8, np.uint16, np.uint32):
        raise TypeError(f"symbols must be uint8/uint16/uint32, got {sym.dtype}")
    return sym.dtype.itemsize


def histogram(sym: np.ndarray, nbins: int) -> np.ndarray:
    """Counts of each symbol (Sec. IV-A)."""
    sym = np.ascontiguousarray(sym)
    hist = np.zeros(nbins, dtype=np.uint32)
    _check(_load().oracle_histogram(_ptr(sym), sym.size, _width(sym), nbins, _ptr(hist)))
    return hist


def lengths(hist: np.ndarray, method: str = "two_queue") -> np.ndarray:
    """Optimal code lengths, leaf first on weight ties (Sec. IV-B1)."""
    hist = np.ascontiguousarray(hist, dtype=np.uint32)
    ln = np.zeros(hist.size, dtype=np.uint8)
    fn = _load().oracle_lengths_two_queue if method == "two_queue" else _load().oracle_lengths_heap
    _check(fn(_ptr(hist), hist.size, _ptr(ln)))
    return ln


def canonical(ln: np.ndarray) -> dict:
    """Canonical codewords and First/Entry decode tables from lengths (Sec. IV-B2)."""
    ln = np.ascontiguousarray(ln, dtype=np.uint8)
    nb = ln.size
    code = np.zeros(nb, dtype=np.uint64)
    first = np.zeros(MAX_LEN + 1, dtype=np.uint64)
    entry = np.zeros(MAX_LEN + 1, dtype=np.uint32)
    count = np.zeros(MAX_LEN + 1, dtype=np.uint32)
    sorted_syms = np.zeros(nb, dtype=np.uint32)
    nused = np.zeros(1, dtype=np.uint32)
    maxl = _check(_load().oracle_canonical(_ptr(ln), nb, _ptr(code), _ptr(first), _ptr(entry),
                                           _ptr(count), _ptr(sorted_syms), _ptr(nused)))
    u = int(nused[0])
    return dict(len=ln, code=code, first=first, entry=entry, count=count,
                sorted_syms=sorted_syms[:u].copy(), nused=u, max_len=maxl, nbins=nb)


def codebook(hist: np.ndarray) -> dict:
    """lengths() followed by canonical()."""
    return canonical(lengths(hist))


def encode(sym: np.ndarray, book: dict, chunk_log2: int = 10, capacity_words: int | None = None):
    """Dense MSB-first bitstream, chunk bit offsets and total bits (Sec. IV-C)."""
    sym = np.ascontiguousarray(sym)
    n = sym.size
    if capacity_words is None:
        capacity_words = (n * max(1, book["max_len"]) + 31) // 32
    out = np.zeros(max(1, capacity_words), dtype=np.uint32)
    nchunks = (n + (1 << chunk_log2) - 1) >> chunk_log2
    offs = np.zeros(nchunks + 1, dtype=np.uint64)
    total = np.zeros(1, dtype=np.uint64)
    _check(_load().oracle_encode(_ptr(sym), n, _width(sym), _ptr(book["code"]), _ptr(book["len"]),
                                 book["nbins"], chunk_log2, _ptr(out), capacity_words,
                                 _ptr(offs), _ptr(total)))
    tb = int(total[0])
    return out[:(tb + 31) // 32].copy(), offs, tb


UNIT_DTYPE = {8: np.uint8, 16: np.uint16, 32: np.uint32}


def encode_format(sym: np.ndarray, book: dict, chunk_log2: int = 10, word_bits: int = 32, aligned: bool = False):
    """The stream as W-bit typed units (Sec. IV-C typed cells), dense or with
    each chunk starting at a unit boundary (Sec. VI un-gathered chunks).
    Returns (units uintW[used], offsets uint64[nchunks+1], total_bits): dense
    offsets are bits, chunk-aligned offsets are units; total_bits counts the
    padding of the chunk-aligned form."""
    sym = np.ascontiguousarray(sym)
    n = sym.size
    W = int(word_bits)
    nchunks = (n + (1 << chunk_log2) - 1) >> chunk_log2
    cap_units = (n * max(1, book["max_len"]) + W - 1) // W + (nchunks if aligned else 0)
    out = np.zeros(max(1, cap_units), dtype=UNIT_DTYPE.get(W, np.uint32))
    offs = np.zeros(nchunks + 1, dtype=np.uint64)
    total = np.zeros(1, dtype=np.uint64)
    _check(_load().oracle_encode_format(_ptr(sym), n, _width(sym), _ptr(book["code"]), _ptr(book["len"]),
                                        book["nbins"], chunk_log2, W, 1 if aligned else 0, _ptr(out), cap_units,
                                        _ptr(offs), _ptr(total)))
    tb = int(total[0])
    return out[:(tb + W - 1) // W].copy(), offs, tb


def decode(stream: np.ndarray, total_bits: int, n: int, book: dict, width: int = 2) -> np.ndarray:
    """Treeless canonical decoding with First/Entry (Sec. IV-B2)."""
    stream = np.ascontiguousarray(stream, dtype=np.uint32)
    if stream.size == 0:
        stream = np.zeros(1, dtype=np.uint32)
    dt = {1: np.uint8, 2: np.uint16, 4: np.uint32}[width]
    out = np.zeros(n, dtype=dt)
    ss = book["sorted_syms"]
    if ss.size == 0:
        ss = np.zeros(1, dtype=np.uint32)
    _check(_load().oracle_decode(_ptr(stream), total_bits, n, _ptr(book["first"]), _ptr(book["entry"]),
                                 _ptr(book["count"]), _ptr(ss), book["max_len"], width, _ptr(out)))
    return out
