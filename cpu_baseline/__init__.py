"""Multithreaded CPU Huffman encoder: the CPU comparison of the paper's
Sec. VI (Table V, multi-thread codebook construction; Table VI, multi-thread
histogram and encoder scaled over cores), on POSIX threads.

A reported baseline for ``bench.py``: it is neither the product (which runs
on the GPU and never calls this) nor the oracle (which it shares no code
with).  Its outputs equal the oracle's bit for bit, which the CPU test suite
checks.  The C source is ``huff_cpu_mt.c``; this module compiles it with the
host C compiler and marshals numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "huff_cpu_mt.c")
_LIB = os.path.join(_HERE, "libhuffcpumt.so")
_lib = None

ERRORS = {-1: "invalid argument", -2: "symbol >= nbins", -3: "symbol has no codeword",
          -4: "output capacity too small", -5: "histogram sum >= 2^32", -7: "thread creation failed"}


class CpuMtError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile huff_cpu_mt.c into libhuffcpumt.so beside it (gcc -O3)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-std=c11", "-pthread", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        vp, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
        L.mt_histogram.argtypes = [vp, u64, i32, u32, vp, i32]
        L.mt_codebook.argtypes = [vp, u32, vp, vp, i32]
        L.mt_encode.argtypes = [vp, u64, i32, vp, vp, u32, i32, vp, u64, vp, vp, i32]
        for f in (L.mt_histogram, L.mt_codebook, L.mt_encode):
            f.restype = i32
        _lib = L
    return _lib


def _check(rc: int, what: str) -> int:
    if rc < 0:
        raise CpuMtError(f"{what}: {ERRORS.get(rc, rc)}")
    return rc


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def default_threads() -> int:
    return max(1, min(256, os.cpu_count() or 1))


def histogram(sym: np.ndarray, nbins: int, threads: int | None = None) -> np.ndarray:
    sym = np.ascontiguousarray(sym)
    h = np.zeros(nbins, np.uint32)
    _check(lib().mt_histogram(_p(sym), sym.size, sym.dtype.itemsize, nbins, _p(h), threads or default_threads()),
           "mt_histogram")
    return h


def codebook(hist: np.ndarray, threads: int | None = None) -> dict:
    """Canonical codebook of a histogram: {'len': uint8[nbins], 'code': uint64[nbins], 'max_len'}."""
    hist = np.ascontiguousarray(hist, dtype=np.uint32)
    ln = np.zeros(hist.size, np.uint8)
    code = np.zeros(hist.size, np.uint64)
    maxl = _check(lib().mt_codebook(_p(hist), hist.size, _p(ln), _p(code), threads or default_threads()),
                  "mt_codebook")
    return {"len": ln, "code": code, "max_len": maxl}


def encode(sym: np.ndarray, book: dict, chunk_log2: int = 10, threads: int | None = None):
    """(words uint32[ceil(bits/32)], chunk_bit_offset uint64[nchunks+1], total_bits)."""
    sym = np.ascontiguousarray(sym)
    ln = np.ascontiguousarray(book["len"], dtype=np.uint8)
    code = np.ascontiguousarray(book["code"], dtype=np.uint64)
    n = sym.size
    nch = (n + (1 << chunk_log2) - 1) >> chunk_log2
    maxl = int(ln.max()) if ln.size else 0
    cap = max(1, (n * maxl + 31) // 32)
    out = np.empty(cap, np.uint32)
    offs = np.zeros(nch + 1, np.uint64)
    tb = ctypes.c_uint64(0)
    _check(lib().mt_encode(_p(sym), n, sym.dtype.itemsize, _p(code), _p(ln), ln.size, chunk_log2, _p(out), cap,
                           _p(offs), ctypes.byref(tb), threads or default_threads()), "mt_encode")
    bits = tb.value
    return out[: (bits + 31) // 32].copy(), offs, bits


def scaling(sym: np.ndarray, nbins: int, thread_counts, chunk_log2: int = 10, reps: int = 2) -> list[dict]:
    """Table VI's measurement on `sym`: for each thread count, the best of
    `reps` runs of histogram (GB/s of input), codebook (ms), encode (GB/s of
    input) and the three in a row (GB/s of input)."""
    sym = np.ascontiguousarray(sym)
    nbytes = sym.nbytes
    rows = []
    for T in thread_counts:
        th, tc, te = [], [], []
        for _ in range(reps):
            t0 = time.perf_counter()
            h = histogram(sym, nbins, T)
            t1 = time.perf_counter()
            b = codebook(h, T)
            t2 = time.perf_counter()
            encode(sym, b, chunk_log2, T)
            t3 = time.perf_counter()
            th.append(t1 - t0)
            tc.append(t2 - t1)
            te.append(t3 - t2)
        tot = [a + b + c for a, b, c in zip(th, tc, te)]
        rows.append({"threads": T, "histogram_GBps": round(nbytes / min(th) / 1e9, 3),
                     "codebook_ms": round(min(tc) * 1e3, 3), "encode_GBps": round(nbytes / min(te) / 1e9, 3),
                     "hist_codebook_encode_GBps": round(nbytes / min(tot) / 1e9, 3)})
    base = rows[0]
    for r in rows:
        k = r["threads"] / base["threads"]
        r["histogram_efficiency"] = round(r["histogram_GBps"] / base["histogram_GBps"] / k, 3)
        r["encode_efficiency"] = round(r["encode_GBps"] / base["encode_GBps"] / k, 3)
    return rows
