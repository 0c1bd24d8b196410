"""The multithreaded CPU baseline (the counterpart of the paper's OpenMP
histogram, codebook and encoder of Tables V and VI) equals the oracle bit
for bit: histogram, code lengths, codewords, stream, chunk offsets and bit
count, for every thread count, including chunk ranges that split 32-bit
words between threads, codewords longer than 32 bits, and the degenerate
inputs."""
import numpy as np
import pytest

import cpu_baseline as mt
import oracle
from paper_2010_10039_gb300 import synth

THREADS = [1, 2, 3, 7, 16]


def _same(sym, nbins, chunk_log2, threads):
    h = mt.histogram(sym, nbins, threads)
    want_h = oracle.histogram(sym, nbins)
    assert np.array_equal(h, want_h)
    b = mt.codebook(h, threads)
    want = oracle.codebook(want_h)
    assert np.array_equal(b["len"], want["len"])
    assert np.array_equal(b["code"], want["code"])
    assert b["max_len"] == want["max_len"]
    w, o, tb = mt.encode(sym, b, chunk_log2, threads)
    ww, wo, wtb = oracle.encode(sym, want, chunk_log2=chunk_log2)
    assert tb == wtb
    assert np.array_equal(w, ww[: (wtb + 31) // 32])
    assert np.array_equal(o, wo)


@pytest.mark.parametrize("threads", THREADS)
@pytest.mark.parametrize("chunk_log2", [4, 10, 17])
def test_u16_field_equals_oracle(threads, chunk_log2):
    _same(synth.laplace_field(400_009, seed=61), 1024, chunk_log2, threads)


@pytest.mark.parametrize("threads", [1, 4, 16])
def test_u8_and_u32_equal_oracle(threads):
    _same(synth.laplace_field(250_001, seed=62, b=5.0, K=256).astype(np.uint8), 256, 10, threads)
    _same(synth.zipf_field(200_003, 8192, seed=63), 8192, 10, threads)
    _same(synth.zipf_field(300_007, 65536, seed=64), 65536, 12, threads)


@pytest.mark.parametrize("threads", [1, 5, 16])
def test_codebook_large_alphabets_and_ties(threads):
    rng = np.random.default_rng(65)
    for nbins in (1024, 16384, 65536):
        h = rng.integers(0, 50, nbins).astype(np.uint32)          # many equal counts and unused symbols
        b = mt.codebook(h, threads)
        want = oracle.codebook(h)
        assert np.array_equal(b["len"], want["len"]) and np.array_equal(b["code"], want["code"])
    h = np.full(4096, 7, np.uint32)                                # all tied
    b = mt.codebook(h, threads)
    want = oracle.codebook(h)
    assert np.array_equal(b["len"], want["len"]) and np.array_equal(b["code"], want["code"])


@pytest.mark.parametrize("threads", [1, 3, 16])
def test_codewords_longer_than_32_bits(threads):
    """Fibonacci counts give a maximally skewed tree (lengths up to 44); the
    stream of a uniform draw over those symbols is full of >32-bit codes."""
    f = [1, 1]
    while sum(f) + f[-1] + f[-2] < (1 << 32) - 1:
        f.append(f[-1] + f[-2])
    h = np.array(f, np.uint32)
    b = mt.codebook(h, threads)
    want = oracle.codebook(h)
    assert want["max_len"] > 40
    assert np.array_equal(b["len"], want["len"]) and np.array_equal(b["code"], want["code"])
    sym = np.random.default_rng(66).integers(0, h.size, 100_003).astype(np.uint16)
    w, o, tb = mt.encode(sym, b, 6, threads)
    ww, wo, wtb = oracle.encode(sym, want, chunk_log2=6)
    assert tb == wtb and np.array_equal(w, ww[: (wtb + 31) // 32]) and np.array_equal(o, wo)


@pytest.mark.parametrize("threads", [1, 16])
def test_degenerate_inputs(threads):
    for sym, nbins in ((np.zeros(0, np.uint16), 1024), (np.array([5], np.uint16), 1024),
                       (np.full(70_001, 9, np.uint16), 1024), (np.array([0, 1] * 33, np.uint8), 2)):
        h = mt.histogram(sym, nbins, threads)
        assert np.array_equal(h, oracle.histogram(sym, nbins))
        b = mt.codebook(h, threads)
        want = oracle.codebook(h)
        assert np.array_equal(b["len"], want["len"]) and np.array_equal(b["code"], want["code"])
        if sym.size:
            w, o, tb = mt.encode(sym, b, 3, threads)
            ww, wo, wtb = oracle.encode(sym, want, chunk_log2=3)
            assert tb == wtb and np.array_equal(w, ww[: (wtb + 31) // 32]) and np.array_equal(o, wo)
        else:
            w, o, tb = mt.encode(sym, b, 10, threads)
            assert tb == 0 and w.size == 0 and o.tolist() == [0]


def test_errors_are_reported():
    sym = np.array([1, 2, 1030], np.uint16)
    with pytest.raises(mt.CpuMtError, match="symbol >= nbins"):
        mt.histogram(sym, 1024, 4)
    b = mt.codebook(np.array([3, 0, 1], np.uint32), 2)
    with pytest.raises(mt.CpuMtError, match="no codeword"):
        mt.encode(np.array([0, 1], np.uint8), b, 4, 2)
    with pytest.raises(mt.CpuMtError, match="2\\^32"):
        mt.codebook(np.array([1 << 31, 1 << 31], np.uint32), 2)


def test_scaling_rows_have_the_table_vi_columns():
    rows = mt.scaling(synth.laplace_field(300_000, seed=67), 1024, [1, 2], reps=1)
    assert [r["threads"] for r in rows] == [1, 2]
    for r in rows:
        for k in ("histogram_GBps", "codebook_ms", "encode_GBps", "hist_codebook_encode_GBps",
                  "histogram_efficiency", "encode_efficiency"):
            assert r[k] > 0
