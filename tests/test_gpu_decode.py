"""GPU canonical decoder (Sec. IV-B2): streams written by the GPU encoder (and
checked against the oracle's) decode back to the input symbols, through the
table path, the long-code search path, the vector and the scalar stores;
corrupted streams and offsets report an error and write nothing out of
range."""
import numpy as np
import pytest

import oracle
from paper_2010_10039_gb300 import synth
from gpu_util import Run, u32

pytestmark = pytest.mark.gpu

TORCH_DT = {1: "uint8", 2: "int16", 4: "int32"}
NP_DT = {1: np.uint8, 2: np.uint16, 4: np.uint32}


def _decode(r, n, width, chunk_log2, out_offset=0, offs=None, stream=None, total_bits=None, nbins=None):
    import torch
    import paper_2010_10039_gb300 as huff
    tb = int(r.total.item()) if total_bits is None else total_bits
    dt = getattr(torch, TORCH_DT[width])
    big = torch.full((n + out_offset + 1,), 0x55, dtype=dt, device="cuda")
    out = big[out_offset:out_offset + n]
    huff.huff_decode(r.out if stream is None else stream, tb, r.offs if offs is None else offs, chunk_log2, n,
                     width, r.book, r.nbins if nbins is None else nbins, out, r.ws)
    got = out.cpu().numpy().view(NP_DT[width])
    guard = big[out_offset + n:].cpu().numpy().view(NP_DT[width])
    return got, guard


def _round_trip(sym, nbins, chunk_log2=10, out_offset=0):
    r = Run(sym, nbins, chunk_log2).all()
    assert r.status() == 0
    got, guard = _decode(r, sym.size, sym.dtype.itemsize, chunk_log2, out_offset)
    assert r.status() == 0
    assert np.array_equal(got, sym)
    assert (guard == 0x55).all()
    return r


@pytest.mark.parametrize("chunk_log2", [5, 8, 10, 12])
@pytest.mark.parametrize("n", [1, 31, 1000, 300_017])
def test_round_trip_u16_chunks_and_ragged_tails(chunk_log2, n):
    _round_trip(synth.laplace_field(n, seed=21), 1024, chunk_log2)


@pytest.mark.parametrize("out_offset", [1, 3, 8])
def test_round_trip_unaligned_output(out_offset):
    """An output that is not 16-byte aligned takes the scalar stores."""
    _round_trip(synth.laplace_field(200_003, seed=22), 1024, 10, out_offset)


def test_round_trip_u8_zipf():
    sym = synth.draw(5, 7, 400_000, synth.cdf_table(synth.zipf_pmf(256, 1.2)), 1)
    _round_trip(sym, 256, 10)


@pytest.mark.parametrize("K", [8192, 65536])
def test_round_trip_u32_large_alphabet(K):
    """Codes up to 17 / 21 bits: everything past 12 bits takes the search path."""
    sym = synth.zipf_field(2_000_000, K, seed=3)
    r = _round_trip(sym, K, 10)
    assert r.book_np()["max_len"] > 12


def test_round_trip_long_codewords():
    """Fibonacci counts give codes up to 44 bits (longer than the 32-bit refill)."""
    import torch
    fib = [1, 1]
    while len(fib) < 45:
        fib.append(fib[-1] + fib[-2])
    h = np.array(fib, dtype=np.uint32)
    rng = np.random.default_rng(6)
    sym = np.concatenate([np.arange(45, dtype=np.uint32), rng.integers(0, 45, size=60_000).astype(np.uint32)])
    r = Run(sym, 45)
    r.codebook(torch.from_numpy(h.view(np.int32)).cuda()).encode()
    assert r.status() == 0
    assert r.book_np()["max_len"] == 44
    got, _ = _decode(r, sym.size, 4, 10)
    assert r.status() == 0
    assert np.array_equal(got, sym)


def test_round_trip_single_symbol():
    _round_trip(np.full(5000, 9, dtype=np.uint16), 1024, 10)


def test_matches_oracle_decode():
    """The oracle's decoder and the GPU's agree on the same stream."""
    sym = synth.gaussian_field(1 << 18, seed=0)
    r = Run(sym, 1024).all()
    words, tb = r.stream_np()
    want = oracle.decode(words, tb, sym.size, r.book_np(), 2)
    got, _ = _decode(r, sym.size, 2, 10)
    assert np.array_equal(got, want) and np.array_equal(got, sym)


def test_hpc_field_full_size():
    sym = synth.laplace_field(512 ** 3, seed=1)
    _round_trip(sym, 1024, 10)


def test_corrupt_offset_reports_error():
    import torch
    sym = synth.laplace_field(100_000, seed=23)
    r = Run(sym, 1024).all()
    offs = r.offs.clone()
    offs[7] += 1
    _decode(r, sym.size, 2, 10, offs=offs)
    assert r.status() != 0


def test_corrupt_stream_reports_error():
    """A one-symbol field has the single code 0: a word of ones in its stream
    is an invalid code, so the error is certain."""
    sym = np.full(100_000, 9, dtype=np.uint16)
    r = Run(sym, 1024).all()
    bad = r.out.clone()
    bad[100] = -1
    got, guard = _decode(r, sym.size, 2, 10, stream=bad)
    assert r.status() != 0
    assert (guard == 0x55).all()


def test_corrupt_stream_detected_or_different():
    """A complete code can resynchronise after a corrupted word, so the chunk
    may still end at its offset: then the symbols differ instead."""
    sym = synth.laplace_field(100_000, seed=24)
    r = Run(sym, 1024).all()
    bad = r.out.clone()
    bad[100] = ~bad[100]
    got, guard = _decode(r, sym.size, 2, 10, stream=bad)
    assert r.status() != 0 or not np.array_equal(got, sym)
    assert (guard == 0x55).all()


def test_codebook_mismatch_reports_error():
    sym = synth.laplace_field(10_000, seed=25)
    r = Run(sym, 1024).all()
    _decode(r, sym.size, 2, 10, nbins=2048)
    assert r.status() != 0
