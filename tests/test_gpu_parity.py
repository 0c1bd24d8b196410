"""GPU path vs CPU oracle, element by element (integer work: bit-exact).

Every test calls the CUDA library through its C-ABI (Python binding) and
compares with the oracle on the same seeded inputs."""
import numpy as np
import pytest

import oracle
from paper_2010_10039_gb300 import synth
from gpu_util import Run, to_dev, u32, u64

pytestmark = pytest.mark.gpu


def _cmp_book(got, want, hist=None):
    assert got["status"] == 0
    assert got["max_len"] == want["max_len"]
    assert got["nused"] == want["nused"]
    assert np.array_equal(got["len"], want["len"]), "lengths"
    assert np.array_equal(got["code"], want["code"]), "codes"
    assert np.array_equal(got["count"], want["count"])
    assert np.array_equal(got["entry"], want["entry"])
    ml = want["max_len"]
    assert np.array_equal(got["first"][1:ml + 1], want["first"][1:ml + 1])
    assert np.array_equal(got["sorted_syms"], want["sorted_syms"])
    if hist is not None:
        assert got["nsymbols"] == int(hist.astype(np.int64).sum())
        assert got["total_bits"] == int((hist.astype(np.int64) * want["len"]).sum())


def _full_check(sym_np, nbins, chunk_log2=10, offset_elems=0, params=None):
    r = Run(sym_np, nbins, chunk_log2, offset_elems, params).all()
    assert r.status() == 0
    h = oracle.histogram(sym_np, nbins)
    assert np.array_equal(r.hist_np(), h)
    want = oracle.codebook(h)
    _cmp_book(r.book_np(), want, h)
    words, offs, tb = oracle.encode(sym_np, want, chunk_log2=chunk_log2)
    got_words, got_tb = r.stream_np()
    assert got_tb == tb
    assert np.array_equal(got_words, words)
    assert np.array_equal(r.offs_np(), offs)
    return r, want, words, tb


def test_plain_pipeline_small_config():
    """1,048,576 u16 symbols, Gaussian sigma=8 over 1024 bins, seed 0: every
    output bit-exact, and the stream decodes back to the input."""
    sym = synth.gaussian_field(1 << 20, seed=0)
    r, want, words, tb = _full_check(sym, 1024)
    assert np.array_equal(oracle.decode(words, tb, sym.size, want, width=2), sym)


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 1023, 1024, 1025, 2047, 2048, 2049, 4095, 4096, 4097,
                               8191, 8192, 8193, 12289, 65536 * 3 + 7])
@pytest.mark.parametrize("width", [1, 2, 4])
def test_sizes_and_ragged_tails(n, width):
    rng = np.random.default_rng(n * 3 + width)
    nb = {1: 256, 2: 1024, 4: 1024}[width]
    p = synth.laplace_pmf(nb, nb // 2, 3.0)
    sym = rng.choice(nb, size=n, p=p).astype({1: np.uint8, 2: np.uint16, 4: np.uint32}[width])
    _full_check(sym, nb)


@pytest.mark.parametrize("offset", [1, 3, 7])
@pytest.mark.parametrize("width", [1, 2])
def test_unaligned_input(offset, width):
    sym = synth.laplace_field(100_003, seed=9).astype(np.uint16)
    if width == 1:
        sym = (sym & 0xFF).astype(np.uint8)
    _full_check(sym, 256 if width == 1 else 1024, offset_elems=offset)


@pytest.mark.parametrize("chunk_log2", [4, 5, 9, 10, 12, 16, 20])
def test_chunk_sizes(chunk_log2):
    sym = synth.laplace_field(300_001, seed=2)
    _full_check(sym, 1024, chunk_log2=chunk_log2)


@pytest.mark.parametrize("r", [0, 1, 2, 3])
@pytest.mark.parametrize("b", [0.3, 2.0, 40.0])
def test_reduce_factors_give_identical_streams(r, b):
    """The reduction factor r (2^r codewords merged per register) is a
    performance knob of Sec. IV-C only: every r gives the same stream."""
    sym = synth.laplace_field(200_003, seed=21, b=b)
    _full_check(sym, 1024, params={"reduce_log2": r})


@pytest.mark.parametrize("r", [0, 2, 3, 4])
def test_reduce_factors_u8(r):
    sym = (synth.laplace_field(150_001, seed=22, b=5.0, K=256)).astype(np.uint8)
    _full_check(sym, 256, params={"reduce_log2": r})


@pytest.mark.parametrize("r", [0, 1, 2])
def test_reduce_factors_u32(r):
    sym = synth.zipf_field(120_001, 8192, seed=23, s=0.9)
    _full_check(sym, 8192, params={"reduce_log2": r})


def test_empty_input():
    import torch
    import paper_2010_10039_gb300 as huff
    r = Run(np.zeros(0, np.uint16), 1024)
    r.histogram()
    assert (r.hist_np() == 0).all()
    r.codebook()
    b = r.book_np()
    assert b["max_len"] == 0 and b["nused"] == 0
    r.encode()
    assert r.status() == 0
    assert int(r.total.item()) == 0 and int(r.offs[0].item()) == 0


def _hist_cases():
    rng = np.random.default_rng(1234)
    cases = []
    for nb in (1, 2, 3, 17, 256, 1024, 4096, 8192, 65536):
        cases.append((f"uniform{nb}", rng.integers(1, 1000, size=nb).astype(np.uint32)))
        cases.append((f"ties{nb}", rng.integers(0, 4, size=nb).astype(np.uint32)))
        cases.append((f"pow2{nb}", (1 << rng.integers(0, 14, size=nb)).astype(np.uint32)))
        r = np.arange(1, nb + 1, dtype=np.float64)
        z = np.maximum(1, np.floor(3e6 * r ** -1.1)).astype(np.uint32)
        cases.append((f"zipf{nb}", z[rng.permutation(nb)]))
        cases.append((f"equal{nb}", np.full(nb, 77, dtype=np.uint32)))
        h = np.zeros(nb, dtype=np.uint32)
        h[rng.integers(0, nb)] = 5
        cases.append((f"single{nb}", h))
        sp = np.zeros(nb, dtype=np.uint32)
        idx = rng.choice(nb, size=max(1, nb // 9), replace=False)
        sp[idx] = rng.integers(1, 30, size=idx.size)
        cases.append((f"sparse{nb}", sp))
    fib = [1, 1]
    while len(fib) < 45:
        fib.append(fib[-1] + fib[-2])
    cases.append(("fibonacci45", np.array(fib, dtype=np.uint32)))
    cases.append(("allzero", np.zeros(300, dtype=np.uint32)))
    # boundaries of the codebook's paths: one id per thread (<= 1024 bins) or
    # slices; shared arrays (<= 4096 bins) or global scratch
    for nb in (1025, 4097):
        cases.append((f"zipf{nb}", np.maximum(1, np.floor(3e6 * np.arange(1, nb + 1, dtype=np.float64) ** -1.1))
                      .astype(np.uint32)[rng.permutation(nb)]))
        cases.append((f"ties{nb}", rng.integers(0, 4, size=nb).astype(np.uint32)))
    # counts of 2^24 and more: four radix passes over a large alphabet
    big = rng.integers(1, 1000, size=8000).astype(np.uint32)
    big[[5, 77, 4000]] = [1 << 30, (1 << 30) + 12345, 1 << 29]
    cases.append(("bigcounts8000", big))
    # a sparse histogram over a small alphabet: only pow2(m) keys are sorted
    sp = np.zeros(1024, dtype=np.uint32)
    sp[rng.choice(1024, size=3, replace=False)] = [7, 7, 2]
    cases.append(("three_of_1024", sp))
    return cases


@pytest.mark.parametrize("name,h", _hist_cases(), ids=[c[0] for c in _hist_cases()])
def test_codebook_matches_oracle(name, h):
    import torch
    nb = h.size
    r = Run(np.zeros(0, np.uint16), nb)
    hd = torch.from_numpy(h.view(np.int32)).cuda()
    r.codebook(hd)
    assert r.status() == 0
    _cmp_book(r.book_np(), oracle.codebook(h), h)


def test_long_codewords_fibonacci():
    """Counts F1..F45 give 44-bit codewords (over 32 bits): codebook and a
    short stream through the 64-bit entry path."""
    import torch
    fib = [1, 1]
    while len(fib) < 45:
        fib.append(fib[-1] + fib[-2])
    h = np.array(fib, dtype=np.uint32)
    want = oracle.codebook(h)
    rng = np.random.default_rng(5)
    sym = rng.integers(0, 45, size=50_000).astype(np.uint32)
    r = Run(sym, 45)
    r.codebook(torch.from_numpy(h.view(np.int32)).cuda()).encode()
    assert r.status() == 0
    _cmp_book(r.book_np(), want)
    words, offs, tb = oracle.encode(sym, want, chunk_log2=10)
    got, gtb = r.stream_np()
    assert gtb == tb and np.array_equal(got, words)
    assert np.array_equal(r.offs_np(), offs)


def _fibonacci_field(nsym, nbins, dtype, seed):
    """A field whose histogram is F1..F(nsym) on nsym ids spread over the
    alphabet: its longest codeword has nsym - 1 bits."""
    fib = [1, 1]
    while len(fib) < nsym:
        fib.append(fib[-1] + fib[-2])
    ids = (np.arange(nsym, dtype=np.int64) * 37 + 5) % nbins
    sym = np.repeat(ids, fib).astype(dtype)
    np.random.default_rng(seed).shuffle(sym)
    return sym


@pytest.mark.parametrize("max_len", [23, 24, 25, 27, 28])
@pytest.mark.parametrize("width", [1, 2])
def test_codewords_just_over_the_table_entry(max_len, width):
    """Longest codewords of 23 to 28 bits through the plain calls: up to 23
    bits the segment path, above it the general encoder of the same launch
    (the batched per-field form takes them on the segment path: see
    test_gpu_batch)."""
    nb = 256 if width == 1 else 1024
    sym = _fibonacci_field(max_len + 1, nb, np.uint8 if width == 1 else np.uint16, max_len)
    r, want, words, tb = _full_check(sym, nb)
    assert want["max_len"] == max_len
    assert np.array_equal(oracle.decode(words, tb, sym.size, want, width=width), sym)


def test_error_symbol_out_of_range():
    import paper_2010_10039_gb300 as huff
    sym = synth.laplace_field(50_000, seed=4)
    sym[12345] = 1500
    r = Run(sym, 1024).histogram()
    assert r.status() == huff.STATUS_CODE["HUFF_ERR_SYMBOL_RANGE"]


def test_error_symbol_without_codeword():
    import torch
    import paper_2010_10039_gb300 as huff
    sym = synth.laplace_field(50_000, seed=4)
    h = oracle.histogram(sym, 1024)
    h2 = h.copy()
    h2[sym[777]] = 0                       # codebook that lacks one used symbol
    r = Run(sym, 1024)
    r.codebook(torch.from_numpy(h2.view(np.int32)).cuda()).encode()
    assert r.status() == huff.STATUS_CODE["HUFF_ERR_NOT_IN_CODEBOOK"]


def test_error_capacity_and_canary():
    import paper_2010_10039_gb300 as huff
    sym = synth.laplace_field(200_000, seed=6)
    h = oracle.histogram(sym, 1024)
    want = oracle.codebook(h)
    _, _, tb = oracle.encode(sym, want)
    cap = (tb + 31) // 32 - 100
    r = Run(sym, 1024, cap_words=cap + 64)
    r.cap = cap
    r.out.fill_(0x5A5A5A5A)
    r.all()
    assert r.status() == huff.STATUS_CODE["HUFF_ERR_CAPACITY"]
    canary = u32(r.out[cap:])
    assert (canary == 0x5A5A5A5A).all(), "wrote past the capacity"


def test_error_histogram_overflow():
    import torch
    import paper_2010_10039_gb300 as huff
    h = np.array([0xFFFFFFFF, 7, 9], dtype=np.uint32)
    r = Run(np.zeros(0, np.uint16), 3)
    r.codebook(torch.from_numpy(h.view(np.int32)).cuda())
    assert r.status() == huff.STATUS_CODE["HUFF_ERR_HIST_OVERFLOW"]
    b = r.book_np()
    assert b["max_len"] == 0 and b["status"] == huff.STATUS_CODE["HUFF_ERR_HIST_OVERFLOW"]


def test_host_side_argument_errors():
    import torch
    import paper_2010_10039_gb300 as huff
    r = Run(synth.laplace_field(1000, seed=1), 1024)
    with pytest.raises(huff.HuffError):
        huff.huff_histogram(r.sym, 0, r.hist, r.ws)
    with pytest.raises(huff.HuffError):
        huff.huff_histogram(to_dev(np.zeros(10, np.uint8)), 300, r.hist, r.ws)
    with pytest.raises(huff.HuffError):
        huff.huff_encode(r.sym, r.book, 1024, r.out, r.offs, r.total, r.ws, {"chunk_log2": 2})


def test_gpu_decode_round_trip():
    import torch
    import paper_2010_10039_gb300 as huff
    sym = synth.laplace_field(500_000, seed=11)
    r = Run(sym, 1024).all()
    tb = int(r.total.item())
    out = torch.zeros(sym.size, dtype=torch.int16, device="cuda")
    huff.huff_decode(r.out, tb, r.offs, 10, sym.size, 2, r.book, 1024, out, r.ws)
    assert r.status() == 0
    assert np.array_equal(out.cpu().numpy().view(np.uint16), sym)


def test_hpc_field_full_size():
    """512^3 u16 Laplace(b=2) + 1 % outliers, seed 1, at full size: histogram,
    codebook, stream, offsets bit-exact vs the oracle (launch configuration of
    the benchmark)."""
    sym = synth.laplace_field(512 ** 3, seed=1)
    _full_check(sym, 1024)


@pytest.mark.parametrize("nbins", [5000, 20000])
def test_long_codes_large_alphabet(nbins):
    """Codes longer than 23 bits over an alphabet too large for the shared
    table: the encoder reads 64-bit codewords from global memory (and the
    32-bit entry table is not built)."""
    import torch
    fib = [1, 1]
    while len(fib) < 44:
        fib.append(fib[-1] + fib[-2])
    h = np.ones(nbins, dtype=np.uint32)
    h[:44] = fib
    want = oracle.codebook(h)
    assert want["max_len"] > 23
    rng = np.random.default_rng(nbins)
    sym = np.concatenate([np.arange(nbins, dtype=np.uint32),
                          rng.integers(0, 48, size=100_000).astype(np.uint32)])
    r = Run(sym, nbins)
    r.codebook(torch.from_numpy(h.view(np.int32)).cuda()).encode()
    assert r.status() == 0
    _cmp_book(r.book_np(), want)
    words, offs, tb = oracle.encode(sym, want, chunk_log2=10)
    got, gtb = r.stream_np()
    assert gtb == tb and np.array_equal(got, words)
    assert np.array_equal(r.offs_np(), offs)


@pytest.mark.parametrize("width", [2, 4])
def test_packed_histogram_heavy_bins(width):
    """Alphabets above 16,384 bins count in packed 16-bit shared counters
    (bins k and k + 32768 share a word) that carry 0x8000 to the global bin.
    Here one bin takes most of the field, so every CTA carries it many times,
    and the other half of the same word (bin 40000 - 32768 = 7232) and a bin
    near the top are heavy too; the input starts off a 16-byte boundary so the
    head and tail are counted as well."""
    n = 20_000_000 + 13
    rng = np.random.default_rng(77)
    sym = np.full(n, 40000, dtype=np.uint16 if width == 2 else np.uint32)
    sym[rng.integers(0, n, size=n // 3)] = 7232
    sym[rng.integers(0, n, size=n // 50)] = 65535
    sym[rng.integers(0, n, size=1000)] = 3
    r = Run(sym, 65536, offset_elems=3).histogram()
    assert r.status() == 0
    assert np.array_equal(r.hist_np(), oracle.histogram(sym, 65536))
    assert np.array_equal(r.hist_np(), np.bincount(sym, minlength=65536).astype(np.uint32))


@pytest.mark.parametrize("K", [8192, 65536])
def test_large_alphabet_full_size(K):
    """67,108,864 u32 Zipf(1.1) symbols over 8,192 / 65,536 permuted ids, seed 3."""
    sym = synth.zipf_field(1 << 26, K, seed=3)
    _full_check(sym, K)
