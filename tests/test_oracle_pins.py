"""Pins for the CPU oracle: checks against facts that do not come from the
oracle itself (hand-worked fixtures, closed forms, brute force, library
routines, information-theoretic bounds)."""
import glob
import heapq
import itertools
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_fixture(path):
    d = {}
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, v = line.split(":", 1)
            d[k.strip()] = v.split()
    return d


FIXTURES = sorted(glob.glob(os.path.join(GOLDEN, "example*.txt")))


@pytest.mark.parametrize("path", FIXTURES, ids=[os.path.basename(p) for p in FIXTURES])
def test_golden_fixture(path):
    fx = _read_fixture(path)
    counts = np.array([int(x) for x in fx["counts"]], dtype=np.uint32)
    want_len = [int(x) for x in fx["lengths"]]
    for method in ("two_queue", "heap"):
        ln = oracle.lengths(counts, method)
        assert ln.tolist() == want_len, method
    assert int((counts.astype(np.int64) * np.array(want_len)).sum()) == int(fx["weighted_length"][0])
    book = oracle.canonical(oracle.lengths(counts))
    codes = [format(int(c), f"0{l}b") for c, l in zip(book["code"], want_len)]
    assert codes == fx["codes"]
    for kv in fx["first"]:
        l, v = map(int, kv.split("="))
        assert int(book["first"][l]) == v
    for kv in fx["entry"]:
        l, v = map(int, kv.split("="))
        assert int(book["entry"][l]) == v
    assert book["sorted_syms"].tolist() == [int(x) for x in fx["sorted_syms"]]
    sym = np.array([int(x) for x in fx["input"]], dtype=np.uint16)
    words, offs, tb = oracle.encode(sym, book, chunk_log2=1)
    assert tb == int(fx["total_bits"][0])
    assert [int(w) for w in words] == [int(x, 16) for x in fx["words"]]
    back = oracle.decode(words, tb, sym.size, book, width=2)
    assert back.tolist() == sym.tolist()


# --------------------------------------------------------------- histogram

@pytest.mark.parametrize("width,nbins", [(1, 256), (2, 1024), (4, 65536), (2, 1)])
def test_histogram_matches_bincount(width, nbins):
    rng = np.random.default_rng(width * 7 + nbins)
    dt = {1: np.uint8, 2: np.uint16, 4: np.uint32}[width]
    sym = rng.integers(0, nbins, size=100_003).astype(dt)
    h = oracle.histogram(sym, nbins)
    assert np.array_equal(h, np.bincount(sym.astype(np.int64), minlength=nbins).astype(np.uint32))
    assert int(h.sum()) == sym.size


def test_histogram_rejects_out_of_range():
    with pytest.raises(oracle.OracleError):
        oracle.histogram(np.array([0, 5, 1024], dtype=np.uint16), 1024)


# ----------------------------------------------------------------- lengths

def _brute_force_min_cost(freq):
    """Minimum sum f*l over ALL length vectors with Kraft sum <= 1 (n <= 7),
    by exhaustive enumeration."""
    n = len(freq)
    f = np.asarray(freq, dtype=np.int64)
    L = np.array(list(itertools.product(range(1, n), repeat=n)), dtype=np.int64)
    kraft = (2.0 ** (-L)).sum(axis=1)
    ok = kraft <= 1.0 + 1e-12
    return int((L[ok] * f).sum(axis=1).min())


def _multiset_min_cost(freq):
    """Same minimum for n = 8: enumerate every multiset of lengths with Kraft
    sum <= 1 and pair the longest lengths with the smallest counts
    (rearrangement inequality)."""
    n = len(freq)
    f = np.sort(np.asarray(freq, dtype=np.int64))[::-1]
    best = None
    for ls in itertools.combinations_with_replacement(range(1, n), n):
        if sum(2.0 ** -l for l in ls) <= 1.0 + 1e-12:
            c = int((np.array(ls) * f).sum())
            best = c if best is None else min(best, c)
    return best


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7, 8])
def test_lengths_brute_force_optimal(n):
    rng = np.random.default_rng(100 + n)
    trials = 30 if n < 8 else 12
    for t in range(trials):
        hi = [3, 10, 1000][t % 3]          # small ranges force many ties
        freq = rng.integers(1, hi + 1, size=n).astype(np.uint32)
        ln = oracle.lengths(freq)
        cost = int((ln.astype(np.int64) * freq).sum())
        ref = _brute_force_min_cost(freq) if n <= 7 else _multiset_min_cost(freq)
        assert cost == ref, (freq, ln)


def _heapq_cost(freq):
    """Textbook fact: the optimal weighted length equals the sum of the weights
    of all joined nodes of any Huffman tree (computed with Python's heapq)."""
    h = [int(x) for x in freq if x > 0]
    if len(h) <= 1:
        return sum(h)
    heapq.heapify(h)
    tot = 0
    while len(h) > 1:
        a, b = heapq.heappop(h), heapq.heappop(h)
        tot += a + b
        heapq.heappush(h, a + b)
    return tot


def _random_hist(rng, nbins, kind):
    if kind == "uniform":
        return rng.integers(0, 1000, size=nbins).astype(np.uint32)
    if kind == "ties":
        return rng.integers(0, 4, size=nbins).astype(np.uint32)
    if kind == "pow2":
        return (1 << rng.integers(0, 12, size=nbins)).astype(np.uint32)
    if kind == "zipf":
        r = np.arange(1, nbins + 1, dtype=np.float64)
        h = np.floor(1e6 * r ** -1.1).astype(np.uint32)
        return h[rng.permutation(nbins)]
    if kind == "sparse":
        h = np.zeros(nbins, dtype=np.uint32)
        idx = rng.choice(nbins, size=max(1, nbins // 10), replace=False)
        h[idx] = rng.integers(1, 50, size=idx.size)
        return h
    raise ValueError(kind)


@pytest.mark.parametrize("nbins", [2, 3, 17, 256, 1024, 8192])
@pytest.mark.parametrize("kind", ["uniform", "ties", "pow2", "zipf", "sparse"])
def test_lengths_two_formulations_and_bounds(nbins, kind):
    rng = np.random.default_rng(nbins * 31 + len(kind))
    h = _random_hist(rng, nbins, kind)
    a = oracle.lengths(h, "two_queue")
    b = oracle.lengths(h, "heap")
    assert np.array_equal(a, b)
    used = h > 0
    assert np.array_equal(a > 0, used)
    cost = int((a.astype(np.int64) * h).sum())
    assert cost == _heapq_cost(h)
    m = int(used.sum())
    if m >= 2:
        kraft = sum(2.0 ** -int(l) for l in a[used])
        assert abs(kraft - 1.0) < 1e-12
        tot = float(h.sum())
        p = h[used] / tot
        H = float(-(p * np.log2(p)).sum())
        beta = cost / tot
        assert H - 1e-9 <= beta < H + 1


def test_lengths_edge_cases():
    assert oracle.lengths(np.zeros(16, dtype=np.uint32)).tolist() == [0] * 16
    h = np.zeros(16, dtype=np.uint32)
    h[9] = 1234
    ln = oracle.lengths(h)
    assert ln[9] == 1 and int(ln.sum()) == 1
    book = oracle.canonical(ln)
    assert int(book["code"][9]) == 0 and book["max_len"] == 1
    # equal counts over 2^k symbols: every length is k, codes are the ids
    for k in (1, 4, 10):
        h = np.full(1 << k, 5, dtype=np.uint32)
        ln = oracle.lengths(h)
        assert (ln == k).all()
        book = oracle.canonical(ln)
        assert book["code"].tolist() == list(range(1 << k))


def test_lengths_reject_overflowing_histogram():
    h = np.array([0xFFFFFFFF, 2], dtype=np.uint32)
    with pytest.raises(oracle.OracleError):
        oracle.lengths(h)


def _fib(m):
    f = [1, 1]
    while len(f) < m:
        f.append(f[-1] + f[-2])
    return f[:m]


def test_fibonacci_longest_codes():
    """Counts F1..F45: the caterpillar tree, lengths 44,44,43,...,1 (the
    longest lengths a histogram summing below 2^32 can produce)."""
    fib = _fib(45)
    assert sum(fib) == 2971215072
    h = np.array(fib, dtype=np.uint32)
    for method in ("two_queue", "heap"):
        ln = oracle.lengths(h, method)
        assert ln.tolist() == [44, 44] + list(range(43, 0, -1))
    book = oracle.codebook(h)
    assert book["max_len"] == 44
    assert int(book["code"][0]) == 0 and int(book["code"][1]) == 1
    assert int(book["code"][44]) == 1            # the single 1-bit codeword is '1'
    sym = np.array([0, 44, 1, 2, 43, 0, 0, 44], dtype=np.uint32)
    words, offs, tb = oracle.encode(sym, book, chunk_log2=2)
    assert tb == 44 + 1 + 44 + 43 + 2 + 44 + 44 + 1
    assert oracle.decode(words, tb, sym.size, book, width=4).tolist() == sym.tolist()


# --------------------------------------------------------------- canonical

@pytest.mark.parametrize("kind", ["uniform", "ties", "zipf", "sparse"])
def test_canonical_properties(kind):
    rng = np.random.default_rng(7 + len(kind))
    h = _random_hist(rng, 1024, kind)
    book = oracle.codebook(h)
    ln, code = book["len"], book["code"]
    used = np.nonzero(ln)[0]
    bits = [format(int(code[s]), f"0{int(ln[s])}b") for s in used]
    # prefix-free: in lexicographic order a prefix would sit right before its extension
    sb = sorted(bits)
    for a, b in zip(sb, sb[1:]):
        assert not b.startswith(a)
    # the orientation Sec. IV-B2 asks for: a shorter codeword is larger than the
    # same-length prefix of every longer codeword
    byl = {}
    for s in used:
        byl.setdefault(int(ln[s]), []).append(int(code[s]))
    lens = sorted(byl)
    for i, l1 in enumerate(lens):
        lo1 = min(byl[l1])
        for l2 in lens[i + 1:]:
            assert max(byl[l2]) >> (l2 - l1) < lo1
    # within one length codewords increase with the symbol id, consecutively
    for l in lens:
        syms = [s for s in used if ln[s] == l]
        cs = [int(code[s]) for s in syms]
        assert cs == list(range(cs[0], cs[0] + len(cs)))
        assert cs[0] == int(book["first"][l])
    # entry[l] counts the shorter codewords; sorted_syms ordered by (len, id)
    for l in lens:
        assert int(book["entry"][l]) == int((ln[used] < l).sum())
    order = sorted(used.tolist(), key=lambda s: (int(ln[s]), s))
    assert book["sorted_syms"].tolist() == order


def _prefix_free_and_oriented(ln, code):
    used = [s for s in range(len(ln)) if ln[s]]
    bits = sorted(format(int(code[s]), f"0{int(ln[s])}b") for s in used)
    for x, y in zip(bits, bits[1:]):
        if y.startswith(x):
            return False
    byl = {}
    for s in used:
        byl.setdefault(int(ln[s]), []).append(int(code[s]))
    lens = sorted(byl)
    return all(max(byl[l2]) >> (l2 - l1) < min(byl[l1]) for i, l1 in enumerate(lens) for l2 in lens[i + 1:])


def test_canonical_incomplete_lengths():
    """Canonical codes from any length vector with Kraft sum <= 1 (not only
    the complete ones Huffman gives) are prefix-free, in the orientation
    Sec. IV-B2 asks for.  Example: lengths (1, 3, 3) have Kraft sum 3/4 and
    give 1, 000, 001 (the rounding up in First matters here: 0, 000, 001
    would not be prefix-free)."""
    book = oracle.canonical(np.array([1, 3, 3], dtype=np.uint8))
    assert [format(int(c), f"0{l}b") for c, l in zip(book["code"], [1, 3, 3])] == ["1", "000", "001"]
    rng = np.random.default_rng(11)
    for t in range(300):
        n = int(rng.integers(1, 40))
        ln = rng.integers(1, 12, size=n)
        while (2.0 ** -ln.astype(np.float64)).sum() > 1.0:
            ln[int(rng.integers(0, n))] += 1
        ln = ln.astype(np.uint8)
        book = oracle.canonical(ln)
        assert _prefix_free_and_oriented(ln, book["code"]), ln.tolist()


# ------------------------------------------------------------------ encode

def _naive_bits(sym, book):
    return "".join(format(int(book["code"][s]), f"0{int(book['len'][s])}b") for s in sym)


def _pack(bitstr):
    pad = (-len(bitstr)) % 32
    b = bitstr + "0" * pad
    return [int(b[i:i + 32], 2) for i in range(0, len(b), 32)]


@pytest.mark.parametrize("n", [0, 1, 31, 32, 33, 1023, 1024, 1025, 5000])
@pytest.mark.parametrize("chunk_log2", [3, 10])
def test_encode_matches_string_concatenation(n, chunk_log2):
    rng = np.random.default_rng(n + 17 * chunk_log2)
    sym = rng.choice(64, size=n, p=np.arange(64, 0, -1) / np.arange(64, 0, -1).sum()).astype(np.uint16)
    h = np.bincount(sym, minlength=64).astype(np.uint32)
    if n == 0:
        h[:] = 1
    book = oracle.codebook(h)
    words, offs, tb = oracle.encode(sym, book, chunk_log2=chunk_log2)
    ref = _naive_bits(sym, book)
    assert tb == len(ref)
    assert [int(w) for w in words] == _pack(ref)
    lens = book["len"][sym].astype(np.int64)
    cs = np.concatenate([[0], np.cumsum(lens)])
    starts = np.arange(0, n, 1 << chunk_log2)
    assert offs.tolist() == cs[starts].tolist() + [len(ref)]
    assert int(tb) == int((h.astype(np.int64) * book["len"]).sum()) or n == 0
    assert oracle.decode(words, tb, n, book, width=2).tolist() == sym.tolist()


def test_encode_errors():
    h = np.array([3, 0, 2], dtype=np.uint32)
    book = oracle.codebook(h)
    with pytest.raises(oracle.OracleError):
        oracle.encode(np.array([0, 1], dtype=np.uint16), book)      # no codeword
    with pytest.raises(oracle.OracleError):
        oracle.encode(np.array([0, 3], dtype=np.uint16), book)      # out of range
    with pytest.raises(oracle.OracleError):
        oracle.encode(np.array([0, 2, 0, 2], dtype=np.uint16), book, capacity_words=0)


def test_round_trip_synthetic_fields():
    from paper_2010_10039_gb300 import synth
    for sym, nb in [(synth.gaussian_field(50_000, seed=0), 1024),
                    (synth.laplace_field(50_000, seed=1), 1024),
                    (synth.zipf_field(50_000, 8192, seed=3), 8192)]:
        h = oracle.histogram(sym, nb)
        book = oracle.codebook(h)
        words, offs, tb = oracle.encode(sym, book, chunk_log2=10)
        assert tb == int((h.astype(np.int64) * book["len"]).sum())
        assert np.array_equal(oracle.decode(words, tb, sym.size, book, width=sym.itemsize), sym)


# ------------------------------------------------------------------ typed units

def _naive_units(sym, book, chunk_log2, W, aligned):
    """The definition written out with Python strings: chunk bit strings, each
    padded to a unit boundary in the aligned form, cut into W-bit units."""
    n = sym.size
    out, offs = "", []
    for c0 in range(0, n, 1 << chunk_log2):
        if aligned:
            out += "0" * ((-len(out)) % W)
        offs.append(len(out) // W if aligned else len(out))
        out += _naive_bits(sym[c0:c0 + (1 << chunk_log2)], book)
    if aligned:
        out += "0" * ((-len(out)) % W)
    offs.append(len(out) // W if aligned else len(out))
    total = len(out)
    padded = out + "0" * ((-len(out)) % W)
    units = [int(padded[i:i + W], 2) for i in range(0, len(padded), W)]
    return units, offs, total


@pytest.mark.parametrize("W", [8, 16, 32])
@pytest.mark.parametrize("aligned", [False, True])
@pytest.mark.parametrize("n,chunk_log2", [(0, 3), (1, 3), (37, 3), (1000, 4), (1025, 6), (3001, 10)])
def test_encode_format_matches_string_definition(W, aligned, n, chunk_log2):
    rng = np.random.default_rng(7 * n + W + chunk_log2 + (100 if aligned else 0))
    sym = rng.choice(40, size=n, p=np.arange(40, 0, -1) / np.arange(40, 0, -1).sum()).astype(np.uint16)
    h = np.bincount(sym, minlength=40).astype(np.uint32)
    if n == 0:
        h[:] = 1
    book = oracle.codebook(h)
    units, offs, tb = oracle.encode_format(sym, book, chunk_log2, W, aligned)
    want_units, want_offs, want_tb = _naive_units(sym, book, chunk_log2, W, aligned)
    assert units.dtype == oracle.UNIT_DTYPE[W]
    assert [int(u) for u in units] == want_units
    assert offs.tolist() == want_offs
    assert tb == want_tb


def test_encode_format_dense_units_are_the_big_endian_words():
    """Dense 8- and 16-bit units are the 32-bit stream's words split most
    significant part first; 32-bit units are the words themselves."""
    from paper_2010_10039_gb300 import synth
    sym = synth.laplace_field(20_011, seed=9)
    book = oracle.codebook(oracle.histogram(sym, 1024))
    words, offs, tb = oracle.encode(sym, book, chunk_log2=10)
    be = words.astype(">u4").tobytes()
    for W in (8, 16, 32):
        units, o, t = oracle.encode_format(sym, book, 10, W, False)
        assert t == tb and np.array_equal(o, offs)
        want = np.frombuffer(be, dtype=f">u{W // 8}")[: (tb + W - 1) // W]
        assert np.array_equal(units, want.astype(oracle.UNIT_DTYPE[W]))


@pytest.mark.parametrize("W", [8, 16, 32])
def test_encode_format_aligned_chunks_decode_alone(W):
    """Every chunk of the aligned form starts at its offset and decodes on its
    own to its symbols; the padding between chunks is zero and shorter than a
    unit."""
    from paper_2010_10039_gb300 import synth
    sym = synth.gaussian_field(9_000, seed=4)
    book = oracle.codebook(oracle.histogram(sym, 1024))
    M = 9
    units, offs, tb = oracle.encode_format(sym, book, M, W, True)
    assert tb == int(offs[-1]) * W and units.size == int(offs[-1])
    bits = "".join(format(int(u), f"0{W}b") for u in units)
    for c in range(offs.size - 1):
        chunk = sym[c << M:(c + 1) << M]
        body = _naive_bits(chunk, book)
        seg = bits[int(offs[c]) * W:int(offs[c + 1]) * W]
        assert seg.startswith(body) and set(seg[len(body):]) <= {"0"} and len(seg) - len(body) < W
        words = _pack(body)
        assert oracle.decode(np.array(words, np.uint32), len(body), chunk.size, book, width=2).tolist() == \
            chunk.tolist()


def test_encode_format_errors():
    book = oracle.codebook(np.array([3, 0, 2], dtype=np.uint32))
    sym = np.array([0, 2, 0, 2], dtype=np.uint16)
    with pytest.raises(oracle.OracleError):
        oracle.encode_format(sym, book, 3, 12, False)               # not a unit width
    with pytest.raises(oracle.OracleError):
        oracle.encode_format(np.array([1], np.uint16), book, 3, 8, True)   # no codeword
