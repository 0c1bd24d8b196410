"""Alphabets above 65,536 symbols (n-gram / k-mer alphabets): the windowed
histogram, the codebook with 32-bit ids, the encoder and the decoder, against
the oracle element by element, up to 2^20 symbols."""
import numpy as np
import pytest

import oracle
from paper_2010_10039_gb300 import synth
from gpu_util import Run
from test_gpu_parity import _cmp_book, _full_check

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nbins", [65_537, 1 << 18, 300_007, 1 << 20])
def test_zipf_field_equals_oracle(nbins):
    """u32 Zipf(1.1) over permuted ids: hot bins pass 32,768 counts in one CTA
    (the carry path), the codebook sorts up to 2^20 keys, and long codes take
    the global codeword table."""
    sym = synth.zipf_field(3_000_017, nbins, seed=81)
    r, want, words, tb = _full_check(sym, nbins)
    import torch
    back = torch.empty_like(r.sym)
    r.huff.huff_decode(r.out, tb, r.offs, 10, sym.size, 4, r.book, nbins, back, r.ws)
    torch.cuda.synchronize()
    assert r.status() == 0
    assert torch.equal(back, r.sym)


def test_every_bin_used_with_ties():
    """2^20 bins, each used 1..4 times (the codebook melds 2^20 leaves with
    massive ties)."""
    rng = np.random.default_rng(82)
    nbins = 1 << 20
    reps = rng.integers(1, 5, nbins)
    sym = np.repeat(np.arange(nbins, dtype=np.uint32), reps)
    rng.shuffle(sym)
    _full_check(sym, nbins)


@pytest.mark.parametrize("nbins", [1 << 18, 1 << 20])
def test_codebook_from_histogram(nbins):
    import torch
    rng = np.random.default_rng(nbins)
    h = (rng.pareto(1.2, nbins) * 10).astype(np.uint32)
    h[rng.integers(0, nbins, nbins // 3)] = 0                 # unused bins
    r = Run(np.zeros(0, np.uint32), nbins)
    r.codebook(torch.from_numpy(h.view(np.int32)).cuda())
    assert r.status() == 0
    _cmp_book(r.book_np(), oracle.codebook(h), h)


def test_symbol_out_of_range_is_reported():
    nbins = 200_000
    sym = synth.zipf_field(500_000, nbins, seed=83)
    sym[12345] = nbins + 7
    r = Run(sym, nbins).histogram()
    assert r.status() == 2                                    # HUFF_ERR_SYMBOL_RANGE


def test_u16_above_65536_bins_is_rejected():
    import paper_2010_10039_gb300 as huff
    L = huff.lib()
    assert L.huff_histogram(0x100000, 100, huff.HUFF_U16, 65537, 0x200000, 0x300000, None) == 1
