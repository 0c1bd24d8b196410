"""huff_encode_noalloc: the encode entry point for callers that cannot
allocate device memory (it uses a fixed array inside the library instead of a
caller workspace).  Its stream, chunk offsets and bit count must equal those
of huff_encode, on two calls in a row (the second call sees the array as the
first one left it).  The cases cover each part of the array: the look-back
descriptors (every case), the 32-bit codebook entries of an alphabet over
4,096 symbols (8,192 and 65,536 bins), 1- and 4-byte symbols and an empty
input.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2010_10039_gb300 import synth
from gpu_util import Run, to_dev, u32, u64

CASES = {
    "u16_1024": lambda: (synth.laplace_field(3_000_017, seed=31), 1024),
    "u16_1024_b6": lambda: (synth.laplace_field(700_001, seed=32, b=6.0), 1024),
    "u32_8192": lambda: (synth.zipf_field(1_000_003, 8192, seed=33), 8192),
    "u32_65536": lambda: (synth.zipf_field(1_500_001, 65536, seed=34), 65536),
    "u8_256": lambda: ((synth.laplace_field(900_001, seed=35, b=5.0, K=256)).astype(np.uint8), 256),
    "empty": lambda: (np.zeros(0, np.uint16), 1024),
}


@pytest.mark.gpu
@pytest.mark.parametrize("name", list(CASES))
def test_noalloc_matches_workspace_encode_twice(name):
    import torch
    import paper_2010_10039_gb300 as huff
    sym_np, nbins = CASES[name]()
    ref = Run(sym_np, nbins).all()                     # workspace path
    assert ref.status() == 0
    tb = int(ref.total.item())
    nw = (tb + 31) // 32
    for _ in range(2):
        out = torch.full_like(ref.out, 0x5A5A5A5A)
        offs = torch.full_like(ref.offs, -1)
        total = torch.full_like(ref.total, -1)
        status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        huff.huff_encode_noalloc(ref.sym, ref.book, nbins, out, offs, total, status,
                                 {"chunk_log2": ref.chunk_log2}, n=ref.n, dtype=ref.dtype, capacity_words=ref.cap)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert int(total.item()) == tb
        assert np.array_equal(u32(out[:nw]), u32(ref.out[:nw]))
        assert np.array_equal(u64(offs), u64(ref.offs))


@pytest.mark.gpu
def test_noalloc_rejects_inputs_beyond_its_array():
    import torch
    import paper_2010_10039_gb300 as huff
    d = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(huff.HuffError):
        huff.huff_encode_noalloc(d, d, 1024, d, d, d, d, n=(1 << 28) + 1, dtype=2, capacity_words=16)


@pytest.mark.gpu
def test_noalloc_rejects_the_paper_layout_merge():
    import torch
    import paper_2010_10039_gb300 as huff
    d = torch.zeros(16, dtype=torch.int32, device="cuda")
    for merge in (huff.HUFF_MERGE_SHUFFLE, 7):
        with pytest.raises(huff.HuffError):
            huff.huff_encode_noalloc(d, d, 1024, d, d, d, d, {"merge": merge}, n=8, dtype=2, capacity_words=16)
