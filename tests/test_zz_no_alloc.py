"""huff_encode_noalloc: the encode entry point for callers that cannot
allocate device memory (it uses a fixed array inside the library instead of a
caller workspace).  Its stream, chunk offsets and bit count must equal those
of huff_encode, on two calls in a row (the second call sees the array as the
first one left it).  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2010_10039_gb300 import synth
from gpu_util import Run, to_dev, u32, u64


@pytest.mark.gpu
def test_noalloc_matches_workspace_encode_twice():
    import torch
    import paper_2010_10039_gb300 as huff
    inputs = [synth.laplace_field(3_000_017, seed=31), synth.laplace_field(700_001, seed=32, b=6.0)]
    for sym_np in inputs:
        ref = Run(sym_np, 1024).all()                      # workspace path
        assert ref.status() == 0
        out = torch.zeros_like(ref.out)
        offs = torch.full_like(ref.offs, -1)
        total = torch.full_like(ref.total, -1)
        status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        huff.huff_encode_noalloc(ref.sym, ref.book, 1024, out, offs, total, status,
                                 {"chunk_log2": ref.chunk_log2}, n=ref.n, dtype=2)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        tb = int(ref.total.item())
        assert int(total.item()) == tb
        nw = (tb + 31) // 32
        assert np.array_equal(u32(out[:nw]), u32(ref.out[:nw]))
        assert np.array_equal(u64(offs), u64(ref.offs))


@pytest.mark.gpu
def test_noalloc_rejects_inputs_beyond_its_array():
    import torch
    import paper_2010_10039_gb300 as huff
    d = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(huff.HuffError):
        huff.huff_encode_noalloc(d, d, 1024, d, d, d, d, n=(1 << 28) + 1, dtype=2, capacity_words=16)
