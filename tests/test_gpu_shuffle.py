"""The paper's three-kernel encode (merge = HUFF_MERGE_SHUFFLE: per-chunk
reduce-merge and log-step shuffle-merge, chunk-length scan, coalescing copy)
gives the same stream and offsets as the oracle and as the fused default."""
import numpy as np
import pytest

import oracle
from paper_2010_10039_gb300 import synth
from gpu_util import Run

pytestmark = pytest.mark.gpu

SHUF = 2


@pytest.mark.parametrize("width,nbins", [(1, 256), (2, 1024), (4, 8192)])
@pytest.mark.parametrize("n", [1, 17, 1023, 1024, 1025, 4096 * 3 + 5, 300_001])
@pytest.mark.parametrize("M,r", [(10, 3), (10, -1), (6, 2), (12, 4), (8, 0)])
def test_shuffle_path_matches_oracle(width, nbins, n, M, r):
    p = synth.laplace_pmf(nbins, nbins // 2, 4.0)
    sym = synth.draw(7, n, n, synth.cdf_table(p), width)
    run = Run(sym, nbins, chunk_log2=M, params={"merge": SHUF, "reduce_log2": r}).all()
    assert run.status() == 0
    want = oracle.codebook(oracle.histogram(sym, nbins))
    words, offs, tb = oracle.encode(sym, want, chunk_log2=M)
    got, gtb = run.stream_np()
    assert gtb == tb
    assert np.array_equal(got, words)
    assert np.array_equal(run.offs_np(), offs)


def test_shuffle_path_hpc_field_prefix():
    sym = synth.laplace_field(1 << 24, seed=1)
    run = Run(sym, 1024, params={"merge": SHUF}).all()
    assert run.status() == 0
    fused = Run(sym, 1024).all()
    a, ta = run.stream_np()
    b, tb = fused.stream_np()
    assert ta == tb and np.array_equal(a, b)
    assert np.array_equal(run.offs_np(), fused.offs_np())


def test_shuffle_path_rejects_unsupported_shapes():
    import paper_2010_10039_gb300 as huff
    sym = synth.gaussian_field(10_000, seed=0)
    for prm in ({"merge": SHUF, "reduce_log2": 5}, {"merge": SHUF, "chunk_log2": 16, "reduce_log2": 2}):
        run = Run(sym, 1024, chunk_log2=prm.get("chunk_log2", 10), params=prm).histogram().codebook()
        with pytest.raises(huff.HuffError):
            run.encode()
