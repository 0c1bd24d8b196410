"""Stream formats on the GPU: 8-, 16- and 32-bit typed units (Sec. IV-C
typed cells) and the chunk-aligned layout (Sec. VI chunks before the dense
gathering).  Every unit, offset and bit count equals the oracle's
encode_format; the device decoder reads each format back to the input; a
buffer sized to the exact number of units is written to its last byte and
no further; a short one records HUFF_ERR_CAPACITY."""
import numpy as np
import pytest

import oracle
from paper_2010_10039_gb300 import synth
from gpu_util import to_dev

CANARY = 0xA5

FIELDS = {
    "u8": lambda n: (synth.laplace_field(n, seed=71, b=5.0, K=256).astype(np.uint8), 256),
    "u16": lambda n: (synth.laplace_field(n, seed=72), 1024),
    "u32": lambda n: (synth.zipf_field(n, 8192, seed=73), 8192),
}
ALIGNED_M = {"u8": (10, 13), "u16": (9, 12), "u32": (8, 11)}


def _encode(sym_np, nbins, W, layout, M, cap_units=None, slack_bytes=64):
    import torch
    import paper_2010_10039_gb300 as huff
    n = sym_np.size
    prm = {"chunk_log2": M, "word_bits": W, "layout": layout}
    sym = to_dev(sym_np)
    hist = torch.empty(nbins, dtype=torch.int32, device="cuda")
    book = torch.empty(huff.huff_codebook_bytes(nbins), dtype=torch.uint8, device="cuda")
    ws = torch.zeros(huff.huff_workspace_bytes(max(1, n), nbins, prm), dtype=torch.uint8, device="cuda")
    huff.huff_workspace_init(ws)
    huff.huff_histogram(sym, nbins, hist, ws)
    huff.huff_build_codebook(hist, nbins, book, ws)
    if cap_units is None:
        cap_units = huff.huff_max_output_units(n, 48, prm)
    nbytes = cap_units * W // 8
    buf = torch.full(((nbytes + slack_bytes + 3) // 4 * 4 + 64,), CANARY, dtype=torch.uint8, device="cuda")
    nch = (n + (1 << M) - 1) >> M
    offs = torch.full((nch + 1,), -1, dtype=torch.int64, device="cuda")
    total = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    huff.huff_encode(sym, book, nbins, buf, offs, total, ws, prm, capacity_words=cap_units)
    torch.cuda.synchronize()
    return dict(huff=huff, sym=sym, book=book, ws=ws, buf=buf, offs=offs, total=total, prm=prm, nbytes=nbytes,
                status=huff.huff_get_status(ws), hist=hist)


@pytest.mark.gpu
@pytest.mark.parametrize("dt", ["u8", "u16", "u32"])
@pytest.mark.parametrize("W", [8, 16, 32])
@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("n", [777_781, 5_003])
def test_format_equals_oracle_and_round_trips(dt, W, layout, n):
    import torch
    sym_np, nbins = FIELDS[dt](n)
    M = 10 if layout == 0 else ALIGNED_M[dt][(n // 7) % 2]
    r = _encode(sym_np, nbins, W, layout, M)
    assert r["status"] == 0
    book = oracle.codebook(oracle.histogram(sym_np, nbins))
    units, offs, tb = oracle.encode_format(sym_np, book, M, W, layout == 1)
    assert int(r["total"].item()) == tb
    got_offs = r["offs"].cpu().numpy().view(np.uint64)
    assert np.array_equal(got_offs, offs)
    raw = r["buf"].cpu().numpy()
    ub = units.size * W // 8
    assert np.array_equal(raw[:ub].view(oracle.UNIT_DTYPE[W]), units)
    # nothing past the stream's last unit within the buffer's whole words
    # that the stream does not own: bytes after the stream stay untouched
    assert (raw[ub:] == CANARY).all()
    # the device decoder reads the format back
    huff = r["huff"]
    back = torch.empty_like(r["sym"])
    huff.huff_decode_ex(r["buf"], tb, r["offs"], r["prm"], n, sym_np.dtype.itemsize, r["book"], nbins, back, r["ws"])
    torch.cuda.synchronize()
    assert huff.huff_get_status(r["ws"]) == 0
    assert torch.equal(back, r["sym"])


@pytest.mark.gpu
@pytest.mark.parametrize("W", [8, 16, 32])
@pytest.mark.parametrize("layout", [0, 1])
def test_exact_and_short_capacity(W, layout):
    sym_np, nbins = FIELDS["u16"](300_007)
    M = 10
    book = oracle.codebook(oracle.histogram(sym_np, nbins))
    units, offs, tb = oracle.encode_format(sym_np, book, M, W, layout == 1)
    r = _encode(sym_np, nbins, W, layout, M, cap_units=units.size)
    assert r["status"] == 0
    raw = r["buf"].cpu().numpy()
    ub = units.size * W // 8
    assert np.array_equal(raw[:ub].view(oracle.UNIT_DTYPE[W]), units)
    assert (raw[ub:] == CANARY).all()
    short = units.size - 3
    r = _encode(sym_np, nbins, W, layout, M, cap_units=short)
    assert r["status"] == 4                                   # HUFF_ERR_CAPACITY
    raw = r["buf"].cpu().numpy()
    assert (raw[short * W // 8:] == CANARY).all()


@pytest.mark.gpu
def test_format_arguments_are_checked():
    import torch
    import paper_2010_10039_gb300 as huff
    sym_np, nbins = FIELDS["u16"](10_000)
    for prm in ({"word_bits": 12}, {"layout": 2}, {"layout": 1, "chunk_log2": 8}, {"layout": 1, "chunk_log2": 13},
                {"word_bits": 8, "merge": 2}, {"layout": 1, "chunk_log2": 10, "merge": 2}):
        p = {"chunk_log2": 10}
        p.update(prm)
        with pytest.raises(RuntimeError):
            huff.huff_encode(to_dev(sym_np), torch.empty(64, dtype=torch.uint8, device="cuda"), nbins,
                             torch.empty(16, dtype=torch.int32, device="cuda"),
                             torch.empty(16, dtype=torch.int64, device="cuda"),
                             torch.empty(1, dtype=torch.int64, device="cuda"),
                             torch.zeros(1 << 16, dtype=torch.uint8, device="cuda"), p)


@pytest.mark.gpu
@pytest.mark.parametrize("W,layout,M", [(8, 0, 10), (16, 1, 11)])
def test_noalloc_takes_the_format(W, layout, M):
    import torch
    import paper_2010_10039_gb300 as huff
    sym_np, nbins = FIELDS["u16"](400_009)
    r = _encode(sym_np, nbins, W, layout, M)
    assert r["status"] == 0
    tb = int(r["total"].item())
    cap = huff.huff_max_output_units(sym_np.size, 48, r["prm"])
    buf = torch.full_like(r["buf"], CANARY)
    offs = torch.full_like(r["offs"], -1)
    total = torch.full_like(r["total"], -1)
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    huff.huff_encode_noalloc(r["sym"], r["book"], nbins, buf, offs, total, status, r["prm"], capacity_words=cap)
    torch.cuda.synchronize()
    assert int(status.item()) == 0 and int(total.item()) == tb
    assert torch.equal(buf, r["buf"]) and torch.equal(offs, r["offs"])
