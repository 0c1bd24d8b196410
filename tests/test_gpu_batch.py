"""Batched form vs the CPU oracle: every field of a batch (one graph of a
histogram, codebook, planner and persistent encode launch per field group)
must equal the oracle's histogram, codebook, stream and offsets for that
field alone (integer work: bit-exact)."""
import numpy as np
import pytest

import oracle
from paper_2010_10039_gb300 import synth
from gpu_util import to_dev, u32, u64

pytestmark = pytest.mark.gpu

WIDTH = {1: np.uint8, 2: np.uint16, 4: np.uint32}


def _field_input(j, n, nbins, width, b=None, seed=11):
    b = b if b is not None else 0.5 + (j % 13) * 1.3
    pmf = synth.laplace_pmf(nbins, nbins // 2, b)
    return synth.draw(seed, j, n, synth.cdf_table(pmf), width)


def _make(fields_np, nbins_list, chunk_list=None, offsets_elems=None):
    import torch
    fields = []
    for i, (a, nb) in enumerate(zip(fields_np, nbins_list)):
        off = offsets_elems[i] if offsets_elems else 0
        if a.size:
            sym = to_dev(a, off)
        else:
            sym = torch.empty(0, dtype={1: torch.uint8, 2: torch.int16, 4: torch.int32}[a.dtype.itemsize],
                              device="cuda")
        m = chunk_list[i] if chunk_list else 10
        m_alloc = 10 if m == -1 else m
        cap = max(1, (a.size * 48 + 31) // 32)
        fields.append({
            "sym": sym, "nbins": nb, "chunk_log2": m,
            "out": torch.zeros(max(1, cap), dtype=torch.int32, device="cuda"),
            "offsets": torch.full((((a.size + (1 << m_alloc) - 1) >> m_alloc) + 1,), -1, dtype=torch.int64,
                                  device="cuda"),
            "total_bits": torch.full((1,), -1, dtype=torch.int64, device="cuda"),
        })
    return fields


def _check_field(plan, i, f, a, nb):
    import paper_2010_10039_gb300 as huff
    h = oracle.histogram(a, nb)
    assert np.array_equal(u32(plan.histogram(i, nb)), h), f"field {i}: histogram"
    want = oracle.codebook(h)
    got = huff.parse_codebook(plan.codebook(i, nb).cpu(), nb)
    assert got["status"] == 0
    assert got["max_len"] == want["max_len"], f"field {i}: max_len"
    assert np.array_equal(got["len"], want["len"]), f"field {i}: lengths"
    assert np.array_equal(got["code"], want["code"]), f"field {i}: codes"
    assert np.array_equal(got["sorted_syms"], want["sorted_syms"]), f"field {i}: sorted_syms"
    m = plan.chunk_log2(i)
    words, offs, tb = oracle.encode(a, want, chunk_log2=m)
    got_tb = int(f["total_bits"].item())
    assert got_tb == tb, f"field {i}: total_bits"
    nw = (tb + 31) // 32
    assert np.array_equal(u32(f["out"][:nw]) if nw else np.zeros(0, np.uint32), words), f"field {i}: stream"
    nch = ((a.size + (1 << m) - 1) >> m) + 1
    assert np.array_equal(u64(f["offsets"][:nch]), offs), f"field {i}: offsets"


def _run_and_check(fields_np, nbins_list, **kw):
    import paper_2010_10039_gb300 as huff
    import torch
    fields = _make(fields_np, nbins_list, kw.pop("chunk_list", None), kw.pop("offsets_elems", None))
    plan = huff.BatchPlan(fields, **kw)
    plan.encode()
    torch.cuda.synchronize()
    st = plan.status()
    assert st == [0] * len(fields), st
    for i, (f, a, nb) in enumerate(zip(fields, fields_np, nbins_list)):
        _check_field(plan, i, f, a, nb)
    return plan, fields


@pytest.mark.parametrize("form", [0, 1, 2])
def test_batch_u16_mixed_sizes_chunks_and_alignment(form):
    """Fields of very different sizes (empty, one symbol, sub-tile and tile
    boundaries, up to 1.5 M symbols), mixed chunk sizes and two unaligned
    inputs, all in one batch; with one persistent encode launch and with one
    launch per field."""
    sizes = [0, 1, 7, 4095, 4096, 4097, 8191, 8193, 32768, 32769, 65536 * 3 + 5, 1 << 20, 1_500_001,
             12345, 100_000, 2, 16, 17, 250_000, 777_777]
    fields_np = [_field_input(j, n, 1024, 2) for j, n in enumerate(sizes)]
    chunks = [10, 10, 4, 12, 10, 16, 10, 8, 10, 11, 10, 13, 10, 10, 20, 10, 4, 5, 10, 9]
    offs = [0] * len(sizes)
    offs[3] = 1
    offs[11] = 3
    plan, _ = _run_and_check(fields_np, [1024] * len(sizes), chunk_list=chunks, offsets_elems=offs,
                             encode_form=form)
    assert plan.info()["encode_form"] == form


@pytest.mark.parametrize("form", [0, 1, 2])
def test_batch_dtypes_and_alphabet_classes(form):
    """u8, u16 and u32 fields over small, medium (table in global memory) and
    large (packed histogram counters) alphabets in one plan: one launch group
    per dtype and alphabet class."""
    fields_np, nbs = [], []
    for j in range(4):
        fields_np.append(_field_input(j, 50_000 + 9_000 * j, 256, 1)); nbs.append(256)
    for j in range(3):
        fields_np.append(_field_input(10 + j, 70_000 + 11 * j, 4096, 2, b=40.0)); nbs.append(4096)
    for j, K in enumerate([8192, 65536]):
        p = synth.zipf_pmf(K, 1.1)
        fields_np.append(synth.draw(3, 20 + j, 300_000, synth.cdf_table(p), 4,
                                    mapping=synth.permutation(3, K))); nbs.append(K)
    for j in range(2):
        fields_np.append(_field_input(30 + j, 123_457, 16384, 4, b=300.0)); nbs.append(16384)
    plan, _ = _run_and_check(fields_np, nbs, encode_form=form)
    assert plan.info()["groups"] >= 4


def test_batch_autotune_gives_the_same_output_and_picks_chunks():
    """The tuner times candidate settings; outputs do not depend on them, and
    fields that leave M open get one of {10, 12, 14} with offsets to match."""
    sizes = [200_000, 3_000, 1_000_000, 65_536, 0, 333_333]
    fields_np = [_field_input(j, n, 1024, 2) for j, n in enumerate(sizes)]
    chunks = [-1, 10, -1, 12, -1, 10]
    plan, _ = _run_and_check(fields_np, [1024] * len(sizes), chunk_list=chunks, autotune=True)
    info = plan.info()
    assert info["candidates"] >= 6
    assert info["chunk_log2"] in (10, 12, 14)
    assert plan.chunk_log2(0) == info["chunk_log2"]
    assert plan.chunk_log2(1) == 10


@pytest.mark.parametrize("r,cap,ctas", [(2, 1, 1), (3, 2, 2), (3, 8, 3), (-1, 4, 0)])
def test_batch_settings_do_not_change_output(r, cap, ctas):
    sizes = [90_001, 4_096 * 5, 500_000, 31]
    fields_np = [_field_input(j, n, 1024, 2) for j, n in enumerate(sizes)]
    _run_and_check(fields_np, [1024] * len(sizes), reduce_log2=r, max_subtiles=cap, ctas_per_sm=ctas)


@pytest.mark.parametrize("form", [0, 1, 2])
def test_batch_long_codewords_next_to_short_ones(form):
    """Fields whose longest codewords have 24 to 28 bits (Fibonacci counts)
    among ordinary ones, and u8 / u32 fields with 28-bit codewords: the
    segment forms take the long codewords from the 64-bit codebook entries
    (up to the ring's worst-case tile: 27 bits for u16, 42 for u8, 48 for
    u32); the others stay with the general encoder."""
    fields_np, nbs = [], []
    for j, (dt, nb) in enumerate([(np.uint8, 256), (np.uint32, 4096)]):
        fib = [1, 1]
        while len(fib) < 29:
            fib.append(fib[-1] + fib[-2])
        ids = (np.arange(29, dtype=np.int64) * 7 + 3) % nb
        a = np.repeat(ids, fib).astype(dt)
        np.random.default_rng(100 + j).shuffle(a)
        fields_np.append(a)
        nbs.append(nb)
    for j, nsym in enumerate([25, 26, 28, 29]):
        fib = [1, 1]
        while len(fib) < nsym:
            fib.append(fib[-1] + fib[-2])
        ids = (np.arange(nsym, dtype=np.int64) * 37 + 5) % 1024
        a = np.repeat(ids, fib).astype(np.uint16)
        np.random.default_rng(j).shuffle(a)
        fields_np.append(a)
        nbs.append(1024)
    for j in range(3):
        fields_np.append(_field_input(40 + j, 200_000 + 7 * j, 1024, 2))
        nbs.append(1024)
    _run_and_check(fields_np, nbs, encode_form=form)


@pytest.mark.parametrize("form", [0, 1, 2])
def test_batch_rerun_with_new_contents(form):
    """The plan captures pointers: new data in the same buffers gives the new
    data's encoding on the next run."""
    import paper_2010_10039_gb300 as huff
    import torch
    sizes = [100_000, 50_000, 7]
    a1 = [_field_input(j, n, 1024, 2, seed=1) for j, n in enumerate(sizes)]
    a2 = [_field_input(j, n, 1024, 2, b=9.0, seed=2) for j, n in enumerate(sizes)]
    fields = _make(a1, [1024] * 3)
    plan = huff.BatchPlan(fields, encode_form=form)
    plan.encode()
    torch.cuda.synchronize()
    for i in range(3):
        _check_field(plan, i, fields[i], a1[i], 1024)
    for f, a in zip(fields, a2):
        f["sym"].copy_(to_dev(a))
    plan.encode()
    plan.encode()
    torch.cuda.synchronize()
    assert plan.status() == [0, 0, 0]
    for i in range(3):
        _check_field(plan, i, fields[i], a2[i], 1024)


@pytest.mark.parametrize("form", [0, 1, 2])
def test_batch_errors_stay_in_their_field(form):
    """A symbol beyond its field's alphabet and an output buffer that is too
    small each mark only their own field; the other fields are exact."""
    import paper_2010_10039_gb300 as huff
    import torch
    sizes = [60_000, 60_000, 60_000, 60_000]
    fields_np = [_field_input(j, n, 1024, 2) for j, n in enumerate(sizes)]
    bad = fields_np[1].copy()
    bad[12_345] = 1000          # >= nbins = 900 below
    fields_np[1] = bad
    nbs = [1024, 900, 1024, 1024]
    fields = _make(fields_np, nbs)
    fields[2]["out"] = fields[2]["out"][:100]     # far too small
    plan = huff.BatchPlan(fields, encode_form=form)
    plan.encode()
    torch.cuda.synchronize()
    st = plan.status()
    assert st[1] == huff.STATUS_CODE["HUFF_ERR_SYMBOL_RANGE"]
    assert st[2] == huff.STATUS_CODE["HUFF_ERR_CAPACITY"]
    assert st[0] == 0 and st[3] == 0
    for i in (0, 3):
        _check_field(plan, i, fields[i], fields_np[i], nbs[i])


def test_batch_more_than_one_group_of_fields():
    """600 fields of one class split into groups of at most 512."""
    rng = np.random.default_rng(5)
    sizes = [int(x) for x in rng.integers(1, 20_000, size=600)]
    fields_np = [_field_input(j, n, 1024, 2) for j, n in enumerate(sizes)]
    plan, _ = _run_and_check(fields_np, [1024] * len(sizes))
    assert plan.info()["groups"] == 2


@pytest.mark.parametrize("form", [0, 1, 2])
def test_batch_launch_count_per_run(form):
    import paper_2010_10039_gb300 as huff
    import torch
    fields_np = [_field_input(j, 10_000, 1024, 2) for j in range(3)] + [np.zeros(0, np.uint16)]
    fields = _make(fields_np, [1024] * 4)
    plan = huff.BatchPlan(fields, encode_form=form)
    k = plan.info()["kernels_per_run"]
    # histogram and codebooks, then the tile planner and one encode; or one encode per non-empty field; or
    # the planner, the entry tables, the segment encoder and the general encoder
    assert k == {0: 4, 1: 5, 2: 6}[form]
    c0 = huff.huff_launch_count()
    plan.encode()
    torch.cuda.synchronize()
    assert huff.huff_launch_count() - c0 == k


@pytest.mark.slow
def test_batch_full_size_workload_sampled_against_oracle():
    """The 512-field workload at full size (1.5 G u16 symbols, drawn on the
    device), tuned plan as the benchmark runs it; fields across the size
    range are checked against the oracle (regenerated on the host)."""
    import paper_2010_10039_gb300 as huff
    import torch
    prm = [synth.batch_field_params(j) for j in range(512)]
    fields = []
    for j, (n, b) in enumerate(prm):
        sym = synth.draw_device(4, j, n, synth.cdf_table(synth.laplace_pmf(1024, 512, b)), 2)
        fields.append({"sym": sym, "nbins": 1024, "chunk_log2": 10,
                       "out": torch.empty((n * 12 + 31) // 32 + 1, dtype=torch.int32, device="cuda"),
                       "offsets": torch.empty((n >> 10) + 2, dtype=torch.int64, device="cuda"),
                       "total_bits": torch.zeros(1, dtype=torch.int64, device="cuda")})
    plan = huff.BatchPlan(fields, autotune=True)
    plan.encode()
    torch.cuda.synchronize()
    assert plan.status() == [0] * 512
    order = sorted(range(512), key=lambda j: prm[j][0])
    for j in (order[0], order[1], order[256], order[400], 7):
        _check_field(plan, j, fields[j], synth.batch_field(j), 1024)
    plan.close()
