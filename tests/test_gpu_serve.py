"""Served form: jobs submitted together run as overlapping batches on the
device, and every job's codebook, stream and offsets equal those of the same
input encoded alone with the plain calls (and the oracle's)."""
import math
import time

import numpy as np
import pytest

import oracle
from paper_2010_10039_gb300 import synth
from gpu_util import Run, to_dev, u32, u64

pytestmark = pytest.mark.gpu


def _request(i, seed=5, n_lo=16384, n_hi=1 << 21):
    """Job i of a small mixed load: half u8 Zipf(1.2) over 256 ids, half u16
    Gaussian or Laplace over 1024 bins with scale log-uniform in [1, 64]."""
    u = [synth.u64_scalar(seed, 20000 + i, k) / 2.0 ** 64 for k in range(4)]
    n = int(round(math.exp(math.log(n_lo) + u[0] * (math.log(n_hi) - math.log(n_lo)))))
    if u[1] < 0.5:
        return synth.draw(seed, i, n, synth.cdf_table(synth.zipf_pmf(256, 1.2)), 1), 256
    scale = math.exp(u[2] * math.log(64.0))
    pmf = synth.gaussian_pmf(1024, 512, scale) if u[3] < 0.5 else synth.laplace_pmf(1024, 512, scale)
    return synth.draw(seed, i, n, synth.cdf_table(pmf), 2), 1024


def _result_arrays(huff, res, n, nbins):
    tb = res["total_bits"]
    nw = (tb + 31) // 32
    words = u32(huff.device_view(res["d_out"], 4 * nw)) if nw else np.zeros(0, np.uint32)
    m = res["chunk_log2"]
    nch = ((n + (1 << m) - 1) >> m) + 1
    offs = u64(huff.device_view(res["d_chunk_bit_offset"], 8 * nch))
    book = huff.parse_codebook(huff.device_view(res["d_codebook"], huff.huff_codebook_bytes(nbins)).cpu(), nbins)
    return words, offs, book, tb


def test_serve_mix_equals_alone():
    import paper_2010_10039_gb300 as huff
    import torch
    jobs = [_request(i) for i in range(40)]
    dev = [to_dev(a) for a, _ in jobs]
    srv = huff.Server(mem_budget_bytes=1 << 30, nstreams=3, max_batch=6)
    try:
        tickets = [srv.submit(d, nb) for d, (_, nb) in zip(dev, jobs)]
        results = [srv.wait(t) for t in tickets]
        st = srv.stats()
        assert st["completed"] == 40 and st["batches"] >= 7
        for (a, nb), res, t in zip(jobs, results, tickets):
            assert res["status"] == 0
            words, offs, book, tb = _result_arrays(huff, res, a.size, nb)
            alone = Run(a, nb, chunk_log2=res["chunk_log2"]).all()
            assert alone.status() == 0
            aw, atb = alone.stream_np()
            assert tb == atb and np.array_equal(words, aw), "stream differs from the job alone"
            assert np.array_equal(offs, alone.offs_np()), "offsets differ from the job alone"
            assert np.array_equal(book["cw"], alone.book_np()["cw"]), "codebook differs from the job alone"
            assert res["t_submit"] <= res["t_admit"] <= res["t_launch"] <= res["t_done"]
            srv.release(t)
        # a few of them against the oracle as well
        for (a, nb) in jobs[:6]:
            h = oracle.histogram(a, nb)
            want = oracle.codebook(h)
            w, o, tb = oracle.encode(a, want, chunk_log2=10)
            alone = Run(a, nb).all()
            gw, gtb = alone.stream_np()
            assert gtb == tb and np.array_equal(gw, w)
        assert srv.stats()["pool_used"] == 0
    finally:
        srv.close()
    torch.cuda.synchronize()


def test_serve_admits_by_memory_budget():
    """A budget for about two jobs: later jobs are admitted only after earlier
    ones are released, and all results are still exact."""
    import paper_2010_10039_gb300 as huff
    jobs = [_request(100 + i, n_lo=200_000, n_hi=300_000) for i in range(8)]
    dev = [to_dev(a) for a, _ in jobs]
    one = 4 * ((300_000 * 10 + 31) // 32 + 1) + 8 * (300_000 // 1024 + 2) + huff.huff_codebook_bytes(1024) + 1024
    srv = huff.Server(mem_budget_bytes=2 * one + 4096, nstreams=2, max_batch=4)
    try:
        tickets = [srv.submit(d, nb) for d, (_, nb) in zip(dev, jobs)]
        done = []
        for (a, nb), t in zip(jobs, tickets):
            res = srv.wait(t)
            assert res["status"] == 0
            words, offs, book, tb = _result_arrays(huff, res, a.size, nb)
            h = oracle.histogram(a, nb)
            want = oracle.codebook(h)
            w, o, otb = oracle.encode(a, want, chunk_log2=10)
            assert tb == otb and np.array_equal(words, w) and np.array_equal(offs, o)
            done.append(res)
            srv.release(t)
        st = srv.stats()
        assert st["pool_peak"] <= st["pool_capacity"]
        # the last jobs could only be admitted after the first ones were released
        assert done[-1]["t_admit"] >= done[0]["t_done"]
    finally:
        srv.close()


def test_serve_rejects_and_limits():
    import paper_2010_10039_gb300 as huff
    import torch
    srv = huff.Server(mem_budget_bytes=1 << 20, max_queue=1, nstreams=1)
    try:
        x = torch.zeros(1000, dtype=torch.int16, device="cuda")
        code = huff.STATUS_CODE
        assert srv.submit_raw(x.data_ptr(), 0, huff.HUFF_U16, 1024)[0] == code["HUFF_ERR_INVALID_ARG"]
        assert srv.submit_raw(x.data_ptr(), 1000, huff.HUFF_U8, 300)[0] == code["HUFF_ERR_INVALID_ARG"]
        assert srv.submit_raw(x.data_ptr() + 1, 100, huff.HUFF_U16, 1024)[0] == code["HUFF_ERR_INVALID_ARG"]
        big = torch.zeros(1 << 22, dtype=torch.int16, device="cuda")
        assert srv.submit_raw(big.data_ptr(), big.numel(), huff.HUFF_U16, 1024)[0] == code["HUFF_ERR_OOM"]
        # one job fills the budget, the next waits in the queue, the one after is refused
        half = torch.zeros(300_000, dtype=torch.int16, device="cuda")
        seen_busy = False
        tickets = []
        for _ in range(4):
            rc, t = srv.submit_raw(half.data_ptr(), half.numel(), huff.HUFF_U16, 1024)
            if rc == code["HUFF_ERR_BUSY"]:
                seen_busy = True
                break
            assert rc == 0
            tickets.append(t)
        assert seen_busy
        for t in tickets:
            res = srv.wait(t)
            assert res["status"] == 0 and res["total_bits"] == 300_000      # one symbol used: 1 bit each
            srv.release(t)
        # released before completion: the ticket is gone, the memory returns
        t = srv.submit(half, 1024)
        srv.release(t)
        with pytest.raises(huff.HuffError) as e:
            srv.poll(t)
        assert e.value.name == "HUFF_ERR_NOT_FOUND"
        with pytest.raises(huff.HuffError):
            srv.wait(t)
        deadline = time.time() + 30
        while srv.stats()["pool_used"] and time.time() < deadline:
            time.sleep(0.01)
        assert srv.stats()["pool_used"] == 0
    finally:
        srv.close()


def test_serve_destroy_with_pending_jobs():
    """Destroying a server with queued and running jobs cancels the queued
    ones, waits for the running ones and leaves the device usable."""
    import paper_2010_10039_gb300 as huff
    jobs = [_request(200 + i, n_lo=1 << 20, n_hi=1 << 21) for i in range(12)]
    dev = [to_dev(a) for a, _ in jobs]
    srv = huff.Server(mem_budget_bytes=8 << 20, nstreams=2, max_batch=2)
    for d, (_, nb) in zip(dev, jobs):
        srv.submit(d, nb)
    t0 = time.time()
    srv.close()
    assert time.time() - t0 < 30
    a, nb = jobs[0]
    r = Run(a, nb).all()
    assert r.status() == 0


@pytest.mark.slow
def test_serve_full_size_requests_sampled_against_oracle():
    """Requests of the served workload at full size (n up to 67 M; u8 Zipf
    and u16 Gaussian/Laplace), drawn on the device and submitted together;
    the small ones are re-encoded by the oracle, every job equals its plain
    single call."""
    import paper_2010_10039_gb300 as huff
    import torch
    reqs = [synth.served_request(i) for i in range(48)]
    dev = [synth.draw_device(5, 100 + i, n, table, w) for i, (w, n, nb, table) in enumerate(reqs)]
    srv = huff.Server(mem_budget_bytes=8 << 30, nstreams=4, max_batch=64)
    try:
        tickets = [srv.submit(d, r[2]) for d, r in zip(dev, reqs)]
        res = [srv.wait(t) for t in tickets]
        assert all(r["status"] == 0 for r in res)
        small = [i for i, r in enumerate(reqs) if r[1] <= (1 << 21)][:4]
        assert small
        for i in small:
            a = synth.served_symbols(i)
            nb = reqs[i][2]
            words, offs, book, tb = _result_arrays(huff, res[i], a.size, nb)
            want = oracle.codebook(oracle.histogram(a, nb))
            w, o, otb = oracle.encode(a, want, chunk_log2=10)
            assert tb == otb and np.array_equal(words, w) and np.array_equal(offs, o)
        for i in (0, 1, 2, int(np.argmax([r[1] for r in reqs]))):
            run = Run(dev[i].cpu().numpy().view({1: np.uint8, 2: np.uint16}[reqs[i][0]]), reqs[i][2]).all()
            assert run.status() == 0
            gw, gtb = run.stream_np()
            words, offs, book, tb = _result_arrays(huff, res[i], reqs[i][1], reqs[i][2])
            assert tb == gtb and np.array_equal(words, gw) and np.array_equal(offs, run.offs_np())
        for t in tickets:
            srv.release(t)
    finally:
        srv.close()
