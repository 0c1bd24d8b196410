"""Bounded device waits end in HUFF_ERR_TIMEOUT instead of a hang.

huff_encode_fault_test runs the encoder with tile 0 never encoded, so the
decoupled look-back of tile 1 waits on a descriptor that nobody publishes.
With a short poll limit that wait must give up: the call returns, the
workspace status reads HUFF_ERR_TIMEOUT, nothing is written past the output
capacity, and the context stays usable (a normal encode on the same
workspace afterwards is bit-exact with one on a fresh workspace)."""
import time

import numpy as np
import pytest

from paper_2010_10039_gb300 import synth
from gpu_util import Run, u32, u64

HUFF_ERR_TIMEOUT = 6
CANARY = 0x5A5A5A5A


@pytest.mark.gpu
@pytest.mark.parametrize("poll_limit", [1, 1024])
def test_lookback_gives_up_with_timeout(poll_limit):
    import torch
    import paper_2010_10039_gb300 as huff
    sym_np = synth.laplace_field(2_000_003, seed=41)
    ref = Run(sym_np, 1024).all()
    assert ref.status() == 0
    tb = int(ref.total.item())

    cap = ref.cap
    slack = 4096
    big = torch.full((cap + slack,), CANARY, dtype=torch.int32, device="cuda")
    out = big[:cap]
    offs = torch.full_like(ref.offs, -1)
    total = torch.full_like(ref.total, -1)
    huff.huff_workspace_init(ref.ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    huff.huff_encode_fault_test(ref.sym, ref.book, 1024, out, offs, total, ref.ws, poll_limit)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    assert ref.status() == HUFF_ERR_TIMEOUT
    assert dt < 10.0, f"faulted launch took {dt:.1f} s"
    assert (u32(big[cap:]) == np.uint32(CANARY)).all(), "write past the output capacity"

    # the context and the workspace stay usable
    huff.huff_workspace_init(ref.ws)
    out2 = torch.full_like(ref.out, CANARY)
    offs2 = torch.full_like(ref.offs, -1)
    total2 = torch.full_like(ref.total, -1)
    huff.huff_encode(ref.sym, ref.book, 1024, out2, offs2, total2, ref.ws, ref.params, capacity_words=cap)
    assert ref.status() == 0
    assert int(total2.item()) == tb
    nw = (tb + 31) // 32
    assert (u32(out2[:nw]) == u32(ref.out[:nw])).all()
    assert (u64(offs2) == u64(ref.offs)).all()


@pytest.mark.gpu
def test_fault_hook_rejects_bad_arguments():
    import torch
    import paper_2010_10039_gb300 as huff
    sym_np = synth.laplace_field(100_000, seed=42)
    r = Run(sym_np, 1024).all()
    L = huff.lib()
    args = lambda n, lim: (r.sym.data_ptr(), n, huff.HUFF_U16, r.book.data_ptr(), 1024, r.out.data_ptr(), r.cap,
                           r.offs.data_ptr(), r.total.data_ptr(), lim, r.ws.data_ptr(), None)
    assert L.huff_encode_fault_test(*args(sym_np.size, 0)) == 1            # poll limit 0
    assert L.huff_encode_fault_test(*args(sym_np.size, (1 << 22) + 1)) == 1
    assert L.huff_encode_fault_test(*args(1000, 16)) == 1                  # a single tile: no tile 1
    torch.cuda.synchronize()
    assert r.status() == 0
