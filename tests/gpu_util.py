"""Helpers for the GPU parity tests: move numpy inputs to the device, run the
C-ABI through the Python binding, bring results back as numpy."""
import numpy as np

TORCH_VIEW = {1: np.uint8, 2: np.int16, 4: np.int32}


def to_dev(a: np.ndarray, offset_elems: int = 0):
    """Device copy of a; with offset_elems > 0 the data starts that many
    elements into a larger allocation (to exercise unaligned inputs)."""
    import torch
    w = a.dtype.itemsize
    if w == 1:
        host = torch.from_numpy(np.ascontiguousarray(a))
    else:
        host = torch.from_numpy(np.ascontiguousarray(a).view(TORCH_VIEW[w]))
    if offset_elems == 0:
        return host.cuda()
    big = torch.zeros(a.size + offset_elems, dtype=host.dtype, device="cuda")
    big[offset_elems:] = host.cuda()
    return big[offset_elems:]


def u32(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


def u64(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


class Run:
    """Buffers + one pass of histogram/codebook/encode through the C-ABI."""

    def __init__(self, sym_np: np.ndarray, nbins: int, chunk_log2: int = 10, offset_elems: int = 0,
                 params=None, cap_words=None):
        import torch
        import paper_2010_10039_gb300 as huff
        self.huff = huff
        self.sym_np = sym_np
        self.n = sym_np.size
        self.nbins = nbins
        self.chunk_log2 = chunk_log2
        prm = {"chunk_log2": chunk_log2}
        if params:
            prm.update(params)
        self.params = prm
        self.sym = to_dev(sym_np, offset_elems) if self.n else torch.empty(0, dtype=torch.int16, device="cuda")
        self.dtype = sym_np.dtype.itemsize
        self.hist = torch.empty(nbins, dtype=torch.int32, device="cuda")
        self.book = torch.empty(huff.huff_codebook_bytes(nbins), dtype=torch.uint8, device="cuda")
        self.ws = torch.zeros(huff.huff_workspace_bytes(max(1, self.n), nbins, prm), dtype=torch.uint8, device="cuda")
        huff.huff_workspace_init(self.ws)
        cap = cap_words if cap_words is not None else max(1, huff.huff_max_output_words(self.n, 48))
        self.out = torch.zeros(max(1, cap), dtype=torch.int32, device="cuda")
        self.cap = cap
        nch = (self.n + (1 << chunk_log2) - 1) >> chunk_log2
        self.offs = torch.full((nch + 1,), -1, dtype=torch.int64, device="cuda")
        self.total = torch.full((1,), -1, dtype=torch.int64, device="cuda")

    def histogram(self):
        self.huff.huff_histogram(self.sym, self.nbins, self.hist, self.ws, n=self.n, dtype=self.dtype)
        return self

    def codebook(self, hist_dev=None):
        self.huff.huff_build_codebook(self.hist if hist_dev is None else hist_dev, self.nbins, self.book, self.ws)
        return self

    def encode(self):
        self.huff.huff_encode(self.sym, self.book, self.nbins, self.out, self.offs, self.total, self.ws,
                              self.params, n=self.n, dtype=self.dtype, capacity_words=self.cap)
        return self

    def all(self):
        return self.histogram().codebook().encode()

    def status(self) -> int:
        return self.huff.huff_get_status(self.ws)

    def hist_np(self):
        return u32(self.hist)

    def book_np(self):
        return self.huff.parse_codebook(self.book.cpu(), self.nbins)

    def stream_np(self):
        tb = int(self.total.item())
        return u32(self.out[: (tb + 31) // 32]) if tb else np.zeros(0, np.uint32), tb

    def offs_np(self):
        return u64(self.offs)
