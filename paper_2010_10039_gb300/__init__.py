"""Python binding of libhuff (GPU Huffman encoding for sm_103a).

The functions below carry the names of the C-ABI in ``include/huff.h`` and
only marshal arguments: torch tensors become device pointers, the current
torch stream becomes the cudaStream_t, and a non-OK status raises
``HuffError``.  Every step of the pipeline runs in the library's CUDA kernels;
there is no CPU fallback.  If ``libhuff.so`` is missing, calls raise.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhuff.so")

HUFF_U8, HUFF_U16, HUFF_U32 = 1, 2, 4
HUFF_MERGE_AUTO, HUFF_MERGE_SCAN, HUFF_MERGE_SHUFFLE = 0, 1, 2
HUFF_MAX_LEN = 64
HUFF_CW_LEN_SHIFT = 58
CODEBOOK_HEADER_BYTES = 1072

STATUS = {
    0: "HUFF_OK", 1: "HUFF_ERR_INVALID_ARG", 2: "HUFF_ERR_SYMBOL_RANGE", 3: "HUFF_ERR_NOT_IN_CODEBOOK",
    4: "HUFF_ERR_CAPACITY", 5: "HUFF_ERR_OOM", 6: "HUFF_ERR_TIMEOUT", 7: "HUFF_ERR_BUSY", 8: "HUFF_ERR_CUDA",
    9: "HUFF_ERR_HIST_OVERFLOW", 10: "HUFF_ERR_NOT_FOUND", 11: "HUFF_ERR_CANCELLED",
}
STATUS_CODE = {v: k for k, v in STATUS.items()}


class HuffError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        self.code = code
        self.name = STATUS.get(code, str(code))
        super().__init__(f"{where}: {self.name}" if where else self.name)


class huff_params(ctypes.Structure):
    _fields_ = [("chunk_log2", ctypes.c_int32), ("reduce_log2", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("merge", ctypes.c_int32),
                ("word_bits", ctypes.c_int32), ("layout", ctypes.c_int32)]


HUFF_LAYOUT_DENSE = 0
HUFF_LAYOUT_CHUNK_ALIGNED = 1


class huff_field(ctypes.Structure):
    _fields_ = [("d_sym", ctypes.c_void_p), ("n", ctypes.c_uint64), ("dtype", ctypes.c_int32),
                ("nbins", ctypes.c_uint32), ("chunk_log2", ctypes.c_int32), ("reserved", ctypes.c_uint32),
                ("d_out", ctypes.c_void_p), ("out_capacity_words", ctypes.c_uint64),
                ("d_chunk_bit_offset", ctypes.c_void_p), ("d_total_bits", ctypes.c_void_p)]


class huff_batch_cfg(ctypes.Structure):
    _fields_ = [("autotune", ctypes.c_int32), ("reduce_log2", ctypes.c_int32),
                ("max_subtiles", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("encode_form", ctypes.c_int32)]


class huff_batch_info(ctypes.Structure):
    _fields_ = [("reduce_log2", ctypes.c_int32), ("max_subtiles", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("chunk_log2", ctypes.c_int32), ("groups", ctypes.c_uint32), ("kernels_per_run", ctypes.c_uint32),
                ("candidates", ctypes.c_uint32), ("tuned_ms", ctypes.c_float), ("device_bytes", ctypes.c_uint64),
                ("encode_form", ctypes.c_uint32), ("per_field_tiles", ctypes.c_uint32)]


class huff_serve_cfg(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_uint64), ("max_inflight", ctypes.c_uint32),
                ("nstreams", ctypes.c_uint32), ("max_batch", ctypes.c_uint32), ("chunk_log2", ctypes.c_int32),
                ("max_batch_symbols", ctypes.c_uint64), ("max_queue", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class huff_request(ctypes.Structure):
    _fields_ = [("d_sym", ctypes.c_void_p), ("n", ctypes.c_uint64), ("dtype", ctypes.c_int32),
                ("nbins", ctypes.c_uint32)]


class huff_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("chunk_log2", ctypes.c_int32), ("total_bits", ctypes.c_uint64),
                ("d_out", ctypes.c_void_p), ("d_chunk_bit_offset", ctypes.c_void_p), ("d_codebook", ctypes.c_void_p),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_launch", ctypes.c_double),
                ("t_done", ctypes.c_double)]


class huff_serve_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("cancelled", ctypes.c_uint64),
                ("batches", ctypes.c_uint64), ("max_batch_jobs", ctypes.c_uint64),
                ("max_concurrent_batches", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("pool_used", ctypes.c_uint64), ("pool_peak", ctypes.c_uint64), ("pool_capacity", ctypes.c_uint64),
                ("symbols_done", ctypes.c_uint64)]


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded libhuff.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libhuff.so is not built ({LIB_PATH}); run paper_2010_10039_gb300/build.py "
                               "or __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, u64, u32, i32, sz = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_size_t
        P = ctypes.POINTER(huff_params)
        sig = {
            "huff_default_params": (None, [P]),
            "huff_reduce_factor": (i32, [ctypes.c_double, i32]),
            "huff_codebook_bytes": (sz, [u32]),
            "huff_max_output_words": (u64, [u64, u32]),
            "huff_max_output_units": (u64, [u64, u32, P]),
            "huff_workspace_bytes": (sz, [u64, u32, P]),
            "huff_workspace_init": (i32, [vp, vp]),
            "huff_histogram": (i32, [vp, u64, i32, u32, vp, vp, vp]),
            "huff_build_codebook": (i32, [vp, u32, vp, vp, vp]),
            "huff_encode": (i32, [vp, u64, i32, vp, u32, P, vp, u64, vp, vp, vp, vp]),
            "huff_decode": (i32, [vp, u64, vp, i32, u64, i32, vp, u32, vp, vp, vp]),
            "huff_decode_ex": (i32, [vp, u64, vp, P, u64, i32, vp, u32, vp, vp, vp]),
            "huff_encode_noalloc": (i32, [vp, u64, i32, vp, u32, P, vp, u64, vp, vp, vp, vp]),
            "huff_encode_fault_test": (i32, [vp, u64, i32, vp, u32, vp, u64, vp, vp, u32, vp, vp]),
            "huff_get_status": (i32, [vp, vp]),
            "huff_status_string": (ctypes.c_char_p, [i32]),
            "huff_launch_count": (u64, []),
            "huff_batch_default_cfg": (None, [ctypes.POINTER(huff_batch_cfg)]),
            "huff_batch_plan_create": (i32, [ctypes.POINTER(huff_field), u32, ctypes.POINTER(huff_batch_cfg), vp,
                                             ctypes.POINTER(vp)]),
            "huff_batch_encode": (i32, [vp, vp]),
            "huff_batch_status": (i32, [vp, ctypes.POINTER(u32), vp]),
            "huff_batch_profile": (i32, [vp, vp, ctypes.POINTER(ctypes.c_float)]),
            "huff_batch_get_info": (i32, [vp, ctypes.POINTER(huff_batch_info)]),
            "huff_batch_codebook": (vp, [vp, u32]),
            "huff_batch_histogram": (vp, [vp, u32]),
            "huff_batch_chunk_log2": (i32, [vp, u32]),
            "huff_batch_plan_destroy": (None, [vp]),
            "huff_serve_default_cfg": (None, [ctypes.POINTER(huff_serve_cfg)]),
            "huff_serve_create": (i32, [ctypes.POINTER(huff_serve_cfg), ctypes.POINTER(vp)]),
            "huff_serve_submit": (i32, [vp, ctypes.POINTER(huff_request), ctypes.POINTER(u64)]),
            "huff_serve_poll": (i32, [vp, u64, ctypes.POINTER(huff_result)]),
            "huff_serve_wait": (i32, [vp, u64, ctypes.POINTER(huff_result)]),
            "huff_serve_release": (i32, [vp, u64]),
            "huff_serve_get_stats": (i32, [vp, ctypes.POINTER(huff_serve_stats)]),
            "huff_serve_destroy": (i32, [vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


# ------------------------------------------------------------------ helpers

def _torch():
    import torch
    return torch


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        torch = _torch()
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def dtype_code(t) -> int:
    """HUFF_U8/U16/U32 for a tensor's element size."""
    torch = _torch()
    size = t.element_size()
    if t.dtype.is_floating_point or t.dtype == torch.bool or size not in (1, 2, 4):
        raise TypeError(f"symbols must be 1/2/4-byte integers, got {t.dtype}")
    return size


def _check(rc: int, where: str) -> None:
    if rc != 0:
        raise HuffError(rc, where)


def _params(p) -> huff_params:
    if isinstance(p, huff_params):
        return p
    q = huff_params()
    lib().huff_default_params(ctypes.byref(q))
    if p:
        for k, v in dict(p).items():
            setattr(q, k, int(v))
    return q


# ------------------------------------------------------------------ C-ABI mirrors

def huff_default_params() -> huff_params:
    return _params(None)


def huff_reduce_factor(avg_bits: float, word_bits: int = 32) -> int:
    return lib().huff_reduce_factor(float(avg_bits), int(word_bits))


def huff_codebook_bytes(nbins: int) -> int:
    return lib().huff_codebook_bytes(nbins)


def huff_max_output_words(n: int, max_len: int) -> int:
    return lib().huff_max_output_words(n, max_len)


def huff_max_output_units(n: int, max_len: int, params=None) -> int:
    return lib().huff_max_output_units(n, max_len, ctypes.byref(_params(params)))


def huff_workspace_bytes(n: int, nbins: int, params=None) -> int:
    return lib().huff_workspace_bytes(n, nbins, ctypes.byref(_params(params)))


def huff_workspace_init(ws, stream=None) -> None:
    _check(lib().huff_workspace_init(_ptr(ws), _stream(stream)), "huff_workspace_init")


def huff_histogram(sym, nbins: int, hist, ws, stream=None, n: int | None = None, dtype: int | None = None) -> None:
    n = sym.numel() if n is None else n
    dt = dtype_code(sym) if dtype is None else dtype
    _check(lib().huff_histogram(_ptr(sym), n, dt, nbins, _ptr(hist), _ptr(ws), _stream(stream)), "huff_histogram")


def huff_build_codebook(hist, nbins: int, codebook, ws, stream=None) -> None:
    _check(lib().huff_build_codebook(_ptr(hist), nbins, _ptr(codebook), _ptr(ws), _stream(stream)),
           "huff_build_codebook")


def huff_encode(sym, codebook, nbins: int, out, offsets, total_bits, ws, params=None, stream=None,
                n: int | None = None, dtype: int | None = None, capacity_words: int | None = None) -> None:
    n = sym.numel() if n is None else n
    dt = dtype_code(sym) if dtype is None else dtype
    cap = out.numel() if capacity_words is None else capacity_words
    p = _params(params)
    _check(lib().huff_encode(_ptr(sym), n, dt, _ptr(codebook), nbins, ctypes.byref(p), _ptr(out), cap,
                             _ptr(offsets), _ptr(total_bits), _ptr(ws), _stream(stream)), "huff_encode")


def huff_encode_noalloc(sym, codebook, nbins: int, out, offsets, total_bits, status, params=None, stream=None,
                        n: int | None = None, dtype: int | None = None, capacity_words: int | None = None) -> None:
    """huff_encode with the library's fixed scratch instead of a workspace
    (for callers that cannot allocate device memory); `status` is one device
    uint32 that receives the first device error."""
    n = sym.numel() if n is None else n
    dt = dtype_code(sym) if dtype is None else dtype
    cap = out.numel() if capacity_words is None else capacity_words
    p = _params(params)
    _check(lib().huff_encode_noalloc(_ptr(sym), n, dt, _ptr(codebook), nbins, ctypes.byref(p), _ptr(out), cap,
                                     _ptr(offsets), _ptr(total_bits), _ptr(status), _stream(stream)),
           "huff_encode_noalloc")


def huff_encode_fault_test(sym, codebook, nbins: int, out, offsets, total_bits, ws, poll_limit: int,
                           stream=None) -> None:
    """Failure-detection hook: an encode whose tile 0 is never encoded and
    whose look-back gives up after `poll_limit` polls; the workspace status
    then reads HUFF_ERR_TIMEOUT."""
    _check(lib().huff_encode_fault_test(_ptr(sym), sym.numel(), dtype_code(sym), _ptr(codebook), nbins, _ptr(out),
                                        out.numel(), _ptr(offsets), _ptr(total_bits), poll_limit, _ptr(ws),
                                        _stream(stream)), "huff_encode_fault_test")


def huff_decode(stream_words, total_bits: int, offsets, chunk_log2: int, n: int, dtype: int, codebook, nbins: int,
                out, ws, stream=None) -> None:
    _check(lib().huff_decode(_ptr(stream_words), total_bits, _ptr(offsets), chunk_log2, n, dtype, _ptr(codebook),
                             nbins, _ptr(out), _ptr(ws), _stream(stream)), "huff_decode")


def huff_decode_ex(stream_units, total_bits: int, offsets, params, n: int, dtype: int, codebook, nbins: int,
                   out, ws, stream=None) -> None:
    p = _params(params)
    _check(lib().huff_decode_ex(_ptr(stream_units), total_bits, _ptr(offsets), ctypes.byref(p), n, dtype,
                                _ptr(codebook), nbins, _ptr(out), _ptr(ws), _stream(stream)), "huff_decode_ex")


def huff_get_status(ws, stream=None) -> int:
    return lib().huff_get_status(_ptr(ws), _stream(stream))


def huff_status_string(code: int) -> str:
    return lib().huff_status_string(code).decode()


def huff_launch_count() -> int:
    return lib().huff_launch_count()


# ------------------------------------------------------------------ codebook view

def parse_codebook(buf_cpu, nbins: int) -> dict:
    """Splits a codebook buffer copied to the host (uint8 tensor or numpy array)
    into its fields (layout of include/huff.h)."""
    import numpy as np
    b = np.asarray(buf_cpu.cpu().numpy() if hasattr(buf_cpu, "cpu") else buf_cpu, dtype=np.uint8)
    hdr = b[:CODEBOOK_HEADER_BYTES]
    u32 = hdr.view(np.uint32)
    out = {"nbins": int(u32[0]), "max_len": int(u32[1])}
    out["first"] = hdr[8:8 + 520].view(np.uint64).copy()
    out["entry"] = hdr[528:528 + 260].view(np.uint32).copy()
    out["count"] = hdr[788:788 + 260].view(np.uint32).copy()
    out["nused"] = int(hdr[1048:1052].view(np.uint32)[0])
    out["status"] = int(hdr[1052:1056].view(np.uint32)[0])
    out["total_bits"] = int(hdr[1056:1064].view(np.uint64)[0])
    out["nsymbols"] = int(hdr[1064:1072].view(np.uint64)[0])
    cw = b[CODEBOOK_HEADER_BYTES:CODEBOOK_HEADER_BYTES + 8 * nbins].view(np.uint64).copy()
    out["cw"] = cw
    out["len"] = (cw >> np.uint64(HUFF_CW_LEN_SHIFT)).astype(np.uint8)
    out["code"] = cw & np.uint64((1 << HUFF_CW_LEN_SHIFT) - 1)
    ss = b[CODEBOOK_HEADER_BYTES + 8 * nbins:CODEBOOK_HEADER_BYTES + 12 * nbins].view(np.uint32)
    out["sorted_syms"] = ss[:out["nused"]].copy()
    return out


# ------------------------------------------------------------------ whole pipeline

class Pipeline:
    """Device buffers (torch allocations) for histogram -> codebook -> encode of
    inputs up to ``max_n`` symbols over ``nbins`` bins, reused across calls."""

    def __init__(self, max_n: int, nbins: int, params=None, device="cuda", max_len_bound: int = 48):
        torch = _torch()
        self.nbins = nbins
        self.params = _params(params)
        self.max_n = max_n
        self.device = torch.device(device)
        self.hist = torch.empty(nbins, dtype=torch.int32, device=self.device)
        self.codebook = torch.empty(huff_codebook_bytes(nbins), dtype=torch.uint8, device=self.device)
        self.ws = torch.zeros(huff_workspace_bytes(max_n, nbins, self.params), dtype=torch.uint8, device=self.device)
        # the stream's units (W = params.word_bits bits each), in whole 32-bit words
        W = self.params.word_bits or 32
        self.cap_units = max(1, huff_max_output_units(max_n, max_len_bound, self.params))
        self.out = torch.empty((self.cap_units * W + 31) // 32, dtype=torch.int32, device=self.device)
        nch = (max_n + (1 << self.params.chunk_log2) - 1) >> self.params.chunk_log2
        self.offsets = torch.empty(nch + 1, dtype=torch.int64, device=self.device)
        self.total_bits = torch.zeros(1, dtype=torch.int64, device=self.device)
        huff_workspace_init(self.ws)

    def run(self, sym, stream=None, stages=("hist", "codebook", "encode")) -> None:
        n = sym.numel()
        if n > self.max_n:
            raise ValueError("input larger than the pipeline was sized for")
        if "hist" in stages:
            huff_histogram(sym, self.nbins, self.hist, self.ws, stream)
        if "codebook" in stages:
            huff_build_codebook(self.hist, self.nbins, self.codebook, self.ws, stream)
        if "encode" in stages:
            huff_encode(sym, self.codebook, self.nbins, self.out, self.offsets, self.total_bits, self.ws,
                        self.params, stream, capacity_words=self.cap_units)

    def status(self, stream=None) -> int:
        return huff_get_status(self.ws, stream)


# ------------------------------------------------------------------ batched form

class BatchPlan:
    """huff_batch_plan over a list of fields.  Each field is a dict with
    ``sym`` (1-D integer tensor on the device), ``nbins``, ``out`` (int32
    tensor), ``offsets`` (int64 tensor), ``total_bits`` (int64 tensor of one
    element) and optionally ``chunk_log2`` (default 10; -1 lets the plan
    choose).  The tensors must outlive the plan."""

    def __init__(self, fields, autotune: bool = False, reduce_log2: int = -1, max_subtiles: int = 0,
                 ctas_per_sm: int = 0, encode_form: int = 0, stream=None):
        self._keep = fields
        self.n = len(fields)
        arr = (huff_field * self.n)()
        for i, f in enumerate(fields):
            sym = f["sym"]
            arr[i].d_sym = _ptr(sym)
            arr[i].n = sym.numel()
            arr[i].dtype = dtype_code(sym)
            arr[i].nbins = int(f["nbins"])
            arr[i].chunk_log2 = int(f.get("chunk_log2", 10))
            arr[i].d_out = _ptr(f["out"])
            arr[i].out_capacity_words = f["out"].numel()
            arr[i].d_chunk_bit_offset = _ptr(f["offsets"])
            arr[i].d_total_bits = _ptr(f["total_bits"])
        cfg = huff_batch_cfg()
        lib().huff_batch_default_cfg(ctypes.byref(cfg))
        cfg.autotune = 1 if autotune else 0
        cfg.reduce_log2 = reduce_log2
        cfg.max_subtiles = max_subtiles
        cfg.ctas_per_sm = ctas_per_sm
        cfg.encode_form = encode_form
        h = ctypes.c_void_p()
        _check(lib().huff_batch_plan_create(arr, self.n, ctypes.byref(cfg), _stream(stream), ctypes.byref(h)),
               "huff_batch_plan_create")
        self.handle = h

    def encode(self, stream=None) -> None:
        _check(lib().huff_batch_encode(self.handle, _stream(stream)), "huff_batch_encode")

    def profile(self, stream=None) -> dict:
        """One run without the graph, with per-stage device times (ms)."""
        ms = (ctypes.c_float * 4)()
        _check(lib().huff_batch_profile(self.handle, _stream(stream), ms), "huff_batch_profile")
        return {"histogram": ms[0], "codebook": ms[1], "plan": ms[2], "encode": ms[3]}

    def status(self, stream=None) -> list[int]:
        st = (ctypes.c_uint32 * self.n)()
        _check(lib().huff_batch_status(self.handle, st, _stream(stream)), "huff_batch_status")
        return list(st)

    def info(self) -> dict:
        inf = huff_batch_info()
        _check(lib().huff_batch_get_info(self.handle, ctypes.byref(inf)), "huff_batch_get_info")
        return {k: getattr(inf, k) for k, _ in huff_batch_info._fields_}

    def codebook_ptr(self, i: int) -> int:
        return lib().huff_batch_codebook(self.handle, i)

    def histogram_ptr(self, i: int) -> int:
        return lib().huff_batch_histogram(self.handle, i)

    def chunk_log2(self, i: int) -> int:
        return lib().huff_batch_chunk_log2(self.handle, i)

    def codebook(self, i: int, nbins: int):
        """Field i's codebook buffer (plan memory) as a device uint8 tensor view."""
        return device_view(self.codebook_ptr(i), huff_codebook_bytes(nbins))

    def histogram(self, i: int, nbins: int):
        """Field i's histogram (plan memory) as a device int32 tensor view."""
        return device_view(self.histogram_ptr(i), 4 * nbins).view(_torch().int32)

    def close(self) -> None:
        if getattr(self, "handle", None):
            lib().huff_batch_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _DeviceBytes:
    def __init__(self, ptr: int, nbytes: int):
        self.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (ptr, False), "version": 3}


def device_view(ptr: int, nbytes: int):
    """A uint8 torch tensor aliasing nbytes of library-owned device memory at ptr
    (valid while the owner lives)."""
    torch = _torch()
    return torch.as_tensor(_DeviceBytes(ptr, nbytes), device="cuda")


# ------------------------------------------------------------------ served form

class Server:
    """huff_server: submit device-resident symbol tensors, wait for results.
    Keyword arguments are huff_serve_cfg fields (mem_budget_bytes, nstreams,
    max_batch, max_inflight, chunk_log2, max_batch_symbols, max_queue)."""

    def __init__(self, **cfg):
        c = huff_serve_cfg()
        lib().huff_serve_default_cfg(ctypes.byref(c))
        for k, v in cfg.items():
            setattr(c, k, int(v))
        h = ctypes.c_void_p()
        _check(lib().huff_serve_create(ctypes.byref(c), ctypes.byref(h)), "huff_serve_create")
        self.handle = h
        self._keep = {}

    def submit(self, sym, nbins: int, keep: bool = True) -> int:
        """Queues an encode of the 1-D integer tensor `sym`; returns the ticket.
        The tensor is kept alive until the ticket is released (keep=True)."""
        r = huff_request(_ptr(sym), sym.numel(), dtype_code(sym), nbins)
        t = ctypes.c_uint64()
        rc = lib().huff_serve_submit(self.handle, ctypes.byref(r), ctypes.byref(t))
        _check(rc, "huff_serve_submit")
        if keep:
            self._keep[t.value] = sym
        return t.value

    def submit_raw(self, ptr: int, n: int, dtype: int, nbins: int) -> tuple[int, int]:
        """Like submit for a raw device pointer; returns (status, ticket)."""
        r = huff_request(ptr, n, dtype, nbins)
        t = ctypes.c_uint64()
        rc = lib().huff_serve_submit(self.handle, ctypes.byref(r), ctypes.byref(t))
        return rc, t.value

    @staticmethod
    def _res(r: huff_result) -> dict:
        return {k: getattr(r, k) for k, _ in huff_result._fields_}

    def poll(self, ticket: int):
        r = huff_result()
        rc = lib().huff_serve_poll(self.handle, ticket, ctypes.byref(r))
        if rc == STATUS_CODE["HUFF_ERR_BUSY"]:
            return None
        _check(rc, "huff_serve_poll")
        return self._res(r)

    def wait(self, ticket: int) -> dict:
        r = huff_result()
        _check(lib().huff_serve_wait(self.handle, ticket, ctypes.byref(r)), "huff_serve_wait")
        return self._res(r)

    def release(self, ticket: int) -> None:
        _check(lib().huff_serve_release(self.handle, ticket), "huff_serve_release")
        self._keep.pop(ticket, None)

    def stats(self) -> dict:
        st = huff_serve_stats()
        _check(lib().huff_serve_get_stats(self.handle, ctypes.byref(st)), "huff_serve_get_stats")
        return {k: getattr(st, k) for k, _ in huff_serve_stats._fields_}

    def close(self) -> None:
        if getattr(self, "handle", None):
            lib().huff_serve_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
