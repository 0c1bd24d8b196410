"""Seeded synthetic symbol streams shaped like the paper's workloads.

This module holds no Huffman arithmetic: it only draws integer symbols.  Both
the CUDA path (benchmarks, parity tests) and the CPU oracle take their inputs
from here, so neither side can influence the other's inputs.

Random source (counter based, no state):

    mix64(z)          the SplitMix64 output finaliser (Steele, Lea & Flood,
                      "Fast splittable pseudorandom number generators",
                      OOPSLA 2014, with the widely published 64-bit constants)
    key(seed, s)      mix64((seed + 1) * G) ^ mix64((s + 1) * K)
    u64(seed, s, i)   mix64(key(seed, s) + (i + 1) * G)    (all mod 2^64)

with G = 0x9E3779B97F4A7C15 (the SplitMix64 increment) and
K = 0xD1B54A32D192ED03.  ``s`` is a stream number; element ``i`` of a stream
only depends on (seed, s, i), so any sub-range can be regenerated on its own.

Symbols come from an integer-exact inverse CDF: with ``u = u64 >> 32`` and a
table ``T[k] = floor(CDF_k * 2^32)`` (``T[K-1] = 2^32``), the symbol is
``min{k : u < T[k]}``.  The table is computed once in double precision from
the probability mass function and then used as plain integers.

Distributions (Sec. V-A describes the paper's data: SZ quantisation codes
centred at the middle bin, k-mer and text alphabets):

* ``gaussian(K, mu, sigma)``   mass of [k-1/2, k+1/2) of N(mu, sigma^2); the
  two tails are folded into bins 0 and K-1.
* ``laplace(K, mu, b)``        same for the Laplace(mu, b) law.
* ``with_outliers(p, eps)``    mixture (1-eps) p + eps / K.
* ``zipf(K, s)``               p(rank) proportional to rank^-s, rank 1..K;
  rank r is given symbol perm[r-1] where perm is a Fisher-Yates shuffle drawn
  from stream 1 (``j = u64(seed, 1, i) mod (i+1)`` for i = K-1 .. 1), or the
  identity when no permutation is asked for.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_G = np.uint64(0x9E3779B97F4A7C15)
_K = np.uint64(0xD1B54A32D192ED03)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1


def _mix64_int(z: int) -> int:
    z &= _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def stream_key(seed: int, stream: int) -> int:
    return _mix64_int((seed + 1) * 0x9E3779B97F4A7C15) ^ _mix64_int((stream + 1) * 0xD1B54A32D192ED03)


def u64_scalar(seed: int, stream: int, i: int) -> int:
    """One draw, pure Python integers (used for small per-field parameters)."""
    return _mix64_int(stream_key(seed, stream) + (i + 1) * 0x9E3779B97F4A7C15)


def _mix64_np(z: np.ndarray) -> np.ndarray:
    z = z ^ (z >> np.uint64(30))
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def u64_range(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Draws u64(seed, stream, i) for i in [start, start + count)."""
    key = np.uint64(stream_key(seed, stream))
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
        z = key + idx * _G
        return _mix64_np(z)


# ----------------------------------------------------------------------------
# probability mass functions (double precision)
# ----------------------------------------------------------------------------

def _phi(x: float) -> float:
    return 0.5 * math.erfc(-x / math.sqrt(2.0))


def gaussian_pmf(K: int, mu: float, sigma: float) -> np.ndarray:
    cdf = np.array([_phi((k + 0.5 - mu) / sigma) for k in range(K)], dtype=np.float64)
    cdf[-1] = 1.0
    return np.diff(np.concatenate([[0.0], cdf]))


def _laplace_cdf(x: float, mu: float, b: float) -> float:
    if x < mu:
        return 0.5 * math.exp((x - mu) / b)
    return 1.0 - 0.5 * math.exp(-(x - mu) / b)


def laplace_pmf(K: int, mu: float, b: float) -> np.ndarray:
    cdf = np.array([_laplace_cdf(k + 0.5, mu, b) for k in range(K)], dtype=np.float64)
    cdf[-1] = 1.0
    return np.diff(np.concatenate([[0.0], cdf]))


def with_outliers(pmf: np.ndarray, eps: float) -> np.ndarray:
    return (1.0 - eps) * pmf + eps / len(pmf)


def zipf_pmf(K: int, s: float) -> np.ndarray:
    w = np.arange(1, K + 1, dtype=np.float64) ** (-s)
    return w / w.sum()


def permutation(seed: int, K: int) -> np.ndarray:
    """Fisher-Yates shuffle of 0..K-1 driven by stream 1."""
    perm = np.arange(K, dtype=np.int64)
    draws = u64_range(seed, 1, 0, K)
    for i in range(K - 1, 0, -1):
        j = int(draws[i]) % (i + 1)
        perm[i], perm[j] = perm[j], perm[i]
    return perm


def cdf_table(pmf: np.ndarray) -> np.ndarray:
    """T[k] = floor(CDF_k * 2^32) as uint64, T[K-1] = 2^32, nondecreasing."""
    cdf = np.cumsum(np.asarray(pmf, dtype=np.float64))
    cdf = cdf / cdf[-1]
    t = np.floor(cdf * 4294967296.0)
    t = np.clip(t, 0, 4294967296.0).astype(np.uint64)
    t[-1] = np.uint64(1 << 32)
    return np.maximum.accumulate(t)


# ----------------------------------------------------------------------------
# symbol streams
# ----------------------------------------------------------------------------

_DTYPES = {1: np.uint8, 2: np.uint16, 4: np.uint32}


def draw(seed: int, stream: int, n: int, table: np.ndarray, width: int,
         mapping: np.ndarray | None = None, threads: int | None = None) -> np.ndarray:
    """n symbols of ``width`` bytes by inverse CDF over ``table``.

    ``mapping`` (optional) renames drawn index k to ``mapping[k]``.
    The work is split in chunks over threads (numpy releases the GIL).
    """
    dt = _DTYPES[width]
    out = np.empty(n, dtype=dt)
    if n == 0:
        return out
    table = np.ascontiguousarray(table, dtype=np.uint64)
    mp = None if mapping is None else np.asarray(mapping).astype(dt)
    chunk = 1 << 22
    starts = list(range(0, n, chunk))

    def work(s0: int) -> None:
        cnt = min(chunk, n - s0)
        u = u64_range(seed, stream, s0, cnt) >> np.uint64(32)
        k = np.searchsorted(table, u, side="right")
        out[s0:s0 + cnt] = k.astype(dt) if mp is None else mp[k]

    nthreads = threads or min(16, os.cpu_count() or 1)
    if len(starts) == 1 or nthreads == 1:
        for s0 in starts:
            work(s0)
    else:
        with ThreadPoolExecutor(max_workers=nthreads) as ex:
            list(ex.map(work, starts))
    return out


# ----------------------------------------------------------------------------
# named workloads (sizes as stated with each function)
# ----------------------------------------------------------------------------

def gaussian_field(n: int, seed: int = 0, K: int = 1024, sigma: float = 8.0) -> np.ndarray:
    """u16 symbols, discretised Gaussian centred at K/2 (1,048,576 x sigma=8, seed 0
    is the small plain-pipeline case)."""
    return draw(seed, 0, n, cdf_table(gaussian_pmf(K, K // 2, sigma)), 2)


def laplace_field(n: int, seed: int = 1, K: int = 1024, b: float = 2.0,
                  outliers: float = 0.01, stream: int = 0) -> np.ndarray:
    """u16 quantisation-code field: Laplace(K/2, b) plus a uniform outlier share
    (512^3 symbols, b=2, 1 % outliers, seed 1 is the HPC field that stands in
    for the paper's Nyx-Quant data)."""
    pmf = laplace_pmf(K, K // 2, b)
    if outliers > 0:
        pmf = with_outliers(pmf, outliers)
    return draw(seed, stream, n, cdf_table(pmf), 2)


def zipf_field(n: int, K: int, s: float = 1.1, seed: int = 3, width: int = 4,
               permute: bool = True) -> np.ndarray:
    """Zipf(s) symbols over K ids; with ``permute`` ranks map through a seeded
    Fisher-Yates permutation (67,108,864 u32 over 8,192 / 65,536 ids, s=1.1,
    seed 3 is the large-alphabet stress case)."""
    mp = permutation(seed, K) if permute else None
    return draw(seed, 0, n, cdf_table(zipf_pmf(K, s)), width, mapping=mp)


def batch_field_params(j: int, seed: int = 4, n_lo: int = 65536, n_hi: int = 16777216,
                       b_lo: float = 0.5, b_hi: float = 16.0) -> tuple[int, float]:
    """Size (log-uniform in [n_lo, n_hi]) and Laplace scale (uniform in
    [b_lo, b_hi]) of field j of the batched workload; both from stream 10000+j."""
    u0 = u64_scalar(seed, 10000 + j, 0) / 2.0 ** 64
    u1 = u64_scalar(seed, 10000 + j, 1) / 2.0 ** 64
    n = int(round(math.exp(math.log(n_lo) + u0 * (math.log(n_hi) - math.log(n_lo)))))
    b = b_lo + u1 * (b_hi - b_lo)
    return n, b


def batch_field(j: int, seed: int = 4, K: int = 1024, n_scale: float = 1.0) -> np.ndarray:
    """Field j of the 512-field batched workload: u16 Laplace(K/2, b_j), no
    outliers, drawn from stream j.  ``n_scale`` shrinks sizes for quick tests."""
    n, b = batch_field_params(j, seed)
    n = max(1, int(n * n_scale))
    return draw(seed, j, n, cdf_table(laplace_pmf(K, K // 2, b)), 2)


# ----------------------------------------------------------------------------
# served workload: Poisson arrivals of mixed requests
# ----------------------------------------------------------------------------

_ZIPF_256_TABLE = None
_SERVED_EDGES = np.arange(1024, dtype=np.float64) + 0.5 - 512.0


def served_arrivals(count: int, rate: float = 2000.0, seed: int = 5) -> np.ndarray:
    """Arrival times (s, from 0) of the first `count` requests: exponential
    gaps of mean 1/rate from stream 2 (inverse CDF of the uniform draws)."""
    u = (u64_range(seed, 2, 0, count) >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    return np.cumsum(-np.log1p(-u) / rate)


def served_request(i: int, seed: int = 5, n_lo: int = 16384, n_hi: int = 67108864):
    """Request i of the served workload as (width, n, nbins, table): half u8
    Zipf(1.2) over 256 ids, half u16 over 1024 bins from a discretised
    Gaussian or Laplace centred at 512 with sigma / b log-uniform in [1, 64];
    n log-uniform in [n_lo, n_hi].  Its symbols are draw(seed, 100 + i, n,
    table, width).  Parameters come from stream 1,000,000 + i."""
    global _ZIPF_256_TABLE
    u = [u64_scalar(seed, 1_000_000 + i, k) / 2.0 ** 64 for k in range(4)]
    n = int(round(math.exp(math.log(n_lo) + u[0] * (math.log(n_hi) - math.log(n_lo)))))
    if u[1] < 0.5:
        if _ZIPF_256_TABLE is None:
            _ZIPF_256_TABLE = cdf_table(zipf_pmf(256, 1.2))
        return 1, n, 256, _ZIPF_256_TABLE
    scale = math.exp(u[2] * math.log(64.0))
    edges = _SERVED_EDGES
    if u[3] < 0.5:
        from scipy.special import ndtr
        cdf = ndtr(edges / scale)
    else:
        cdf = np.where(edges < 0, 0.5 * np.exp(edges / scale), 1.0 - 0.5 * np.exp(-edges / scale))
    cdf[-1] = 1.0
    return 2, n, 1024, cdf_table(np.diff(np.concatenate([[0.0], cdf])))


def served_symbols(i: int, seed: int = 5, **kw) -> np.ndarray:
    """The symbols of served request i, drawn on the host (for the oracle)."""
    width, n, nbins, table = served_request(i, seed, **kw)
    return draw(seed, 100 + i, n, table, width)


def empirical_bits(pmf: np.ndarray) -> float:
    """Shannon entropy of a pmf in bits (diagnostics only)."""
    p = np.asarray(pmf, dtype=np.float64)
    p = p[p > 0]
    return float(-(p * np.log2(p)).sum())


# ----------------------------------------------------------------------------
# the same draws on the GPU (libhuffsynth.so, built next to libhuff.so)
# ----------------------------------------------------------------------------

_synth_lib = None


def _synthgen():
    global _synth_lib
    if _synth_lib is None:
        import ctypes
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libhuffsynth.so")
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is not built (paper_2010_10039_gb300/build.py builds it)")
        L = ctypes.CDLL(path)
        L.synth_draw.restype = ctypes.c_int
        L.synth_draw.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p, ctypes.c_uint32,
                                 ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p]
        _synth_lib = L
    return _synth_lib


def draw_device(seed: int, stream: int, n: int, table, width: int, mapping=None, out=None, start: int = 0):
    """``draw`` on the current CUDA device: returns (or fills) a torch tensor of
    n symbols (uint8 / int16 / int32 storage for widths 1 / 2 / 4) equal bit for
    bit to ``draw(seed, stream, n, table, width, mapping)[start:]``."""
    import torch
    tdt = {1: torch.uint8, 2: torch.int16, 4: torch.int32}[width]
    if out is None:
        out = torch.empty(n, dtype=tdt, device="cuda")
    t = torch.from_numpy(np.ascontiguousarray(table, dtype=np.uint64).view(np.int64)).cuda()
    mp = None
    if mapping is not None:
        mp = torch.from_numpy(np.asarray(mapping).astype(np.uint32).view(np.int32)).cuda()
    rc = _synthgen().synth_draw(out.data_ptr() if n else None, n, width, t.data_ptr(), len(table),
                                mp.data_ptr() if mp is not None else None, seed, stream, start,
                                torch.cuda.current_stream().cuda_stream)
    if rc != 0:
        raise RuntimeError(f"synth_draw failed with CUDA error {rc}")
    return out
