"""Seeded synthetic inputs for HOQRI workloads.

This module is the only code shared by the CUDA path's tests/benchmarks and the
CPU oracle.  It draws random numbers and nothing else: it holds none of the
method's arithmetic (no mode products, no Kronecker products, no QR of the
method's iterates).  Every stream is a counter-based Philox generator keyed by
(master seed, purpose, mode, chunk), so a workload is reproducible bit for bit
on any machine and independent of the thread count used to draw it.

Workload shapes follow the paper's synthetic experiments (Sec. 6.1: I^N sparse
tensors, nnz = 10I or 100I, rank 10^N) and five benchmark configurations:

* ``c1``: 200^3, nnz 1e4 raw draws (repeats summed), uniform i.i.d. indices,
  uniform(0,1) values, K=5, FP64.
* ``c2``: 2e5 x 1e5 x 5e4, 5e7 distinct nonzeros, Zipf(1.1) indices over a
  seeded permutation, lognormal(0,1) values, K=16, FP32.
* ``c3``: 5e4 x 2e4 x 2e4 x 5e3, 1e8 distinct nonzeros, Zipf(1.2),
  uniform(0,1), K=8, split-BF16 tensor cores.
* ``c4``: 1e5^3, 2e7 uniform positions of a planted 10^3 Tucker model plus
  N(0, 0.01^2) noise.
* ``c5``: serving mix (order 3 or 4, dims U[1e3,1e6], log10 nnz ~ N(5.5,0.5)
  clipped to [4,7], Zipf(1.1), ranks from {4,8,16,32}).
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

MASTER_SEED = 0x484F5152  # "HOQR"

# purpose codes for the Philox key
_P_IDX, _P_PERM, _P_VAL, _P_FACT, _P_CORE, _P_NOISE, _P_MIX, _P_ARR, _P_SUB = range(1, 10)

_CHUNK = 1 << 22  # samples per independent Philox sub-stream


def _rng(seed: int, purpose: int, sub: int = 0) -> np.random.Generator:
    """Counter-based stream keyed by (seed, purpose, sub)."""
    key = np.array([seed & 0xFFFFFFFFFFFFFFFF, ((purpose & 0xFFFF) << 40) | (sub & ((1 << 40) - 1))],
                   dtype=np.uint64)
    return np.random.Generator(np.random.Philox(key=key))


def _chunked(n: int, fn) -> None:
    """Run fn(chunk_id, lo, hi) over fixed-size chunks on a thread pool."""
    spans = [(c, lo, min(n, lo + _CHUNK)) for c, lo in enumerate(range(0, n, _CHUNK))]
    if len(spans) <= 1:
        for sp in spans:
            fn(*sp)
        return
    with ThreadPoolExecutor(max(1, min(16, os.cpu_count() or 1))) as ex:
        list(ex.map(lambda sp: fn(*sp), spans))


def zipf_cdf(I: int, s: float) -> np.ndarray:
    """CDF of the truncated Zipf law P(r) proportional to r^-s on ranks 1..I."""
    c = np.cumsum(np.arange(1, I + 1, dtype=np.float64) ** (-s))
    return c / c[-1]


def draw_indices(I: int, n: int, seed: int, mode: int, dist: str, s: float = 1.1) -> np.ndarray:
    """n i.i.d. indices in [0, I): uniform, or a Zipf(s) rank (inverse CDF of a
    seeded uniform) mapped through a seeded random permutation of [0, I)."""
    out = np.empty(n, dtype=np.int32)
    if dist == "uniform":
        def fn(c, lo, hi):
            out[lo:hi] = _rng(seed, _P_IDX, (mode << 24) | c).integers(0, I, size=hi - lo)
    elif dist == "zipf":
        cdf = zipf_cdf(I, s)
        perm = _rng(seed, _P_PERM, mode).permutation(I).astype(np.int32)

        def fn(c, lo, hi):
            u = _rng(seed, _P_IDX, (mode << 24) | c).random(hi - lo)
            r = np.minimum(np.searchsorted(cdf, u, side="right"), I - 1)
            out[lo:hi] = perm[r]
    else:
        raise ValueError(dist)
    _chunked(n, fn)
    return out


def draw_values(n: int, seed: int, values: str, salt: int = 0) -> np.ndarray:
    """n i.i.d. values, uniform(0,1) or lognormal(0,1)."""
    if values not in ("uniform", "lognormal"):
        raise ValueError(values)
    out = np.empty(n, dtype=np.float64)

    def fn(c, lo, hi):
        r = _rng(seed, _P_VAL, (salt << 24) | c)
        out[lo:hi] = r.random(hi - lo) if values == "uniform" else r.lognormal(0.0, 1.0, hi - lo)
    _chunked(n, fn)
    return out


@dataclass
class SparseTensor:
    """COO tensor, 0-based int32 indices (the raw stream may repeat coordinates)."""
    dims: tuple
    idx: list            # N arrays of int32, length nnz
    vals: np.ndarray     # float64 or float32, length nnz
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return len(self.dims)

    @property
    def nnz(self) -> int:
        return int(self.vals.shape[0])


def _sorted_unique(a: np.ndarray) -> np.ndarray:
    a = np.sort(a)
    if a.size == 0:
        return a
    keep = np.empty(a.size, dtype=bool)
    keep[0] = True
    np.not_equal(a[1:], a[:-1], out=keep[1:])
    return a[keep]


def random_sparse(dims, nnz: int, seed: int, dist: str = "uniform", s: float = 1.1,
                  values: str = "uniform", dtype=np.float64, distinct: bool = False) -> SparseTensor:
    """Sparse tensor with per-mode i.i.d. uniform or Zipf(s) indices.

    distinct=False: nnz raw draws; repeated coordinates stay in the stream (the
    consumer sums them).  distinct=True: coordinates are drawn until at least
    nnz distinct ones exist, a seeded subset of exactly nnz of them is kept in a
    seeded random order, and each gets one value draw (needs prod(dims) < 2^63)."""
    dims = tuple(int(d) for d in dims)
    N = len(dims)
    if not distinct:
        idx = [draw_indices(I, nnz, seed, m, dist, s) for m, I in enumerate(dims)]
        v = draw_values(nnz, seed, values)
        return SparseTensor(dims, idx, v.astype(dtype),
                            dict(dist=dist, s=s, values=values, seed=seed, distinct=False))
    if math.prod(dims) >= (1 << 63):
        raise ValueError("distinct sampling needs prod(dims) < 2^63")
    strides = [math.prod(dims[m + 1:]) for m in range(N)]
    uniq = np.empty(0, dtype=np.int64)
    draw, rnd = nnz, 0
    while True:
        keys = np.zeros(draw, dtype=np.int64)
        for m, I in enumerate(dims):
            keys += draw_indices(I, draw, seed + 7919 * rnd, m, dist, s).astype(np.int64) * strides[m]
        uniq = _sorted_unique(np.concatenate([uniq, keys]))
        del keys
        if uniq.size >= nnz:
            break
        rnd += 1
        draw = int((nnz - uniq.size) * 1.6) + 4096
    r = _rng(seed, _P_SUB, 0)
    if uniq.size > nnz:
        uniq = uniq[np.sort(r.choice(uniq.size, size=nnz, replace=False))]
    uniq = uniq[r.permutation(nnz)]
    idx = [((uniq // strides[m]) % dims[m]).astype(np.int32) for m in range(N)]
    v = draw_values(nnz, seed, values, salt=1)
    return SparseTensor(dims, idx, v.astype(dtype),
                        dict(dist=dist, s=s, values=values, seed=seed, distinct=True))


def gaussian_factors(dims, ranks, seed: int) -> list:
    """Seeded Gaussian I_n x K_n matrices (float64): the raw draw for the random
    initialisation the paper allows (Alg. 2, 'initialize randomly')."""
    return [_rng(seed, _P_FACT, m).standard_normal((I, K)) for m, (I, K) in enumerate(zip(dims, ranks))]


def orthonormal_factors(dims, ranks, seed: int) -> list:
    """Initial factors: numpy's LAPACK QR of the seeded Gaussian draw, columns
    signed so diag(R) > 0 (input preparation; the library and the oracle both
    receive these same arrays)."""
    out = []
    for Z in gaussian_factors(dims, ranks, seed):
        q, r = np.linalg.qr(Z)
        q = q * np.where(np.diag(r) < 0, -1.0, 1.0)[None, :]
        out.append(np.ascontiguousarray(q))
    return out


def planted_tucker(dims, ranks, nnz: int, sigma: float, seed: int, dtype=np.float64):
    """Planted Tucker model observed at nnz distinct uniform positions plus noise.

    Ground truth: Gaussian core and random orthonormal factors.  Entries at the
    sampled positions are rescaled so their RMS is 1, then N(0, sigma^2) noise
    is added.  Returns (SparseTensor, U_true list, G_true scaled)."""
    N = len(dims)
    pos = random_sparse(dims, nnz, seed, dist="uniform", values="uniform", distinct=True)
    Ut = orthonormal_factors(dims, ranks, seed ^ 0x5A5A)
    Gt = _rng(seed, _P_CORE).standard_normal(tuple(ranks))
    # ground-truth model value at each observed position (data synthesis only):
    # the core contracted with the last mode's rows by a matrix product, then a
    # row-wise dot with the Khatri-Rao product of the other modes' rows
    vals = np.empty(nnz, dtype=np.float64)
    GflatT = np.ascontiguousarray(Gt.reshape(-1, ranks[-1]).T)
    B = 1 << 16
    for s0 in range(0, nnz, B):
        rows = [np.take(Ut[m], pos.idx[m][s0:s0 + B], axis=0) for m in range(N)]
        W = rows[-1] @ GflatT
        kr = rows[0]
        for m in range(1, N - 1):
            kr = (kr[:, :, None] * rows[m][:, None, :]).reshape(kr.shape[0], -1)
        vals[s0:s0 + B] = np.einsum("zp,zp->z", kr, W)
    scale = 1.0 / math.sqrt(float(np.mean(vals * vals)))
    noise = np.empty(nnz, dtype=np.float64)

    def fn(c, lo, hi):
        noise[lo:hi] = _rng(seed, _P_NOISE, c).standard_normal(hi - lo)
    _chunked(nnz, fn)
    vals = vals * scale + sigma * noise
    X = SparseTensor(pos.dims, pos.idx, vals.astype(dtype),
                     dict(dist="planted", sigma=sigma, seed=seed, scale=scale, distinct=True))
    return X, Ut, Gt * scale


@dataclass
class ServeRequest:
    rid: int
    arrival_s: float
    dims: tuple
    ranks: tuple
    nnz: int
    seed: int


def serving_mix(n_req: int, rate_hz: float, seed: int, dim_range=(1_000, 1_000_000),
                log_nnz=(5.5, 0.5, 4.0, 7.0), rank_set=(4, 8, 16, 32),
                p_order3: float = 0.7, max_pm=None) -> list:
    """Poisson arrivals of decomposition requests (order 3 w.p. p_order3 else 4).

    Ranks are redrawn per request until K_n <= I_n and K_n <= prod_{m!=n} K_m
    (and prod_{m!=n} K_m <= max_pm when max_pm is given)."""
    r = _rng(seed, _P_MIX)
    ra = _rng(seed, _P_ARR)
    t = 0.0
    out = []
    for q in range(n_req):
        t += ra.exponential(1.0 / rate_hz)
        N = 3 if r.random() < p_order3 else 4
        dims = tuple(int(v) for v in r.integers(dim_range[0], dim_range[1] + 1, size=N))
        mu, sd, lo, hi = log_nnz
        nnz = int(round(10 ** float(np.clip(r.normal(mu, sd), lo, hi))))
        while True:
            ranks = tuple(int(v) for v in r.choice(rank_set, size=N))
            if all(ranks[n] <= dims[n] and ranks[n] <= math.prod(ranks[:n] + ranks[n + 1:]) and
                   (max_pm is None or math.prod(ranks[:n] + ranks[n + 1:]) <= max_pm) for n in range(N)):
                break
        out.append(ServeRequest(q, t, dims, ranks, nnz, (seed * 1000003 + q) & 0x7FFFFFFF))
    return out


# ---- the benchmark workloads -------------------------------------------------------------

CONFIGS = {
    "c1": dict(dims=(200, 200, 200), nnz=10_000, dist="uniform", values="uniform",
               ranks=(5, 5, 5), iters=10, prec="fp64", distinct=False),
    "c2": dict(dims=(200_000, 100_000, 50_000), nnz=50_000_000, dist="zipf", s=1.1,
               values="lognormal", ranks=(16, 16, 16), iters=20, prec="fp32", distinct=True),
    "c3": dict(dims=(50_000, 20_000, 20_000, 5_000), nnz=100_000_000, dist="zipf", s=1.2,
               values="uniform", ranks=(8, 8, 8, 8), iters=10, prec="bf16x3", distinct=True),
    "c4": dict(dims=(100_000, 100_000, 100_000), nnz=20_000_000, dist="planted", sigma=0.01,
               ranks=(10, 10, 10), iters=10, prec="fp32", distinct=True),
}


def config_seed(name: str) -> int:
    return MASTER_SEED + int(name[1:])


def make_config(name: str, scale: float = 1.0, dtype=None):
    """Build a benchmark workload, optionally with nnz scaled down (dims kept).

    Returns (SparseTensor, U0 list of float64 orthonormal factors, cfg dict)."""
    cfg = dict(CONFIGS[name])
    seed = config_seed(name)
    nnz = max(1, int(round(cfg["nnz"] * scale)))
    if dtype is None:
        dtype = np.float64 if cfg["prec"] == "fp64" else np.float32
    if cfg["dist"] == "planted":
        X, Ut, Gt = planted_tucker(cfg["dims"], cfg["ranks"], nnz, cfg["sigma"], seed, dtype=dtype)
        X.meta["U_true"] = Ut
        X.meta["G_true"] = Gt
    else:
        X = random_sparse(cfg["dims"], nnz, seed, dist=cfg["dist"], s=cfg.get("s", 1.1),
                          values=cfg["values"], dtype=dtype, distinct=cfg["distinct"])
    U0 = orthonormal_factors(cfg["dims"], cfg["ranks"], seed + 0x100)
    cfg["nnz_target"] = nnz
    return X, U0, cfg
