"""Seeded input generators (no field arithmetic here)."""
from __future__ import annotations

import dataclasses

import numpy as np


def _rng(seed) -> np.random.Generator:
    if isinstance(seed, np.random.Generator):
        return seed
    return np.random.Generator(np.random.PCG64(seed))


def source(seed, k: int, W: int) -> np.ndarray:
    """Uniform 16-bit source symbols, ``[k][W]`` uint16."""
    return _rng(seed).integers(0, 65536, size=(k, W), dtype=np.uint16)


def received_uniform(seed, npos: int, W: int) -> np.ndarray:
    """Uniform received words in [0, 65536], ``[npos][W]`` uint32."""
    return _rng(seed).integers(0, 65537, size=(npos, W), dtype=np.uint32)


def erased_uniform(seed, n: int, k: int) -> np.ndarray:
    """n - k erased positions drawn uniformly without replacement (sorted)."""
    return np.sort(_rng(seed).choice(n, n - k, replace=False)).astype(np.uint32)


def erased_burst(seed, n: int, k: int) -> np.ndarray:
    """A contiguous burst [b, b + n - k) with b uniform in [0, k] (no wrap)."""
    b = int(_rng(seed).integers(0, k + 1))
    return np.arange(b, b + (n - k), dtype=np.uint32)


def received_positions(n: int, erased) -> np.ndarray:
    """Ascending positions that survive the erasures."""
    mask = np.ones(n, dtype=bool)
    mask[np.asarray(erased, dtype=np.int64)] = False
    return np.nonzero(mask)[0].astype(np.uint32)


@dataclasses.dataclass(frozen=True)
class Config:
    """One named workload: code length n, dimension k, W codewords per batch."""

    name: str
    n: int
    k: int
    W: int
    seed: int
    erasure: str = "uniform"

    @property
    def packet_bytes(self) -> int:
        return 2 * self.W

    def source(self) -> np.ndarray:
        return source(self.seed, self.k, self.W)

    def positions(self, variant: str | None = None) -> np.ndarray:
        kind = variant or self.erasure
        rng = _rng(self.seed + 1000)
        if kind == "burst":
            er = erased_burst(rng, self.n, self.k)
        else:
            er = erased_uniform(rng, self.n, self.k)
        return received_positions(self.n, er)


# The fixed-shape workloads: coderate 1/2 with 1 KB, 4 KB and 2 KB packets.
CONFIGS = {
    "k256_n512_w512": Config("k256_n512_w512", 512, 256, 512, 1),
    "k4096_n8192_w2048": Config("k4096_n8192_w2048", 8192, 4096, 2048, 2),
    "k32768_n65536_w1024_burst": Config("k32768_n65536_w1024_burst", 65536, 32768, 1024, 3,
                                        "burst"),
    "k32768_n65536_w1024_uniform": Config("k32768_n65536_w1024_uniform", 65536, 32768, 1024,
                                          3, "uniform"),
}


def ragged_groups(seed: int = 4, groups: int = 4096, log2n=(8, 16), log2bytes=(8, 12),
                  rates=((1, 2), (2, 3), (3, 4), (7, 8))):
    """Ragged batch: per group n = 2^U{lo..hi}, k = floor(n * rate), W = bytes / 2.

    Returns a list of dicts with n, k, W and the received positions of the
    group's own uniform erasure pattern.
    """
    rng = _rng(seed)
    out = []
    for g in range(groups):
        n = 1 << int(rng.integers(log2n[0], log2n[1] + 1))
        num, den = rates[int(rng.integers(0, len(rates)))]
        k = (n * num) // den
        W = (1 << int(rng.integers(log2bytes[0], log2bytes[1] + 1))) // 2
        er = erased_uniform(rng, n, k)
        out.append({"n": n, "k": k, "W": W, "positions": received_positions(n, er),
                    "seed": int(rng.integers(0, 2**31))})
    return out


def serving_requests(seed: int = 5, rate_per_s: float = 5000.0, duration_s: float = 1.0,
                     log2n=(9, 16), rates=((1, 2), (3, 4)), log2bytes=(10, 14),
                     decode_fraction: float = 0.5, patterns_per_shape: int = 64):
    """Poisson arrivals of encode / decode requests.

    Decode requests draw their erasure pattern from ``patterns_per_shape``
    recurring patterns per (n, k) so that resident locator tables matter.
    """
    rng = _rng(seed)
    t = 0.0
    reqs = []
    pattern_seeds = {}
    while True:
        t += float(rng.exponential(1.0 / rate_per_s))
        if t >= duration_s:
            break
        n = 1 << int(rng.integers(log2n[0], log2n[1] + 1))
        num, den = rates[int(rng.integers(0, len(rates)))]
        k = (n * num) // den
        W = (1 << int(rng.integers(log2bytes[0], log2bytes[1] + 1))) // 2
        op = "decode" if rng.random() < decode_fraction else "encode"
        pat = int(rng.integers(0, patterns_per_shape))
        key = (n, k, pat)
        if key not in pattern_seeds:
            pattern_seeds[key] = int(rng.integers(0, 2**31))
        reqs.append({"t": t, "op": op, "n": n, "k": k, "W": W, "pattern": pat,
                     "pattern_seed": pattern_seeds[key], "seed": int(rng.integers(0, 2**31))})
    return reqs
