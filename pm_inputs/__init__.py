"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no part of the pattern-morphing method: it only draws random
numbers and shapes them into raw inputs (an R-MAT edge list as generated, with
its self-loops and duplicate edges still in it; Zipf vertex labels; random
connected query patterns; Poisson request arrivals).  Graph preparation
(dropping self-loops and duplicates, symmetrising, ordering) is a step of the
method and is done separately by each side.

Every random draw comes from SplitMix64 (S. Vigna, "Further scramblings of
Marsaglia's xorshift generators", 2014; the output function of
java.util.SplittableRandom) evaluated at a counter, so a draw depends only on
(seed, stream, index) and is the same on any machine.
"""
from __future__ import annotations

import os
import hashlib
import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied elementwise to uint64 counters."""
    with np.errstate(over="ignore"):
        z = np.asarray(x, dtype=np.uint64) + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """Doubles in [0, 1) from the 53 high bits of SplitMix64(key(seed, stream) + idx)."""
    key = splitmix64(np.uint64((seed * 0x100000001B3 + stream * 0x9E3779B1) & 0xFFFFFFFFFFFFFFFF))
    with np.errstate(over="ignore"):
        z = splitmix64(np.asarray(idx, dtype=np.uint64) + key)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def rmat_edges(scale: int, edge_factor: int, a: float = 0.57, b: float = 0.19,
               c: float = 0.19, seed: int = 1, chunk: int = 1 << 22):
    """Raw R-MAT edge list (Chakrabarti, Zhan, Faloutsos, SDM 2004).

    2**scale * edge_factor directed draws; at each of ``scale`` levels an edge
    picks the quadrant (0,0), (0,1), (1,0), (1,1) with probabilities a, b, c,
    d = 1-a-b-c, which sets one bit of (src, dst), most significant bit first.
    No noise and no id permutation.  Returns (src, dst) int32 arrays of length
    2**scale * edge_factor with self-loops and duplicates as drawn.
    """
    n_edges = (1 << scale) * edge_factor
    src = np.zeros(n_edges, dtype=np.int32)
    dst = np.zeros(n_edges, dtype=np.int32)
    ab, abc = a + b, a + b + c
    for lo in range(0, n_edges, chunk):
        hi = min(n_edges, lo + chunk)
        e = np.arange(lo, hi, dtype=np.uint64)
        s = np.zeros(hi - lo, dtype=np.int64)
        d = np.zeros(hi - lo, dtype=np.int64)
        for level in range(scale):
            u = uniform01(seed, 1000 + level, e)
            bit = 1 << (scale - 1 - level)
            s_bit = u >= ab                      # quadrants (1,0) and (1,1)
            d_bit = ((u >= a) & (u < ab)) | (u >= abc)   # quadrants (0,1) and (1,1)
            s += s_bit * bit
            d += d_bit * bit
        src[lo:hi] = s
        dst[lo:hi] = d
    return src, dst


def cached_rmat(scale: int, edge_factor: int, seed: int, cache_dir: str | None = None):
    """rmat_edges with an on-disk cache (keyed by all parameters) for large scales."""
    cache_dir = cache_dir or os.environ.get("PM_INPUT_CACHE", "/tmp/pm_inputs_cache")
    os.makedirs(cache_dir, exist_ok=True)
    path = os.path.join(cache_dir, f"rmat_s{scale}_e{edge_factor}_seed{seed}_v1.npz")
    if os.path.exists(path):
        z = np.load(path)
        return z["src"], z["dst"]
    src, dst = rmat_edges(scale, edge_factor, seed=seed)
    tmp = path + f".{os.getpid()}.tmp.npz"
    np.savez(tmp, src=src, dst=dst)
    os.replace(tmp, path)
    return src, dst


def zipf_labels(n: int, n_labels: int, s: float = 1.2, seed: int = 4) -> np.ndarray:
    """Vertex labels, iid per vertex: P(label = i) proportional to (i+1)**-s, i < n_labels.

    Drawn by inverse CDF from one uniform per vertex (indexed by vertex id)."""
    w = np.arange(1, n_labels + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(w / w.sum())
    cdf[-1] = 1.0
    u = uniform01(seed, 7, np.arange(n, dtype=np.uint64))
    return np.searchsorted(cdf, u, side="right").astype(np.uint8)


def gnp_edges(n: int, p: float, seed: int):
    """Erdos-Renyi G(n, p) edge list over pairs a < b (for tiny brute-force graphs)."""
    a, b = np.triu_indices(n, 1)
    keep = uniform01(seed, 11, np.arange(len(a), dtype=np.uint64)) < p
    return a[keep].astype(np.int32), b[keep].astype(np.int32)


def _connected(k: int, mask: int) -> bool:
    seen, stack = {0}, [0]
    while stack:
        v = stack.pop()
        for w in range(k):
            if w not in seen:
                a, b = min(v, w), max(v, w)
                if mask >> pair_index(k, a, b) & 1:
                    seen.add(w)
                    stack.append(w)
    return len(seen) == k


def pair_index(k: int, a: int, b: int) -> int:
    """Bit position of pair (a, b), a < b, in lexicographic pair order."""
    return a * (2 * k - a - 1) // 2 + (b - a - 1)


def random_patterns(count: int, kmin: int = 3, kmax: int = 6, seed: int = 5):
    """Random connected unlabeled query patterns.

    Sizes cycle through kmin..kmax (uniform over sizes); each pattern is a
    uniformly random edge mask over its pairs, redrawn until connected (so
    uniform over labelled connected graphs of that size); even indices are
    vertex-induced, odd ones edge-induced.  Returns a list of
    (k, edge_mask, induced) with induced 1 = vertex-induced, 0 = edge-induced.
    """
    out = []
    draw = 0
    sizes = list(range(kmin, kmax + 1))
    for i in range(count):
        k = sizes[i % len(sizes)]
        npairs = k * (k - 1) // 2
        while True:
            u = uniform01(seed, 21, np.array([draw], dtype=np.uint64))[0]
            draw += 1
            mask = int(u * (1 << npairs))
            if _connected(k, mask):
                break
        out.append((k, mask, 1 if i % 2 == 0 else 0))
    return out


def poisson_arrivals(rate_per_s: float, duration_s: float, seed: int = 6):
    """Arrival times (s) of a Poisson process: exponential gaps by inverse CDF."""
    times, t, i = [], 0.0, 0
    while True:
        u = uniform01(seed, 31, np.array([i], dtype=np.uint64))[0]
        i += 1
        t += -np.log1p(-u) / rate_per_s
        if t >= duration_s:
            return np.array(times)
        times.append(t)


def uniform_ints(seed: int, stream: int, count: int, lo: int, hi: int) -> np.ndarray:
    """count integers uniform in [lo, hi)."""
    u = uniform01(seed, stream, np.arange(count, dtype=np.uint64))
    return (lo + np.floor(u * (hi - lo))).astype(np.int64)


def edge_list_digest(src: np.ndarray, dst: np.ndarray) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(src, dtype=np.int32).tobytes())
    h.update(np.ascontiguousarray(dst, dtype=np.int32).tobytes())
    return h.hexdigest()
