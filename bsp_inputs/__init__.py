"""Seeded synthetic inputs shaped like the paper's sorting benchmarks (Sec. 6.3).

Shared by the tests, the bench and the oracle runs.  It holds none of the sort's
arithmetic: only random key generation.  Every generator is deterministic in its
arguments.  Keys of "virtual processor" i (block i of p contiguous blocks) come
from their own Philox stream keyed by (seed, 21 + 1001*i), the paper's per-processor
seed rule (Sec. 6.3, input [U]); libc random() itself is not portable, so its range
[0, 2^31 - 1] is kept and its generator is replaced.

INT_MAX in the paper's definitions is 2^31 ("the maximum integer value plus one").
"""
from __future__ import annotations

import numpy as np

INT_MAX = 2**31


def _blocks(n: int, p: int):
    m = -(-n // p) if p > 0 else n
    for i in range(p):
        lo = min(n, i * m)
        hi = min(n, lo + m)
        yield i, lo, hi


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=np.array([seed & (2**64 - 1), stream],
                                                             dtype=np.uint64)))


def _per_block(n: int, p: int, seed: int, fill) -> np.ndarray:
    out = np.empty(n, np.int32)
    for i, lo, hi in _blocks(n, p):
        if hi > lo:
            out[lo:hi] = fill(_rng(seed, 21 + 1001 * i), i, hi - lo)
    return out


def uniform_u32(n: int, seed: int = 1) -> np.ndarray:
    """uint32 keys uniform on [0, 2^32)."""
    return _rng(seed, 7).integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)


def uniform(n: int, p: int, seed: int = 1) -> np.ndarray:
    """[U]: random() values, uniform on [0, 2^31 - 1]."""
    return _per_block(n, p, seed, lambda g, i, c: g.integers(0, INT_MAX, size=c, dtype=np.int64))


def gaussian(n: int, p: int, seed: int = 1) -> np.ndarray:
    """[G]: the mean of four random() calls, floor((a+b+c+d)/4)."""
    def fill(g, i, c):
        v = g.integers(0, INT_MAX, size=(4, c), dtype=np.int64)
        return v.sum(axis=0) // 4
    return _per_block(n, p, seed, fill)


def bucket_sorted(n: int, p: int, seed: int = 1) -> np.ndarray:
    """[B]: each processor holds p buckets of n/p^2 keys, bucket j uniform on
    [j*INT_MAX/p, (j+1)*INT_MAX/p - 1]."""
    def fill(g, i, c):
        out = np.empty(c, np.int64)
        per = -(-c // p)
        for j in range(p):
            lo, hi = j * per, min(c, (j + 1) * per)
            if hi > lo:
                out[lo:hi] = g.integers(j * INT_MAX // p, (j + 1) * INT_MAX // p,
                                        size=hi - lo, dtype=np.int64)
        return out
    return _per_block(n, p, seed, fill)


def staggered(n: int, p: int, seed: int = 1) -> np.ndarray:
    """[S]: processor i < p/2 draws from [(2i+1)INT_MAX/p, (2i+2)INT_MAX/p - 1],
    processor i >= p/2 from [(i-p/2)INT_MAX/p, (i-p/2+1)INT_MAX/p - 1]."""
    def fill(g, i, c):
        if i < p // 2:
            lo, hi = (2 * i + 1) * INT_MAX // p, (2 * i + 2) * INT_MAX // p
        else:
            lo, hi = (i - p // 2) * INT_MAX // p, (i - p // 2 + 1) * INT_MAX // p
        return g.integers(lo, max(hi, lo + 1), size=c, dtype=np.int64)
    return _per_block(n, p, seed, fill)


def g_group(n: int, p: int, seed: int = 1, g: int = 2) -> np.ndarray:
    """[g-G]: blocks are taken g at a time; block i of group j = i // g splits
    its keys into g runs, run t uniform on slice k = (j*g + p/2 + t) mod p of
    p equal slices of [0, INT_MAX) (slice k = [k*INT_MAX/p, (k+1)*INT_MAX/p - 1])."""
    def fill(gen_, i, c):
        j = i // g
        out = np.empty(c, np.int64)
        per = -(-c // g)
        for t in range(g):
            a, b = t * per, min(c, (t + 1) * per)
            if b > a:
                k = (j * g + p // 2 + t) % p
                lo, hi = k * INT_MAX // p, (k + 1) * INT_MAX // p
                out[a:b] = gen_.integers(lo, max(hi, lo + 1), size=b - a, dtype=np.int64)
        return out
    return _per_block(n, p, seed, fill)


def det_duplicates(n: int, p: int, seed: int = 1) -> np.ndarray:
    """[DD]: the first p/2 blocks hold only the value lg n, the next p/4
    blocks only lg(n/p), the next p/8 only lg(n/p^2), and so on while a
    whole block group is left; in the last block the first n/(2p) keys are
    lg(n/p), the next n/(4p) lg(n/(2p)), and so on, the final keys taking
    the last value.  lg x is floor(log2 x) (negative below 1).  No randomness."""
    def lg(x: float) -> int:
        return int(np.floor(np.log2(x)))
    out = np.empty(n, np.int32)
    blocks = list(_blocks(n, p))
    b, i = 0, 1
    while b < p - 1:
        cnt = max(1, p >> i)
        cnt = min(cnt, p - 1 - b)
        for q in range(b, b + cnt):
            _, lo, hi = blocks[q]
            out[lo:hi] = lg(n / float(p) ** (i - 1))
        b += cnt
        i += 1
    _, lo, hi = blocks[p - 1]
    pos, i = lo, 1
    while pos < hi:
        c = max(1, (hi - lo) >> i)
        out[pos:min(hi, pos + c)] = lg(n / (p * 2.0 ** (i - 1)))
        pos += c
        i += 1
    return out


def zero_entropy(n: int, value: int = 2**30) -> np.ndarray:
    """Every key equal."""
    return np.full(n, value, np.int32)


def zipf_values(distinct: int = 256) -> np.ndarray:
    """The int32 value of Zipf rank k (1-based): an injective scramble of k."""
    k = np.arange(1, distinct + 1, dtype=np.uint64)
    return ((k * np.uint64(2654435761)) & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.int32)


def zipf(n: int, s: float = 1.1, distinct: int = 256, seed: int = 1) -> np.ndarray:
    """Ranks 1..distinct with P(k) proportional to k^-s, mapped through zipf_values."""
    w = np.arange(1, distinct + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(w / w.sum())
    cdf[-1] = 1.0
    u = _rng(seed, 11).random(n)
    rank = np.searchsorted(cdf, u, side="right")
    return zipf_values(distinct)[np.minimum(rank, distinct - 1)]


def gmm(n: int, components: int = 8, alpha: float = 0.3, seed: int = 1) -> np.ndarray:
    """float64 keys from a Gaussian mixture: weights Dirichlet(alpha), means
    U[-1e3, 1e3], sigma log-uniform on [1e-2, 1e2]."""
    g = _rng(seed, 13)
    w = g.dirichlet(np.full(components, alpha))
    mu = g.uniform(-1e3, 1e3, components)
    sigma = 10.0 ** g.uniform(-2.0, 2.0, components)
    comp = g.choice(components, size=n, p=w)
    return mu[comp] + sigma[comp] * g.standard_normal(n)


def batched_sizes(count: int, lo_log2: float = 8.0, hi_log2: float = 22.0, seed: int = 1) -> np.ndarray:
    """Instance sizes log-uniform on [2^lo, 2^hi]."""
    u = _rng(seed, 17).uniform(lo_log2, hi_log2, count)
    return np.floor(2.0 ** u).astype(np.int64)


# the paper's other inputs (Sec. 6.3), beside the five of the 2^26 config
EXTRA_DISTRIBUTIONS = {
    "two_group": lambda n, p, seed: g_group(n, p, seed, 2),
    "det_duplicates": lambda n, p, seed: det_duplicates(n, p, seed),
}

DISTRIBUTIONS = {
    "uniform": lambda n, p, seed: uniform(n, p, seed),
    "gaussian": lambda n, p, seed: gaussian(n, p, seed),
    "zero_entropy": lambda n, p, seed: zero_entropy(n),
    "staggered": lambda n, p, seed: staggered(n, p, seed),
    "bucket_sorted": lambda n, p, seed: bucket_sorted(n, p, seed),
}
