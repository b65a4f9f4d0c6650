"""CPU oracle of the iterative version of Sort_Det_BSP (Sec. 5.1): m rounds of
k-way partitioning, k^m = p.

TEST INFRASTRUCTURE ONLY: imported by tests/.  The product path (the package
``paper_1408_6729_gb300``) never imports it.

Sec. 5.1 describes the iterative version in one paragraph: phases 2
(partitioning) and 3 (merging) are repeated m times, each time splitting every
bucket of the previous round into k buckets of about equal size, with
multi-way merging at the end of each round; the paper defers the details to
its references.  This module takes the following reading, with Fig. 1's steps
applied inside every group of processors:

* p processors, k^m = p.  Processor r holds the contiguous block
  [r*mb, (r+1)*mb) of the input, mb = ceil(n/p), sorted stably (Fig. 1 step 3).
  Records compare by (pad, phi(key), tag) (Sec. 5.1.1); tag = r*M + j for the
  record at local index j of processor r, M = s*ceil(mb/s) (Lemma 5.1's
  padding), so the tag order is the input order.
* Round t = 1..m works inside groups of g = p / k^(t-1) consecutive
  processors (round 1: one group of all p).  In a group:
  - every processor's sorted sequence is padded with +infinity records (pad
    flag 1) to the group's common length Mg = s*ceil(L/s), L the longest
    sequence of the group (at least s), and its records at positions
    j*x - 1, x = Mg/s, j = 1..s, are its sample (Fig. 1 step 4);
  - the g*s sample records are sorted and the records of 1-indexed rank i*q,
    q = g*s/k, i = 1..k-1, are the group's splitters (Fig. 1 steps 5-6);
  - a record goes to bucket #{i : S_i precedes or equals it} (Fig. 1 step 9);
    pads are not routed;
  - bucket c of the group goes to the c-th subgroup of h = g/k processors: its
    segments, in source-processor order (Fig. 1 step 11), are cut into h
    consecutive parts at floor(N_c*j/h), j = 0..h, and the j-th processor of
    the subgroup merges the pieces of part j stably, ties to the earlier
    source (Fig. 1 step 12; Sec. 5.1.1).
* After round m every processor holds one bucket, sorted; the output is the
  buckets in processor order.

m = 1 is Sort_Det_BSP with R = p virtual processors exactly.

Keys are uint32, int32, float32 or float64; phi maps a key's bits to an
unsigned integer whose order is the key order (IEEE 754 totalOrder for
floats).  Everything here is plain numpy; the sort and merge steps use numpy's
lexsort on (pad, phi, tag), which is exact.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

REC = np.dtype([("pad", np.uint8), ("phi", np.uint64), ("tag", np.int64), ("pos", np.int64)])


def phi(keys: np.ndarray) -> np.ndarray:
    """Order-preserving map of a key's bits to an unsigned integer."""
    keys = np.ascontiguousarray(keys)
    if keys.dtype == np.uint32:
        return keys.astype(np.uint64)
    if keys.dtype == np.int32:
        return (keys.view(np.uint32) ^ np.uint32(0x80000000)).astype(np.uint64)
    if keys.dtype == np.float32:
        u = keys.view(np.uint32)
        return np.where(u >> 31 == 1, ~u, u | np.uint32(0x80000000)).astype(np.uint64)
    if keys.dtype == np.float64:
        u = keys.view(np.uint64)
        return np.where(u >> np.uint64(63) == 1, ~u, u | np.uint64(1 << 63))
    raise TypeError(f"unsupported key type {keys.dtype}")


def _sorted(recs: np.ndarray) -> np.ndarray:
    """Records in the total order (pad, phi, tag)."""
    return recs[np.lexsort((recs["tag"], recs["phi"], recs["pad"]))]


def _precedes_or_equals(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Elementwise a <= b in the total order (broadcasting)."""
    return (a["pad"] < b["pad"]) | ((a["pad"] == b["pad"]) & (
        (a["phi"] < b["phi"]) | ((a["phi"] == b["phi"]) & (a["tag"] <= b["tag"]))))


@dataclass
class Round:
    """One group of one round: its first processor, its size g, the segment
    length x of its regular sample, its k-1 splitters and its k bucket sizes
    (keys only)."""
    first: int
    size: int
    x: int
    splitters: np.ndarray          # k-1 records
    bucket_sizes: np.ndarray       # k counts of real keys


@dataclass
class IterResult:
    keys: np.ndarray               # sorted keys
    positions: np.ndarray          # input position of each output key (a stable argsort)
    bucket_sizes: np.ndarray       # p: keys each processor holds at the end
    rounds: list                   # rounds[t]: the Round of every group of round t+1
    loads: np.ndarray              # (m+1) x p: keys each processor holds before round 1 and after each round
    proc_of: np.ndarray            # final processor of every input position


def _round_count(p: int, k: int) -> int:
    if k < 2:
        raise ValueError("k must be at least 2")
    m, q = 0, 1
    while q < p:
        q *= k
        m += 1
    if q != p:
        raise ValueError("p must be a power of k")
    return m


def sort_iterative(keys: np.ndarray, p: int, k: int, s: int) -> IterResult:
    """Sort by m = log_k(p) rounds of k-way regular-oversampling partitioning."""
    keys = np.ascontiguousarray(keys)
    n = keys.shape[0]
    if p < 1 or s < 1:
        raise ValueError("p and s must be positive")
    m = 0 if p == 1 else _round_count(p, k)
    mb = -(-n // p) if n else 0
    M0 = s * max(1, -(-mb // s))
    f = phi(keys)

    # Fig. 1 step 3: contiguous blocks, each sorted
    procs = []
    for r in range(p):
        lo, hi = min(n, r * mb), min(n, (r + 1) * mb)
        recs = np.zeros(hi - lo, REC)
        recs["phi"] = f[lo:hi]
        recs["tag"] = r * M0 + np.arange(hi - lo)
        recs["pos"] = np.arange(lo, hi)
        procs.append(_sorted(recs))
    loads = [np.array([len(a) for a in procs], np.int64)]
    rounds = []
    # pads of round 1 take the tags r*M0 + j of the padded blocks (Lemma 5.1's
    # proof); pads of later rounds take tags above every round-1 tag
    pad_base = 0

    g = p
    for t in range(m):
        new = [None] * p
        this = []
        for first in range(0, p, g):
            group = procs[first:first + g]
            L = max(len(a) for a in group)
            Mg = s * max(1, -(-L // s))
            x = Mg // s
            # Fig. 1 step 4: pad, then the records at positions j*x - 1
            sample = []
            for r, a in enumerate(group):
                pads = np.zeros(Mg - len(a), REC)
                pads["pad"] = 1
                pads["phi"] = np.uint64(0xFFFFFFFFFFFFFFFF)
                pads["tag"] = pad_base + (first + r) * Mg + len(a) + np.arange(Mg - len(a))
                pads["pos"] = -1
                padded = np.concatenate([a, pads])
                sample.append(padded[np.arange(1, s + 1) * x - 1])
            # Fig. 1 steps 5-6: sort the sample, splitters of rank i*q
            Y = _sorted(np.concatenate(sample))
            q = g * s // k
            S = Y[np.arange(1, k) * q - 1]
            # Fig. 1 step 9: bucket = number of splitters at or below the record
            segs = []
            for a in group:
                b = _precedes_or_equals(S[None, :], a[:, None]).sum(axis=1) if len(a) else np.zeros(0, int)
                segs.append([a[b == c] for c in range(k)])
            sizes = np.array([sum(len(sg[c]) for sg in segs) for c in range(k)], np.int64)
            this.append(Round(first, g, x, S.copy(), sizes))
            # Fig. 1 steps 10-12: bucket c to subgroup c, cut into h parts, each merged
            h = g // k
            for c in range(k):
                pieces = [sg[c] for sg in segs]  # source-processor order
                allc = np.concatenate(pieces) if pieces else np.zeros(0, REC)
                Nc = len(allc)
                for j in range(h):
                    part = allc[Nc * j // h: Nc * (j + 1) // h]
                    new[first + c * h + j] = _sorted(part)
        procs = new
        pad_base = max(pad_base, p * M0) + p * max(r.x for r in this) * s
        rounds.append(this)
        loads.append(np.array([len(a) for a in procs], np.int64))
        g //= k

    out = np.concatenate(procs) if procs else np.zeros(0, REC)
    positions = out["pos"].astype(np.int64)
    proc_of = np.empty(n, np.int64)
    for r, a in enumerate(procs):
        proc_of[a["pos"]] = r
    return IterResult(keys[positions], positions, np.array([len(a) for a in procs], np.int64),
                      rounds, np.stack(loads), proc_of)
