"""Sampled key-degree histogram, written out plainly -- TEST INFRASTRUCTURE
ONLY (only tests/ may use it).  The definition the chooser's features use:

* row i of an n-row column is sampled iff sample_hash(i, seed) % mod == 0,
  with sample_hash the 32-bit finalizer of MurmurHash3 applied to
  (i mod 2^32) xor seed (Austin Appleby's public-domain mixer);
* a sampled key's estimated degree is c * n / m, c its count among the m
  sampled rows;
* its bucket is the largest b in [0, 31] with c * n >= m * 2^b (0 when
  c * n < 2m), i.e. floor(log2(degree)) computed exactly in integers;
* the histogram is the fraction of distinct sampled keys per bucket."""

import numpy as np

M32 = 0xFFFFFFFF


def sample_hash(i, seed):
    h = (int(i) & M32) ^ (int(seed) & M32)
    h ^= h >> 16
    h = (h * 0x85EBCA6B) & M32
    h ^= h >> 13
    h = (h * 0xC2B2AE35) & M32
    h ^= h >> 16
    return h


def degree_histogram(col, mod=100, seed=0):
    col = np.asarray(col)
    n = len(col)
    sampled = [int(col[i]) for i in range(n) if sample_hash(i, seed) % mod == 0]
    m = len(sampled)
    out = np.zeros(32, dtype=np.float64)
    if m == 0:
        return out
    counts = {}
    for k in sampled:
        counts[k] = counts.get(k, 0) + 1
    for c in counts.values():
        b = 0
        while b < 31 and c * n >= m * (1 << (b + 1)):
            b += 1
        out[b] += 1
    return out / len(counts)
