"""Row sampling for skeletonization (Sec. II-B).

Part of the oracle (test infrastructure only).

The paper says only that nearest-neighbour information is used to sample the
block K_{[1:N] alpha} whose pivoted QR yields the skeletons.  The reading used
throughout this project, for a non-root node alpha owning permuted positions
[o, o + n):

1. candidates: every kNN entry of every point of alpha that lies outside alpha,
   as a permuted position; ``hits(c)`` is how often c occurs;
2. n_samp = min(samp_factor * s_max, N - n); keep the first n_samp distinct
   candidates in the order (hits descending, position ascending);
3. if fewer than n_samp were kept, fill uniformly without replacement from the
   complement of alpha.  The node draws from its own SplitMix64 stream, whose
   state starts at s0 = splitmix64(splitmix64(seed) ^ uid) with uid = 2^l + i for
   node (l, i): draw q = 0, 1, 2, ... is r_q = splitmix64(s0 + q * gamma) (mod 2^64,
   gamma = 0x9E3779B97F4A7C15), i.e. the q-th output of that stream.  Take
   j = r_q mod (N - n) and map it to the position j if j < o, else j + n; skip
   positions already taken; when n_samp = N - n the sample is the whole complement;
4. return the sample in ascending position order.
"""
from __future__ import annotations

import numpy as np

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


def splitmix64(x: int) -> int:
    """One output of SplitMix64 (Steele, Lea, Flood 2014) for the 64-bit state ``x``.

    The state is advanced by the golden gamma 0x9E3779B97F4A7C15 and the result is
    passed through the variant-13 finaliser (shifts 30, 27, 31).
    """
    z = (x + GAMMA) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def sample_rows(knn_pos: np.ndarray, o: int, n: int, N: int, n_samp: int,
                seed: int, uid: int) -> np.ndarray:
    """Sampled target rows (permuted positions) for the node owning [o, o + n).

    ``knn_pos`` holds the kNN lists of the node's points as permuted positions,
    shape (n, kappa).
    """
    n_samp = min(n_samp, N - n)
    if n_samp <= 0:
        return np.empty(0, dtype=np.int64)
    if n_samp == N - n:
        return np.concatenate([np.arange(0, o), np.arange(o + n, N)]).astype(np.int64)
    cand = knn_pos.ravel()
    cand = cand[(cand < o) | (cand >= o + n)]
    chosen = []
    if cand.size:
        vals, counts = np.unique(cand, return_counts=True)
        order = np.lexsort((vals, -counts))          # hits descending, position ascending
        chosen = [int(v) for v in vals[order[:n_samp]]]
    taken = set(chosen)
    q = 0
    comp = N - n
    s0 = splitmix64(splitmix64(seed & MASK64) ^ uid)
    while len(chosen) < n_samp:
        r = splitmix64((s0 + q * GAMMA) & MASK64)
        j = r % comp
        pos = j if j < o else j + n
        if pos not in taken:
            taken.add(pos)
            chosen.append(pos)
        q += 1
    return np.sort(np.array(chosen, dtype=np.int64))
