"""Sparse-sign sketch drawn from the SplitMix64 stream (oracle; test infrastructure).

The paper (Section 3) lists "sparse dimension reduction maps" among the
oblivious subspace embeddings and uses the Count sketch (Section 5.2), a sparse
map with one +-1 per column of Theta^T.  The sparse-sign sketch used here is the
same kind of map with ``zeta`` nonzeros +-1 per column: S is d x n (S = Theta^T),
column r of S holds ``zeta`` distinct row indices in [0, d) with random signs.
Values are +-1 and unscaled; a positive scalar factor on S would only rescale
the R factor of the sketch, which the following CholQR absorbs exactly.

Index/sign generation (bit-exact between the oracle and the CUDA library, which
implement it independently from this definition):

* SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): the i-th output (i >= 1) of
  the stream seeded with ``seed`` is ``mix(seed + i * 0x9E3779B97F4A7C15)`` with
  ``mix(z) = z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27;
  z *= 0x94D049BB133111EB; z ^= z >> 31`` (all mod 2^64).
* Row r of V owns outputs i = 64 r + c + 1 for draw counter c = 0..63.
* Draw c gives the candidate index ``((h >> 32) * d) >> 32`` (multiply-shift
  range reduction) and sign -1 if bit 0 of h is set, else +1.
* A candidate equal to an index already taken by the row is skipped; the row's
  entries are the first ``zeta`` distinct candidates in draw order.  A row that
  has not found ``zeta`` distinct indices after 64 draws is an error.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
MIX1 = np.uint64(0xBF58476D1CE4E5B9)
MIX2 = np.uint64(0x94D049BB133111EB)
DRAWS_PER_ROW = 64


class SketchError(ValueError):
    pass


def splitmix64_mix(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * MIX1
        z = (z ^ (z >> np.uint64(27))) * MIX2
    return z ^ (z >> np.uint64(31))


def splitmix64_output(seed: int, i) -> np.ndarray:
    """i-th output (i >= 1) of the SplitMix64 stream seeded with ``seed``."""
    i = np.asarray(i, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed) + i * GAMMA
    return splitmix64_mix(state)


def draw(seed: int, rows: np.ndarray, c: int) -> np.ndarray:
    rows = np.asarray(rows, dtype=np.uint64)
    with np.errstate(over="ignore"):
        i = rows * np.uint64(DRAWS_PER_ROW) + np.uint64(c + 1)
    return splitmix64_output(seed, i)


def candidate_index(h: np.ndarray, d: int) -> np.ndarray:
    return (((h >> np.uint64(32)) * np.uint64(d)) >> np.uint64(32)).astype(np.int64)


def candidate_sign(h: np.ndarray) -> np.ndarray:
    return np.where((h & np.uint64(1)) != 0, -1, 1).astype(np.int8)


def sparse_sign_entries(row0: int, nrows: int, d: int, zeta: int, seed: int):
    """Indices (nrows x zeta, int32) and signs (nrows x zeta, int8) of S's columns."""
    if not (1 <= zeta <= d):
        raise SketchError(f"need 1 <= zeta <= d, got zeta={zeta}, d={d}")
    idx = np.full((nrows, zeta), -1, dtype=np.int64)
    sgn = np.zeros((nrows, zeta), dtype=np.int8)
    cnt = np.zeros(nrows, dtype=np.int64)
    allrows = np.arange(nrows, dtype=np.int64)
    for c in range(DRAWS_PER_ROW):
        need = cnt < zeta
        if not need.any():
            break
        r = allrows[need]
        h = draw(seed, r + row0, c)
        ix = candidate_index(h, d)
        dup = (idx[r] == ix[:, None]).any(axis=1)
        take = ~dup
        rt = r[take]
        idx[rt, cnt[rt]] = ix[take]
        sgn[rt, cnt[rt]] = candidate_sign(h[take])
        cnt[rt] += 1
    if (cnt < zeta).any():
        raise SketchError("a row did not find zeta distinct indices in 64 draws")
    return idx.astype(np.int32), sgn


class Sketch:
    """S (d x n) with ``zeta`` +-1 entries per column, materialised for the oracle."""

    def __init__(self, n: int, d: int, zeta: int, seed: int):
        self.n, self.d, self.zeta, self.seed = int(n), int(d), int(zeta), int(seed)
        self.idx, self.sign = sparse_sign_entries(0, self.n, self.d, self.zeta, self.seed)
        import scipy.sparse as sp
        rows = np.repeat(np.arange(self.n), self.zeta)
        self.S = sp.csr_matrix(
            (self.sign.ravel().astype(np.float64), (self.idx.ravel(), rows)),
            shape=(self.d, self.n))

    def apply(self, W: np.ndarray) -> np.ndarray:
        """S @ W for W with n rows (sparse-times-dense; exact sums up to rounding order)."""
        W = np.asarray(W, dtype=np.float64)
        return np.asarray(self.S @ W)

    def dense(self) -> np.ndarray:
        return self.S.toarray()
