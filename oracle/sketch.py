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


# --- Gaussian and Count-Gauss sketches (Section 5.2) ---------------------------------
# Gaussian entries from the SplitMix64 stream (written from the published
# definitions, independently of the CUDA library):
#   stream seed  seed_g = seed XOR GAUSS_SALT
#   entry (k, r) of a Gaussian map with d rows uses output i = r * d + k + 1;
#   m1 = top 24 bits of h, u1 = float32(m1 + 1/2) / 2^24 in (0, 1) (the sum rounded to
#   float32), u2 = (bits 16..39 of h) / 2^24;
#   theta = sqrt(-2 ln u1) cos(2 pi u2) (Box and Muller 1958), rounded to float32
#   (the CUDA side evaluates it in float32 arithmetic, within a few float32 ulps).
GAUSS_SALT = 0x2545F4914F6CDD1D


def gaussian_entries(seed: int, rows: np.ndarray, d: int) -> np.ndarray:
    """theta[r, k] for the given rows r and k < d (len(rows) x d, float64 holding
    float32 values)."""
    rows = np.asarray(rows, dtype=np.uint64)
    k = np.arange(d, dtype=np.uint64)
    with np.errstate(over="ignore"):
        i = rows[:, None] * np.uint64(d) + k[None, :] + np.uint64(1)
    h = splitmix64_output(int(np.uint64(seed) ^ np.uint64(GAUSS_SALT)), i)
    u1 = ((h >> np.uint64(40)).astype(np.float64) + 0.5).astype(np.float32).astype(np.float64) * 2.0 ** -24
    u2 = ((h >> np.uint64(16)) & np.uint64(0xFFFFFF)).astype(np.float64) * 2.0 ** -24
    g = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return g.astype(np.float32).astype(np.float64)


class GaussianSketch:
    """Dense Gaussian map S (d x n), entries N(0, 1) (unscaled, like the sparse
    sign map: a scalar factor only rescales the sketch's R)."""

    def __init__(self, n: int, d: int, seed: int):
        self.n, self.d, self.seed = int(n), int(d), int(seed)
        self.S = gaussian_entries(self.seed, np.arange(self.n), self.d).T.copy()

    def apply(self, W: np.ndarray) -> np.ndarray:
        return self.S @ np.asarray(W, dtype=np.float64)

    def dense(self) -> np.ndarray:
        return self.S


class CountGaussSketch:
    """S = G C (Section 5.2, Count-Gaussian): C is the d_inner x n Count sketch (one
    +-1 per column: the sparse-sign map with zeta = 1 and the same seed), G the
    d x d_inner Gaussian map whose entry (k, j) is gaussian_entries(seed, [j], d)[k]."""

    def __init__(self, n: int, d: int, d_inner: int, seed: int):
        self.n, self.d, self.d_inner, self.seed = int(n), int(d), int(d_inner), int(seed)
        self.C = Sketch(self.n, self.d_inner, 1, self.seed)
        self.G = gaussian_entries(self.seed, np.arange(self.d_inner), self.d).T.copy()

    def apply(self, W: np.ndarray) -> np.ndarray:
        return self.G @ self.C.apply(W)

    def dense(self) -> np.ndarray:
        return self.G @ self.C.dense()
