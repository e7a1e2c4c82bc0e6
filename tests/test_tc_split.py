"""The arithmetic the tensor-core GNN layers rest on, checked on the CPU with a
bit-level bfloat16 round-to-nearest-even (itself checked against torch's conversion):

* a float32 value splits into three bfloat16 pieces x0 = bf16(x), x1 = bf16(x - x0),
  x2 = bf16(x - x0 - x1) with every difference exact in float32 and x = x0 + x1 + x2
  exactly (x has 24 significant bits; each piece takes 8);
* the product of two bfloat16 values is exact in float32 (8 x 8 significant bits);
* the hi/lo split of the weight-gradient operands, u = u_hi + u_lo + r, leaves
  |r| <= 2^-16 |u|, so the four piece products give u * v within 2^-15 relative.
No GPU."""
import numpy as np
import pytest


def bf16_rn(x: np.ndarray) -> np.ndarray:
    """float32 -> nearest bfloat16 (ties to even), returned as float32 (finite input)."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def _samples(n: int, seed: int, lo: int = -100, hi: int = 100) -> np.ndarray:
    rng = np.random.default_rng(seed)
    mant = rng.uniform(1.0, 2.0, n)
    exp = rng.integers(lo, hi, n)
    sign = rng.choice([-1.0, 1.0], n)
    x = (sign * mant * np.exp2(exp)).astype(np.float32)
    # binade edges and values whose rounding carries into the next binade
    edges = np.array([1.0, 1.0 + 2.0 ** -23, 2.0 - 2.0 ** -23, 1.0 + 2.0 ** -8,
                      1.0 + 2.0 ** -8 + 2.0 ** -9, 1.5 + 2.0 ** -16 + 2.0 ** -23, 3.999999],
                     dtype=np.float32)
    return np.concatenate([x, edges, -edges])


def test_bf16_emulation_matches_torch():
    torch = pytest.importorskip("torch")
    x = _samples(200_000, 1)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(bf16_rn(x), ref)


def test_three_pieces_are_exact():
    x = _samples(500_000, 2)
    x0 = bf16_rn(x)
    r1 = x - x0                                   # float32 arithmetic
    assert np.array_equal(r1.astype(np.float64), x.astype(np.float64) - x0.astype(np.float64))
    x1 = bf16_rn(r1)
    r2 = r1 - x1
    assert np.array_equal(r2.astype(np.float64), r1.astype(np.float64) - x1.astype(np.float64))
    x2 = bf16_rn(r2)
    assert np.array_equal(x2, r2)                 # the last remainder fits in bfloat16
    total = x0.astype(np.float64) + x1.astype(np.float64) + x2.astype(np.float64)
    assert np.array_equal(total, x.astype(np.float64))


def test_bf16_products_exact_in_float32():
    a = bf16_rn(_samples(300_000, 3, -60, 60))
    b = bf16_rn(_samples(300_000, 4, -60, 60))
    p32 = (a * b).astype(np.float64)              # float32 product
    assert np.array_equal(p32, a.astype(np.float64) * b.astype(np.float64))


def test_hi_lo_split_bound():
    u = _samples(300_000, 5)
    v = _samples(300_000, 6)

    def split(x):
        hi = bf16_rn(x)
        return hi, bf16_rn(x - hi)

    uh, ul = split(u)
    vh, vl = split(v)
    u64, v64 = u.astype(np.float64), v.astype(np.float64)
    ru = np.abs(u64 - uh.astype(np.float64) - ul.astype(np.float64))
    assert np.all(ru <= 2.0 ** -16 * np.abs(u64))
    prod = ((uh.astype(np.float64) + ul) * (vh.astype(np.float64) + vl))
    assert np.all(np.abs(prod - u64 * v64) <= 2.0 ** -15 * np.abs(u64 * v64))
