// Sparse-sign sketch from the SplitMix64 stream, and Gaussian entries (oracle; test
// infrastructure).  Section 3 lists sparse dimension-reduction maps among the oblivious
// subspace embeddings and Section 5.2 uses the Count sketch, the map with one +-1 per
// column; the sparse-sign map has zeta distinct +-1 entries per column of S (d x n).
// Definitions (the CUDA library implements the same definitions independently):
//   * SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): output i >= 1 of the stream
//     seeded with `seed` is mix(seed + i * 0x9E3779B97F4A7C15), mix(z): z ^= z >> 30,
//     z *= 0xBF58476D1CE4E5B9, z ^= z >> 27, z *= 0x94D049BB133111EB, z ^= z >> 31;
//   * row r of V owns outputs 64 r + c + 1 for its draws c = 0..63; draw c gives the
//     candidate index ((h >> 32) * d) >> 32 and sign -1 when bit 0 of h is set;
//   * the row's entries are its first zeta distinct candidates in draw order.
#include "common.hpp"

namespace oracle {

static uint64_t mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t splitmix64_output(uint64_t seed, uint64_t i) { return mix(seed + i * 0x9E3779B97F4A7C15ULL); }

bool sparse_sign_entries(int64_t row0, int64_t nrows, int d, int zeta, uint64_t seed,
                         int32_t* idx, int8_t* sgn) {
  if (zeta < 1 || zeta > d) return false;
  for (int64_t r = 0; r < nrows; ++r) {
    const uint64_t row = (uint64_t)(row0 + r);
    int cnt = 0;
    for (int c = 0; c < 64 && cnt < zeta; ++c) {
      const uint64_t h = splitmix64_output(seed, row * 64 + (uint64_t)c + 1);
      const int32_t ix = (int32_t)(((h >> 32) * (uint64_t)d) >> 32);
      bool dup = false;
      for (int t = 0; t < cnt; ++t) dup = dup || idx[r * zeta + t] == ix;
      if (dup) continue;
      idx[r * zeta + cnt] = ix;
      sgn[r * zeta + cnt] = (h & 1ULL) ? -1 : 1;
      ++cnt;
    }
    if (cnt < zeta) return false;
  }
  return true;
}

Sketch::Sketch(int64_t n_, int d_, int zeta_, uint64_t seed_)
    : n(n_), d(d_), zeta(zeta_), seed(seed_), idx((size_t)(n_ * zeta_)), sgn((size_t)(n_ * zeta_)) {
  if (!sparse_sign_entries(0, n, d, zeta, seed, idx.data(), sgn.data()))
    throw std::runtime_error("sketch: a row did not find zeta distinct indices");
}

// S W: row r of W is added (with its signs) to the rows idx[r, :] of the result.
Mat Sketch::apply(const Mat& W) const {
  Mat out(d, W.n);
  for (int64_t j = 0; j < W.n; ++j)
    for (int64_t r = 0; r < n; ++r)
      for (int t = 0; t < zeta; ++t) out(idx[r * zeta + t], j) += sgn[r * zeta + t] * W(r, j);
  return out;
}

// Entry (k, r) of a Gaussian map with d rows (Section 5.2): stream seed
// seed ^ 0x2545F4914F6CDD1D, output r d + k + 1; u1 = float32(m1 + 1/2) / 2^24 with m1
// the top 24 bits of h (the sum rounded to float32), u2 = (bits 16..39 of h) / 2^24;
// theta = sqrt(-2 ln u1) cos(2 pi u2) (Box and Muller 1958) rounded to float32.
double gaussian_entry(uint64_t seed, uint64_t r, int k, int d) {
  const uint64_t h = splitmix64_output(seed ^ 0x2545F4914F6CDD1DULL, r * (uint64_t)d + (uint64_t)k + 1);
  const double u1 = (double)(float)((double)(h >> 40) + 0.5) * std::ldexp(1.0, -24);
  const double u2 = (double)((h >> 16) & 0xFFFFFFULL) * std::ldexp(1.0, -24);
  const double g = std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2);
  return (double)(float)g;
}

}  // namespace oracle
