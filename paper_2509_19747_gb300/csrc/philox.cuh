// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11)
// and the seeded streams of the RandRAND test matrices.
//
// The paper draws X from oblivious subspace embeddings (Sec. 2) but fixes no
// generator.  The streams below make every random matrix a pure function of
// (seed, position), so any thread can draw any entry with no state:
//   Gaussian Omega (stream 2): counter (i, j>>2, 2, 0) -> 4 normals for
//     columns 4(j>>2) .. 4(j>>2)+3 of row i, scaled by 1/sqrt(k);
//   sparse-sign rows of Omega (stream 2) / columns of Theta (stream 3):
//     counters (line, t, stream, 0), t = 0, 1, ..., two candidates per draw
//     (column = mulhi(w_even, ncols), sign = top bit of w_odd), duplicates
//     within a line skipped, gamma accepted per line;
//   power-iteration start vectors (stream 4): counter (i, 0, 4, 0);
//   SRHT (X = l^-1/2 S H D, the first n of s columns, s = 2^ceil(log2 n)):
//     sign d_i negative iff the top bit of word 0 of counter (i, 0, 5, 0) is
//     set; row j of X is row pi(j) of the Sylvester Walsh-Hadamard matrix,
//     pi a keyed permutation of [0, s): four balanced Feistel rounds on b
//     bits (b = log2 s, or b + 1 with cycle-walking when b is odd), round r
//     mapping (L, R) to (R, L ^ (word 0 of counter (R, r, 6, 0) mod 2^(b/2)));
//   multi-level embedding X = X2 X1 (Sec. 2 eq:multilevelose): column i of
//     X1 (l1 x n) by the sparse-sign recipe on stream 7 with l1 candidates;
//     X2^T (l1 x k) by the Gaussian recipe on stream 8, counter (r, j>>2, 8,
//     0) for row r, scaled by 1/sqrt(k).
// Uniforms carry 24 bits, u = ((w >> 8) + 0.5) 2^-24, exact in float32.
#pragma once
#include <cstdint>

namespace rr {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

constexpr uint32_t kStreamOmega = 2;
constexpr uint32_t kStreamTheta = 3;
constexpr uint32_t kStreamPower = 4;
constexpr uint32_t kStreamSrhtSign = 5;
constexpr uint32_t kStreamSrhtPerm = 6;
constexpr uint32_t kStreamMlSparse = 7;
constexpr uint32_t kStreamMlGauss = 8;

struct U32x4 {
  uint32_t v[4];
};

__host__ __device__ inline U32x4 philox4x32_10(U32x4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += kPhiloxW0;
      k1 += kPhiloxW1;
    }
    const uint64_t p0 = (uint64_t)kPhiloxM0 * c.v[0];
    const uint64_t p1 = (uint64_t)kPhiloxM1 * c.v[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    U32x4 o;
    o.v[0] = hi1 ^ c.v[1] ^ k0;
    o.v[1] = lo1;
    o.v[2] = hi0 ^ c.v[3] ^ k1;
    o.v[3] = lo0;
    c = o;
  }
  return c;
}

__host__ __device__ inline U32x4 philox_draw(uint64_t seed, uint32_t c0, uint32_t c1,
                                             uint32_t c2) {
  U32x4 c = {{c0, c1, c2, 0u}};
  return philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
}

// one pass of the SRHT row permutation on `bits` bits (bits even, > 0)
__host__ __device__ inline uint64_t srht_feistel(uint64_t x, int bits, uint64_t seed) {
  const int h = bits / 2;
  const uint64_t mask = (1ull << h) - 1;
  uint64_t L = x >> h, R = x & mask;
  for (int r = 0; r < 4; ++r) {
    const uint64_t f = philox_draw(seed, (uint32_t)R, (uint32_t)r, kStreamSrhtPerm).v[0] & mask;
    const uint64_t t = L ^ f;
    L = R;
    R = t;
  }
  return (L << h) | R;
}

// pi(j) for the SRHT of width s = 2^b (j < s); the cycle-walk ends within s
// steps because pi restricted to a cycle returns to [0, s)
__host__ __device__ inline int64_t srht_row(int64_t j, int64_t s, uint64_t seed) {
  int b = 0;
  while ((1ll << b) < s) ++b;
  if (b == 0) return 0;
  const int bits = (b % 2 == 0) ? b : b + 1;
  uint64_t x = srht_feistel((uint64_t)j, bits, seed);
  for (int64_t it = 0; x >= (uint64_t)s && it < 2 * s; ++it) x = srht_feistel(x, bits, seed);
  return (int64_t)x;
}

// 24-bit uniform in (0,1), exact in float and double.
__device__ inline float u24f(uint32_t w) { return ((float)(w >> 8) + 0.5f) * 5.9604644775390625e-8f; }
__device__ inline double u24d(uint32_t w) { return ((double)(w >> 8) + 0.5) * 5.9604644775390625e-8; }

// Box-Muller: four words -> four N(0,1), in double.
__device__ inline void box_muller4(const U32x4& w, double z[4]) {
  const double r01 = sqrt(-2.0 * log(u24d(w.v[0])));
  const double r23 = sqrt(-2.0 * log(u24d(w.v[2])));
  double s01, c01, s23, c23;
  sincospi(2.0 * u24d(w.v[1]), &s01, &c01);
  sincospi(2.0 * u24d(w.v[3]), &s23, &c23);
  z[0] = r01 * c01;
  z[1] = r01 * s01;
  z[2] = r23 * c23;
  z[3] = r23 * s23;
}

// Box-Muller in float (the float32 / bf16 paths).
__device__ inline void box_muller4(const U32x4& w, float z[4]) {
  const float r01 = sqrtf(-2.0f * logf(u24f(w.v[0])));
  const float r23 = sqrtf(-2.0f * logf(u24f(w.v[2])));
  float s01, c01, s23, c23;
  sincospif(2.0f * u24f(w.v[1]), &s01, &c01);
  sincospif(2.0f * u24f(w.v[3]), &s23, &c23);
  z[0] = r01 * c01;
  z[1] = r01 * s01;
  z[2] = r23 * c23;
  z[3] = r23 * s23;
}

// gamma distinct indices in [0, ncols) and signs for line `line` of a
// sparse-sign matrix; gamma <= kMaxGamma.
constexpr int kMaxGamma = 16;
__device__ inline void sparse_sign_line(uint64_t seed, uint32_t stream, uint32_t line,
                                        uint32_t ncols, int gamma, int32_t* cols,
                                        int8_t* sgn) {
  int filled = 0;
  // gamma <= ncols is checked on the host, so every line completes; the cap
  // only bounds the loop (expected draws ~ gamma/2 for gamma << ncols).
  for (uint32_t t = 0; filled < gamma && t < (1u << 20); ++t) {
    const U32x4 w = philox_draw(seed, line, t, stream);
#pragma unroll
    for (int pair = 0; pair < 2; ++pair) {
      if (filled >= gamma) break;
      const uint32_t c = (uint32_t)(((uint64_t)w.v[2 * pair] * ncols) >> 32);
      bool dup = false;
      for (int q = 0; q < filled; ++q) dup |= (cols[q] == (int32_t)c);
      if (dup) continue;
      cols[filled] = (int32_t)c;
      sgn[filled] = (w.v[2 * pair + 1] >> 31) ? (int8_t)-1 : (int8_t)1;
      ++filled;
    }
  }
  for (uint32_t c = 0; filled < gamma && c < ncols; ++c) {  // unreachable in practice
    bool dup = false;
    for (int q = 0; q < filled; ++q) dup |= (cols[q] == (int32_t)c);
    if (!dup) { cols[filled] = (int32_t)c; sgn[filled] = 1; ++filled; }
  }
}

}  // namespace rr
