"""ORACLE (test infrastructure only) -- counter-based random numbers.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never does.

The paper draws its test matrix X from an oblivious subspace embedding
(Sec. 2: Gaussian entries N(0, 1/l); sparse random operators with gamma
entries +-1/sqrt(gamma) per column) but fixes no generator.  So that the
oracle and the CUDA library can draw the *same* random matrices from a seed,
each implements, independently, Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11) from its published
definition, and the derived streams below.

Stream layout (counter = (c0, c1, c2, c3), key = (seed lo 32, seed hi 32)):

* Gaussian test matrix Omega (n x k), stream 2: counter (i, j >> 2, 2, 0)
  gives four words -> four N(0,1) numbers for columns 4(j>>2) .. 4(j>>2)+3
  of row i; Omega_ij = z / sqrt(k).
* Sparse-sign Omega (n x k, gamma nonzeros per row = per column of X),
  stream 2: row i reads counters (i, t, 2, 0), t = 0, 1, ...; each block of
  four words gives two candidates (w0 -> column, w1 -> sign) and (w2, w3);
  the column is floor(w * k / 2^32), the sign is negative iff the top bit of
  the sign word is set; a candidate whose column was already chosen for the
  row is skipped; the row is complete after gamma accepted columns.
  Nonzero value = sign / sqrt(gamma).
* Theta (l_sk x n, gamma_sk nonzeros per column), stream 3: the same recipe
  with column i of Theta in place of row i of Omega and l_sk in place of k.
* Power-iteration start vectors, stream 4: counter (i, 0, 4, 0), word c
  gives entry i of start vector c (c = 0, 1) as N(0,1) numbers.
* SRHT (Sec. 2, fast randomized transforms): X = l^-1/2 S H D, first n of s
  columns (s the smallest power of two >= n).  Sign d_i (stream 5): negative
  iff the top bit of word 0 of counter (i, 0, 5, 0) is set.  H: Sylvester
  Walsh-Hadamard, H[r][i] = (-1)^popcount(r & i).  S (uniform subsampling
  without replacement): row j of X is row pi(j) of H, pi a keyed permutation
  of [0, s): four balanced Feistel rounds on b bits (b = log2 s; b + 1 when
  odd, then cycle-walking back into [0, s)), round r mapping (L, R) to
  (R, L xor (word 0 of counter (R, r, 6, 0)) mod 2^(b/2)).
* Multi-level embedding X = X2 X1 (Sec. 2 eq:multilevelose): X1 (l1 x n,
  gamma1 nonzeros +-1/sqrt(gamma1) per column) by the sparse-sign recipe on
  stream 7 with column i of X1 as line i and l1 candidates; X2 (l x l1)
  Gaussian with entries N(0, 1/l), X2[j][r] from the Gaussian recipe of
  Omega on stream 8 with (r, j) in place of (i, j).  Omega = X^T = X1^T X2^T.

Uniforms use 24 bits so that they are exact in float32 and float64:
u = ((w >> 8) + 0.5) * 2^-24 in (0, 1).  Box-Muller pairs:
(z0, z1) = sqrt(-2 ln u0) (cos 2 pi u1, sin 2 pi u1), likewise (z2, z3).
"""
from __future__ import annotations

import math

import numpy as np

# Philox4x32 round multipliers and Weyl key increments (Salmon et al. 2011).
PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
PHILOX_ROUNDS = 10

STREAM_OMEGA = 2
STREAM_THETA = 3
STREAM_POWER = 4
STREAM_SRHT_SIGN = 5
STREAM_SRHT_PERM = 6
STREAM_ML_SPARSE = 7
STREAM_ML_GAUSS = 8

_MASK32 = np.uint64(0xFFFFFFFF)


def seed_key(seed: int) -> tuple[int, int]:
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32


def philox4x32_10(ctr: np.ndarray, key: tuple[int, int]) -> np.ndarray:
    """Philox4x32 with 10 rounds.

    ctr: (N, 4) array of uint32 counters.  key: two 32-bit words.
    Returns (N, 4) uint32.  Each round maps (R0, R1, R2, R3) to
    (hi(M1 R2) ^ R1 ^ K0, lo(M1 R2), hi(M0 R0) ^ R3 ^ K1, lo(M0 R0)); the key
    advances by the Weyl increments between rounds.
    """
    c = np.asarray(ctr, dtype=np.uint64).reshape(-1, 4)
    r0, r1, r2, r3 = c[:, 0].copy(), c[:, 1].copy(), c[:, 2].copy(), c[:, 3].copy()
    k0 = int(key[0]) & 0xFFFFFFFF
    k1 = int(key[1]) & 0xFFFFFFFF
    m0 = np.uint64(PHILOX_M0)
    m1 = np.uint64(PHILOX_M1)
    for rnd in range(PHILOX_ROUNDS):
        if rnd > 0:
            k0 = (k0 + PHILOX_W0) & 0xFFFFFFFF
            k1 = (k1 + PHILOX_W1) & 0xFFFFFFFF
        p0 = r0 * m0            # < 2^64: exact in uint64
        p1 = r2 * m1
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        r0, r1, r2, r3 = (hi1 ^ r1 ^ np.uint64(k0), lo1,
                          hi0 ^ r3 ^ np.uint64(k1), lo0)
    return np.stack([r0, r1, r2, r3], axis=1).astype(np.uint32)


def uniform24(w: np.ndarray) -> np.ndarray:
    """Map 32-bit words to uniforms in (0, 1) with 24 bits: exact in f32."""
    return ((np.asarray(w, dtype=np.uint64) >> np.uint64(8)).astype(np.float64) + 0.5) * 2.0 ** -24


def box_muller4(words: np.ndarray) -> np.ndarray:
    """(N, 4) words -> (N, 4) standard normals, in float64."""
    u = uniform24(words)
    r01 = np.sqrt(-2.0 * np.log(u[:, 0]))
    r23 = np.sqrt(-2.0 * np.log(u[:, 2]))
    t01 = 2.0 * np.pi * u[:, 1]
    t23 = 2.0 * np.pi * u[:, 3]
    return np.stack([r01 * np.cos(t01), r01 * np.sin(t01),
                     r23 * np.cos(t23), r23 * np.sin(t23)], axis=1)


def gaussian_normals(n: int, k: int, seed: int, stream: int = STREAM_OMEGA) -> np.ndarray:
    """n x k array of N(0,1) numbers; entry (i, j) from counter (i, j>>2, stream, 0)."""
    q = (k + 3) // 4
    ii, jj = np.meshgrid(np.arange(n, dtype=np.uint64), np.arange(q, dtype=np.uint64), indexing="ij")
    ctr = np.zeros((n * q, 4), dtype=np.uint64)
    ctr[:, 0] = ii.ravel()
    ctr[:, 1] = jj.ravel()
    ctr[:, 2] = stream
    z = box_muller4(philox4x32_10(ctr, seed_key(seed)))
    return z.reshape(n, 4 * q)[:, :k]


def gaussian_omega(n: int, k: int, seed: int) -> np.ndarray:
    """Gaussian test matrix Omega = X^T, entries N(0, 1/k) (Sec. 2)."""
    return gaussian_normals(n, k, seed) / np.sqrt(k)


def sparse_sign_pattern(nrows: int, ncols: int, gamma: int, seed: int,
                        stream: int) -> tuple[np.ndarray, np.ndarray]:
    """For each of `nrows` lines, `gamma` distinct indices in [0, ncols) and
    signs +-1, in acceptance order (see the module docstring)."""
    if gamma > ncols:
        raise ValueError("gamma must not exceed the number of columns")
    key = seed_key(seed)
    cols = np.full((nrows, gamma), -1, dtype=np.int64)
    sgn = np.zeros((nrows, gamma), dtype=np.int8)
    filled = np.zeros(nrows, dtype=np.int64)
    t = 0
    active = np.arange(nrows)
    while active.size:
        ctr = np.zeros((active.size, 4), dtype=np.uint64)
        ctr[:, 0] = active
        ctr[:, 1] = t
        ctr[:, 2] = stream
        w = philox4x32_10(ctr, key).astype(np.uint64)
        for pair in range(2):
            cand = ((w[:, 2 * pair] * np.uint64(ncols)) >> np.uint64(32)).astype(np.int64)
            neg = ((w[:, 2 * pair + 1] >> np.uint64(31)) & np.uint64(1)).astype(bool)
            f = filled[active]
            # unfilled slots hold -1, so comparing against the whole row only
            # tests the columns accepted so far
            dup = (cols[active] == cand[:, None]).any(axis=1)
            take = (f < gamma) & ~dup
            rows_t = active[take]
            cols[rows_t, f[take]] = cand[take]
            sgn[rows_t, f[take]] = np.where(neg[take], -1, 1)
            filled[rows_t] += 1
        active = active[filled[active] < gamma]
        t += 1
    return cols, sgn


def sparse_sign_omega_dense(n: int, k: int, gamma: int, seed: int) -> np.ndarray:
    """Dense n x k copy of the sparse-sign Omega (rows of Omega = columns of
    the sparse random operator X of Sec. 2), values +-1/sqrt(gamma)."""
    cols, sgn = sparse_sign_pattern(n, k, gamma, seed, STREAM_OMEGA)
    Om = np.zeros((n, k))
    rows = np.repeat(np.arange(n), gamma)
    np.add.at(Om, (rows, cols.ravel()), sgn.ravel() / np.sqrt(gamma))
    return Om


def theta_dense(l_sk: int, n: int, gamma_sk: int, seed: int) -> np.ndarray:
    """Dense l_sk x n copy of the sparse embedding Theta of Alg. 3."""
    cols, sgn = sparse_sign_pattern(n, l_sk, gamma_sk, seed, STREAM_THETA)
    Th = np.zeros((l_sk, n))
    rows = np.repeat(np.arange(n), gamma_sk)
    np.add.at(Th, (cols.ravel(), rows), sgn.ravel() / np.sqrt(gamma_sk))
    return Th


def power_start(n: int, which: int, seed: int) -> np.ndarray:
    """Start vector `which` (0 or 1) of the power iterations, N(0,1) entries."""
    return gaussian_normals(n, 4, seed, STREAM_POWER)[:, which].copy()


def round_bf16(a: np.ndarray) -> np.ndarray:
    """Round float64 values to bfloat16 (via float32, round-to-nearest-even)
    and return them as float64."""
    a32 = np.asarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    r = ((u + np.uint64(0x7FFF) + ((u >> np.uint64(16)) & np.uint64(1))) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def round_f32(a: np.ndarray) -> np.ndarray:
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def srht_size(n: int) -> int:
    """The smallest power of two s >= n."""
    s = 1
    while s < n:
        s <<= 1
    return s


def _feistel(x: np.ndarray, bits: int, seed: int) -> np.ndarray:
    h = bits // 2
    mask = np.uint64((1 << h) - 1)
    x = np.asarray(x, dtype=np.uint64)
    L, R = x >> np.uint64(h), x & mask
    for r in range(4):
        ctr = np.zeros((x.size, 4), dtype=np.uint32)
        ctr[:, 0] = R.astype(np.uint32)
        ctr[:, 1] = r
        ctr[:, 2] = STREAM_SRHT_PERM
        f = philox4x32_10(ctr, seed_key(seed))[:, 0].astype(np.uint64) & mask
        L, R = R, L ^ f
    return (L << np.uint64(h)) | R


def srht_rows(k: int, s: int, seed: int) -> np.ndarray:
    """pi(0), ..., pi(k-1): the rows of H that S keeps (distinct)."""
    b = s.bit_length() - 1
    if b == 0:
        return np.zeros(k, dtype=np.int64)
    bits = b if b % 2 == 0 else b + 1
    x = _feistel(np.arange(k, dtype=np.uint64), bits, seed)
    while np.any(x >= np.uint64(s)):          # cycle-walking (bits = b + 1)
        out = x >= np.uint64(s)
        x[out] = _feistel(x[out], bits, seed)
    return x.astype(np.int64)


def srht_signs(n: int, seed: int) -> np.ndarray:
    ctr = np.zeros((n, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(n, dtype=np.uint32)
    ctr[:, 2] = STREAM_SRHT_SIGN
    w = philox4x32_10(ctr, seed_key(seed))[:, 0]
    return np.where(w >> np.uint32(31), -1.0, 1.0)


def srht_omega(n: int, k: int, seed: int) -> np.ndarray:
    """Omega = X^T (n x k): Omega_ij = d_i H[pi(j)][i] / sqrt(k)."""
    s = srht_size(n)
    rows = srht_rows(k, s, seed)
    i = np.arange(n, dtype=np.int64)
    par = np.bitwise_count(i[:, None] & rows[None, :]) & 1
    return srht_signs(n, seed)[:, None] * np.where(par, -1.0, 1.0) * (1.0 / math.sqrt(k))


def multilevel_defaults(n: int, k: int) -> tuple[int, int]:
    """(l1, gamma1) of the multi-level embedding: the paper's experiment with
    sparse + Gaussian embeddings takes density gamma1 = log n and l1 = l log n
    (Sec. 7, inverse-PDE example).  Reading: natural logarithm rounded up,
    gamma1 at most 16 and at most l1."""
    g = max(1, math.ceil(math.log(n)))
    g = min(g, 16)
    return g * k, g


def multilevel_parts(n: int, k: int, l1: int, gamma1: int, seed: int):
    """The two factors of X = X2 X1: the sparse pattern of X1 (for each
    column i, gamma1 distinct rows in [0, l1) and their signs) and the dense
    X2^T (l1 x k), entries N(0, 1/k)."""
    cols, sgn = sparse_sign_pattern(n, l1, gamma1, seed, STREAM_ML_SPARSE)
    X2T = gaussian_normals(l1, k, seed, STREAM_ML_GAUSS) / math.sqrt(k)
    return cols, sgn, X2T


def multilevel_x1(n: int, l1: int, gamma1: int, cols: np.ndarray, sgn: np.ndarray):
    """X1 (l1 x n) as a scipy sparse matrix."""
    import scipy.sparse as sp
    rows = cols.ravel()
    colidx = np.repeat(np.arange(n), gamma1)
    return sp.csr_matrix((sgn.ravel() / math.sqrt(gamma1), (rows, colidx)), shape=(l1, n))


def multilevel_omega(n: int, k: int, seed: int, l1: int = 0, gamma1: int = 0) -> np.ndarray:
    """Omega = X^T = X1^T X2^T (n x k) of the multi-level embedding
    (Sec. 2 eq:multilevelose); l1 = gamma1 = 0 take multilevel_defaults."""
    if l1 <= 0 or gamma1 <= 0:
        l1, gamma1 = multilevel_defaults(n, k)
    cols, sgn, X2T = multilevel_parts(n, k, l1, gamma1, seed)
    X1 = multilevel_x1(n, l1, gamma1, cols, sgn)
    return np.asarray(X1.T @ X2T)
