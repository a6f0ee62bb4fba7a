"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module builds problem *data* only: operators A, right-hand sides b and
kernel points.  It holds none of the RandRAND arithmetic (no sketch, no
orthogonalisation, no preconditioner, no Krylov step); the random test
matrices the method itself draws come from the counter-based generator that
each side implements on its own.

Every generator takes an integer seed and draws from ``numpy.random.Generator``
(PCG64) streams ``default_rng([seed, stream])`` so that each array is
reproducible on any host:

    stream 0 -- operator fixtures (Haar factor, mixture points, diffusion field)
    stream 1 -- right-hand sides b

The workloads mirror the paper's problem classes:

* dense PSD ``A = U diag(lam) U^T`` with a prescribed spectrum (the synthetic
  spectra of Sec. 7.1, here with the fully specified decay ``lam_i = i^-2``);
* Gaussian-kernel ridge systems ``(K + mu I) x = b``, ``K_ij =
  exp(-|x_i - x_j|^2 / (2 h^2))`` (the kernel ridge regression systems of
  Sec. 7.2.2, eq:kernel), with points from a Gaussian mixture standing in for
  the paper's datasets, which are not available offline;
* a sparse SPD 5-point variable-coefficient diffusion operator in CSR form
  (a sparse operator class with moderate spectral decay, the regime the
  basis-less variants of Sec. 4.2 target).
"""
from __future__ import annotations

import dataclasses

import numpy as np

STREAM_OPERATOR = 0
STREAM_RHS = 1


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.default_rng([int(seed) & 0xFFFFFFFFFFFFFFFF, int(stream)])


# --------------------------------------------------------------------------
# Dense PSD matrix with a prescribed spectrum
# --------------------------------------------------------------------------
@dataclasses.dataclass
class DenseProblem:
    A: np.ndarray          # n x n float64, symmetric, row-major (C order)
    U: np.ndarray          # n x n Haar-orthogonal factor
    lam: np.ndarray        # eigenvalues of A in decreasing order


def haar_orthogonal(n: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed orthogonal matrix: QR of an N(0,1) matrix with the
    column signs fixed so that diag(R) > 0 (Mezzadri 2007)."""
    g = rng.standard_normal((n, n))
    q, r = np.linalg.qr(g)
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return q * s


def dense_power_spectrum(n: int = 2000, seed: int = 0x52521,
                         power: float = 2.0) -> DenseProblem:
    """A = U diag(i^-power) U^T, i = 1..n, U Haar from the seed."""
    U = haar_orthogonal(n, _rng(seed, STREAM_OPERATOR))
    lam = np.arange(1, n + 1, dtype=np.float64) ** (-power)
    A = (U * lam) @ U.T
    A = 0.5 * (A + A.T)
    return DenseProblem(A=np.ascontiguousarray(A), U=U, lam=lam)


# --------------------------------------------------------------------------
# Gaussian mixture points for the kernel operator
# --------------------------------------------------------------------------
def mixture_points(n: int = 20000, d: int = 8, components: int = 10,
                   seed: int = 0x52522, mean_std: float = 2.0) -> np.ndarray:
    """n points in R^d from an equal-weight Gaussian mixture.

    Component means ~ N(0, mean_std^2 I); each point = its component's mean +
    N(0, I).  Returned as float32: the kernel operator is defined by these
    exact float32 coordinates on both sides of every comparison.
    """
    rng = _rng(seed, STREAM_OPERATOR)
    means = mean_std * rng.standard_normal((components, d))
    labels = rng.integers(0, components, size=n)
    pts = means[labels] + rng.standard_normal((n, d))
    return np.ascontiguousarray(pts.astype(np.float32))


# --------------------------------------------------------------------------
# Variable-coefficient diffusion on a square grid, CSR
# --------------------------------------------------------------------------
@dataclasses.dataclass
class CsrMatrix:
    n: int
    rowptr: np.ndarray     # int32, n+1
    colidx: np.ndarray     # int32, nnz (sorted within each row)
    vals: np.ndarray       # float32 or float64, nnz

    @property
    def nnz(self) -> int:
        return int(self.colidx.shape[0])

    def to_dense(self) -> np.ndarray:
        D = np.zeros((self.n, self.n), dtype=np.float64)
        for i in range(self.n):
            lo, hi = self.rowptr[i], self.rowptr[i + 1]
            D[i, self.colidx[lo:hi]] = self.vals[lo:hi]
        return D


def lognormal_field(side: int, corr_len: float, sigma: float,
                    rng: np.random.Generator) -> np.ndarray:
    """kappa = exp(sigma * g) on a side x side grid.

    g: white noise on a (2 side)^2 periodic grid filtered in Fourier space by
    the square root of the spectral density of the Gaussian covariance
    exp(-r^2 / (2 corr_len^2)), cropped to side x side and normalised to
    zero mean and unit variance.
    """
    big = 2 * side
    w = rng.standard_normal((big, big))
    f = np.fft.fftfreq(big)
    f2 = f[:, None] ** 2 + f[None, :] ** 2
    amp = np.exp(-(np.pi ** 2) * corr_len ** 2 * f2)
    g = np.real(np.fft.ifft2(np.fft.fft2(w) * amp))[:side, :side]
    g = (g - g.mean()) / g.std()
    return np.exp(sigma * g)


def diffusion_csr(side: int = 512, seed: int = 0x52523, corr_len: float = 16.0,
                  sigma: float = 1.0, dtype=np.float32) -> CsrMatrix:
    """5-point finite-volume diffusion -div(kappa grad u) on a side^2 grid, h=1.

    Edge coefficient = harmonic mean of the two cells' kappa.  Homogeneous
    Dirichlet boundary: each missing neighbour adds the cell's own kappa to
    the diagonal.  Rows in lexicographic order (row = iy * side + ix),
    columns sorted; nnz = 5 n - 4 side.
    """
    kap = lognormal_field(side, corr_len, sigma, _rng(seed, STREAM_OPERATOR))
    n = side * side
    rows, cols, vals = [], [], []
    idx = np.arange(n).reshape(side, side)

    def hmean(a, b):
        return 2.0 * a * b / (a + b)

    diag = np.zeros((side, side))
    # x-direction edges
    cx = hmean(kap[:, :-1], kap[:, 1:])
    diag[:, :-1] += cx
    diag[:, 1:] += cx
    rows.append(idx[:, :-1].ravel()); cols.append(idx[:, 1:].ravel()); vals.append(-cx.ravel())
    rows.append(idx[:, 1:].ravel()); cols.append(idx[:, :-1].ravel()); vals.append(-cx.ravel())
    # y-direction edges
    cy = hmean(kap[:-1, :], kap[1:, :])
    diag[:-1, :] += cy
    diag[1:, :] += cy
    rows.append(idx[:-1, :].ravel()); cols.append(idx[1:, :].ravel()); vals.append(-cy.ravel())
    rows.append(idx[1:, :].ravel()); cols.append(idx[:-1, :].ravel()); vals.append(-cy.ravel())
    # Dirichlet boundary contributions
    diag[0, :] += kap[0, :]
    diag[-1, :] += kap[-1, :]
    diag[:, 0] += kap[:, 0]
    diag[:, -1] += kap[:, -1]
    rows.append(idx.ravel()); cols.append(idx.ravel()); vals.append(diag.ravel())

    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals)
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    rowptr = np.cumsum(rowptr)
    return CsrMatrix(n=n, rowptr=rowptr.astype(np.int32),
                     colidx=c.astype(np.int32), vals=v.astype(dtype))


# --------------------------------------------------------------------------
# Right-hand sides
# --------------------------------------------------------------------------
def gaussian_rhs(n: int, nrhs: int, seed: int) -> np.ndarray:
    """b ~ N(0, I), n x nrhs float64, column-major (Fortran order) so that
    column j is contiguous, matching the library's layout."""
    b = _rng(seed, STREAM_RHS).standard_normal((nrhs, n))
    return np.asfortranarray(b.T)


# --------------------------------------------------------------------------
# Named workloads (the sizes of the benchmark configurations)
# --------------------------------------------------------------------------
SEED_DENSE = 0x52521
SEED_KERNEL = 0x52522
SEED_CSR = 0x52523
SEED_BATCH = 0x52524
SEED_SERVE = 0x52525
