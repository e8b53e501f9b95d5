"""Seeded synthetic inputs: the driven, dissipatively coupled Bose dimer and random test operators.

This module only builds input operators (Hamiltonian parts, jump operator,
initial state, observable) and seeded parameter draws. It contains none of the
method's arithmetic (no generator basis, no expansion, no structure constants),
so both the CUDA path's tests and the CPU oracle may use it.

Model (Sec. III, Eq. 12 and Eq. 13), N Fock states of M = N - 1 bosons, basis
|n, M - n>, n = 0..N-1 (index n = 0 is |0, M>):
    H(t) = J * HJ + U * HU + eps(t) * H1,  eps(t) = E + A sin(omega t),
    HJ = -(b1^+ b2 + b1 b2^+),  HU = 1/2 sum_i n_i (n_i - 1),  H1 = n1 - n2,
    L  = (b1^+ + b2^+)(b1 - b2),  rate gamma / M.
This is the normalisation of the benchmark workloads; the paper's own Eq. 12
(+J hopping, 2U/(N-1) interaction, eps (n2 - n1)) is ``paper_variant=True``.
"""
from dataclasses import dataclass

import numpy as np


@dataclass
class CSR:
    """Complex N x N matrix in CSR form with separate real and imaginary arrays."""
    n: int
    rowptr: np.ndarray  # int32, n+1
    col: np.ndarray     # int32, nnz
    re: np.ndarray      # float64, nnz
    im: np.ndarray      # float64, nnz

    @property
    def nnz(self):
        return int(self.rowptr[-1])

    def to_dense(self):
        out = np.zeros((self.n, self.n), dtype=np.complex128)
        for r in range(self.n):
            for e in range(self.rowptr[r], self.rowptr[r + 1]):
                out[r, self.col[e]] += self.re[e] + 1j * self.im[e]
        return out

    @staticmethod
    def from_entries(n, entries):
        """entries: dict {(row, col): complex}; zero values are dropped."""
        rows = [[] for _ in range(n)]
        for (r, c), v in entries.items():
            if v != 0:
                rows[r].append((c, complex(v)))
        rowptr = np.zeros(n + 1, dtype=np.int32)
        cols, re, im = [], [], []
        for r in range(n):
            for c, v in sorted(rows[r]):
                cols.append(c)
                re.append(v.real)
                im.append(v.imag)
            rowptr[r + 1] = len(cols)
        return CSR(n, rowptr, np.array(cols, dtype=np.int32), np.array(re, dtype=np.float64),
                   np.array(im, dtype=np.float64))

    @staticmethod
    def from_dense(X, tol=0.0):
        X = np.asarray(X)
        n = X.shape[0]
        ent = {(r, c): X[r, c] for r in range(n) for c in range(n) if abs(X[r, c]) > tol}
        return CSR.from_entries(n, ent)

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.re + 1j * self.im, self.col, self.rowptr), shape=(self.n, self.n))


# parameters of the driven dimer workloads (rate gamma / M on the jump operator)
DIMER_PARAMS = dict(J=1.0, U=0.5, E=1.0, A=1.5, omega=1.0, gamma=0.1)


def _hop(n, M):
    """<n+1, M-n-1| b1^+ b2 |n, M-n> = sqrt((n+1)(M-n))."""
    return np.sqrt((n + 1.0) * (M - n))


@dataclass
class Dimer:
    N: int
    HJ: CSR
    HU: CSR
    H1: CSR
    L: CSR
    params: dict
    rate: float          # gamma / M, the rate in front of the dissipator
    rho0_index: int      # rho0 = |k><k| with k = rho0_index
    obs_diag: np.ndarray  # diagonal of n1 - n2

    def rho0_dense(self):
        r = np.zeros((self.N, self.N), dtype=np.complex128)
        r[self.rho0_index, self.rho0_index] = 1.0
        return r


def dimer(N, params=None, paper_variant=False):
    """Operators of the driven Bose dimer with N Fock states (M = N - 1 bosons)."""
    p = dict(DIMER_PARAMS)
    if params:
        p.update(params)
    M = N - 1
    hj, hu, h1, lo = {}, {}, {}, {}
    sgn_j = 1.0 if paper_variant else -1.0
    for n in range(N):
        n1, n2 = n, M - n
        if paper_variant:
            hu[(n, n)] = 2.0 / (N - 1) * (n1 * (n1 - 1) + n2 * (n2 - 1)) if N > 1 else 0.0
            h1[(n, n)] = float(n2 - n1)
        else:
            hu[(n, n)] = 0.5 * (n1 * (n1 - 1) + n2 * (n2 - 1))
            h1[(n, n)] = float(n1 - n2)
        lo[(n, n)] = float(n1 - n2)  # b1^+ b1 - b2^+ b2
        if n + 1 < N:
            t = _hop(n, M)
            hj[(n + 1, n)] = sgn_j * t
            hj[(n, n + 1)] = sgn_j * t
            lo[(n + 1, n)] = -t   # - b1^+ b2
            lo[(n, n + 1)] = t    # + b2^+ b1
    obs = np.array([float(n - (M - n)) for n in range(N)])
    rate = p["gamma"] / M if M > 0 else p["gamma"]
    return Dimer(N, CSR.from_entries(N, hj), CSR.from_entries(N, hu), CSR.from_entries(N, h1),
                 CSR.from_entries(N, lo), p, rate, 0, obs)


# ---------------------------------------------------------------- seeded draws

MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 (Steele, Lea, Flood 2014; Vigna's reference constants), a counter-based stream."""

    def __init__(self, seed):
        self.state = seed & MASK64

    def next_u64(self):
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self):
        """Double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))


def batch_instances(n=256, seed=1812, sizes=(50, 100, 200)):
    """Seeded batch of dimer instances: N ~ U{sizes}, A ~ U[0.5, 3], gamma = 10^U[-2, 0]."""
    g = SplitMix64(seed)
    out = []
    for _ in range(n):
        N = sizes[min(int(g.uniform() * len(sizes)), len(sizes) - 1)]
        A = 0.5 + 2.5 * g.uniform()
        gamma = 10.0 ** (-2.0 + 2.0 * g.uniform())
        out.append(dict(N=N, A=A, gamma=gamma))
    return out


def random_operator(N, density, seed, hermitian=False, traceless=False):
    """Seeded sparse complex N x N operator (roughly density * N^2 entries)."""
    rng = np.random.default_rng(seed)
    X = np.zeros((N, N), dtype=np.complex128)
    mask = rng.random((N, N)) < density
    X[mask] = rng.normal(size=mask.sum()) + 1j * rng.normal(size=mask.sum())
    if hermitian:
        X = X + X.conj().T
    if traceless:
        X = X - np.trace(X) / N * np.eye(N)
    return CSR.from_dense(X)


def random_banded(N, half_bandwidth, seed, hermitian=False, real=False):
    """Seeded dense-band N x N operator: every entry with |col - row| <= half_bandwidth drawn
    normal (complex unless ``real``); Hermitian by X + X^+ when asked."""
    rng = np.random.default_rng(seed)
    X = np.zeros((N, N), dtype=np.complex128)
    rows, cols = np.nonzero(np.abs(np.subtract.outer(np.arange(N), np.arange(N))) <= half_bandwidth)
    X[rows, cols] = rng.normal(size=rows.size)
    if not real:
        X[rows, cols] += 1j * rng.normal(size=rows.size)
    if hermitian:
        X = X + X.conj().T
    return CSR.from_dense(X)


def random_density_matrix(N, rank, seed):
    """Seeded dense density matrix rho = X X^+ / Tr(X X^+), X an N x rank complex Gaussian draw.

    Every entry of rho is nonzero (almost surely), so every row of the unfolded system sees a
    nonzero input; Hermitian, unit trace, positive semidefinite of the given rank.
    Returns (re, im) as two dense float64 arrays."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((N, rank)) + 1j * rng.standard_normal((N, rank))
    rho = X @ X.conj().T
    rho /= np.trace(rho).real
    rho = 0.5 * (rho + rho.conj().T)
    return np.ascontiguousarray(rho.real), np.ascontiguousarray(rho.imag)


def random_kossakowski(N, seed, scale=1.0):
    """Seeded full-rank Kossakowski matrix over the N^2 - 1 generators: A = c 1 + H with H a
    Hermitian Gaussian matrix (entries of variance scale^2 / D) and c = 3 scale, three times the
    radius of H's spectrum (about 2 scale), so A is positive definite.  Returns (re, im).  H is
    symmetrised tile by tile (a whole-matrix transpose of D^2 entries is slow)."""
    D = N * N - 1
    rng = np.random.default_rng(seed)
    X = (rng.standard_normal((D, D)) + 1j * rng.standard_normal((D, D))) * (scale / np.sqrt(2 * D))
    H = np.empty((D, D), dtype=np.complex128)
    tb = 512
    for i0 in range(0, D, tb):
        for j0 in range(0, D, tb):
            H[i0:i0 + tb, j0:j0 + tb] = (X[i0:i0 + tb, j0:j0 + tb] + X[j0:j0 + tb, i0:i0 + tb].conj().T) / np.sqrt(2.0)
    del X
    H[np.diag_indices(D)] += 3.0 * scale
    return np.ascontiguousarray(H.real), np.ascontiguousarray(H.imag)
