"""The orthonormal SU(N) generator basis, dense, for the oracle (test infrastructure only).

Sec. II (the bulleted list of symmetric, antisymmetric and diagonal generators)
defines the basis; Eq. 6 expands rho over it. Readings taken where the paper is
silent or garbled:

* ordering (the paper fixes none): index s in [0, P2) is S^(j,k), j<k in
  lexicographic order, with P2 = N(N-1)/2; s in [P2, 2 P2) is J^(j,k) in the same
  pair order; s in [2 P2, N^2-1) is D^l, l = 1..N-1. All indices 0-based.
* D^l carries a factor i in the paper's list, which would make it
  anti-Hermitian; the basis must be Hermitian and trace-orthonormal
  (Tr(F_i F_k) = delta_ik, stated right after the list), so D^l is taken real:
  D^l = (sum_{k<l} G_kk - l G_ll) / sqrt(l (l+1)) with 0-based k, l.
* F_0 = identity is not trace-normalised (Tr(1 1) = N); orthonormality holds for
  the N^2-1 traceless elements, F_0 enters only through rho = 1/N + sum v F.
"""
import numpy as np


def n_pairs(N):
    """P2 = N(N-1)/2, the number of S (and of J) generators (Sec. II list)."""
    return N * (N - 1) // 2


def bloch_dim(N):
    """M = N^2 - 1, the number of traceless generators (Sec. II)."""
    return N * N - 1


def pair_index(N, j, k):
    """Position of the pair (j, k), j < k, in lexicographic order (ordering reading)."""
    assert 0 <= j < k < N
    return j * N - j * (j + 1) // 2 + (k - j - 1)


def labels(N):
    """List of (kind, a, b) for every basis index s: ('S', j, k), ('J', j, k), ('D', l, -1)."""
    out = []
    pairs = [(j, k) for j in range(N) for k in range(j + 1, N)]
    out += [("S", j, k) for (j, k) in pairs]
    out += [("J", j, k) for (j, k) in pairs]
    out += [("D", l, -1) for l in range(1, N)]
    return out


def generator(N, label):
    """Dense N x N matrix of one generator (Sec. II list, with the D^l reading)."""
    kind, a, b = label
    F = np.zeros((N, N), dtype=np.complex128)
    if kind == "S":
        F[a, b] = 1.0 / np.sqrt(2.0)
        F[b, a] = 1.0 / np.sqrt(2.0)
    elif kind == "J":
        F[a, b] = -1j / np.sqrt(2.0)
        F[b, a] = 1j / np.sqrt(2.0)
    else:
        l = a
        c = 1.0 / np.sqrt(l * (l + 1.0))
        for k in range(l):
            F[k, k] = c
        F[l, l] = -l * c
    return F


def basis(N):
    """All traceless generators stacked as an array of shape (N^2-1, N, N)."""
    return np.stack([generator(N, lab) for lab in labels(N)])


def expand(X, B=None):
    """Coefficients x_s = Tr(F_s X) of an N x N matrix X (Sec. IV step 2.1, by definition).

    For Hermitian X the coefficients are real; for any X, X = Tr(X)/N + sum_s x_s F_s.
    """
    N = X.shape[0]
    if B is None:
        B = basis(N)
    return np.einsum("sij,ji->s", B, X)


def rho_from_v(v, B=None, N=None):
    """rho = F_0/N + sum_j v_j F_j (Eq. 6)."""
    if B is None:
        B = basis(N)
    N = B.shape[1]
    return np.eye(N, dtype=np.complex128) / N + np.einsum("s,sij->ij", np.asarray(v, dtype=np.complex128), B)


def expand_sparse(X):
    """Tr(F_s X) for a scipy.sparse N x N matrix X, s = 0..N^2-2, written out per generator.

    S^(j,k): (X_jk + X_kj)/sqrt2; J^(j,k): i (X_jk - X_kj)/sqrt2; D^l: c_l (sum_{k<l} X_kk - l X_ll).
    These are Tr(F X) for the matrices of the Sec. II list, evaluated entry by entry.
    """
    import scipy.sparse as sp
    X = sp.csr_matrix(X)
    N = X.shape[0]
    P2 = n_pairs(N)
    out = np.zeros(bloch_dim(N), dtype=np.complex128)
    Xc = X.tocoo()
    for i, j, x in zip(Xc.row, Xc.col, Xc.data):
        if i == j:
            continue
        a, b = (i, j) if i < j else (j, i)
        p = pair_index(N, a, b)
        out[p] += x / np.sqrt(2.0)
        out[P2 + p] += (1j if i < j else -1j) * x / np.sqrt(2.0)
    d = np.asarray(X.diagonal(), dtype=np.complex128)
    for l in range(1, N):
        c = 1.0 / np.sqrt(l * (l + 1.0))
        out[2 * P2 + l - 1] = c * (d[:l].sum() - l * d[l])
    return out


def expand_dense(X):
    """Tr(F_s X) for a dense N x N array X, the entry formulas of ``expand_sparse`` on whole arrays.

    S^(j,k): (X_jk + X_kj)/sqrt2 and J^(j,k): i (X_jk - X_kj)/sqrt2 over the pairs j < k in
    lexicographic order (numpy's upper-triangle order is row-major, the same order);
    D^l: c_l (sum_{k<l} X_kk - l X_ll) from a running sum of the diagonal.
    """
    X = np.asarray(X, dtype=np.complex128)
    N = X.shape[0]
    j, k = np.triu_indices(N, 1)
    up, lo = X[j, k], X[k, j]
    d = np.diag(X)
    l = np.arange(1, N)
    below = np.cumsum(d)[:-1]                      # sum_{k<l} X_kk for l = 1..N-1
    dpart = (below - l * d[1:]) / np.sqrt(l * (l + 1.0))
    return np.concatenate([(up + lo) / np.sqrt(2.0), 1j * (up - lo) / np.sqrt(2.0), dpart])


def populations_from_v(v, N):
    """diag rho of Eq. 6: rho_jj = 1/N + sum_l v_{D^l} (D^l)_jj, with (D^l)_jj = c_l for j < l,
    -l c_l for j = l and 0 above (only the D generators have diagonal entries)."""
    vd = np.asarray(v, dtype=float)[2 * n_pairs(N):]
    pop = np.full(N, 1.0 / N)
    for l in range(1, N):
        c = 1.0 / np.sqrt(l * (l + 1.0))
        pop[:l] += vd[l - 1] * c
        pop[l] -= vd[l - 1] * l * c
    return pop
