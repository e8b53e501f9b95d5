"""Structure constants f_mns, d_mns by brute force (test infrastructure only).

Eq. 5: f_mns = -i Tr(F_s [F_m, F_n]), d_mns = Tr(F_s {F_m, F_n}), m, n, s >= 1.
Evaluated on the dense generators of ``basis.py`` -- O(N^6), for N up to ~12.
"""
import numpy as np

from . import basis as _b


def structure_constants(N, B=None):
    """Return dense real tensors (f, d) of shape (M, M, M), M = N^2-1 (Eq. 5)."""
    if B is None:
        B = _b.basis(N)
    M = B.shape[0]
    # products P[m, n] = F_m F_n, all pairs at once
    P = np.einsum("mij,njk->mnik", B, B)
    comm = P - P.transpose(1, 0, 2, 3)
    acomm = P + P.transpose(1, 0, 2, 3)
    # Tr(F_s X) = sum_ij (F_s)_ji X_ij
    f = -1j * np.einsum("sji,mnij->mns", B, comm)
    d = np.einsum("sji,mnij->mns", B, acomm)
    assert np.abs(f.imag).max() < 1e-13 and np.abs(d.imag).max() < 1e-13
    return f.real.copy(), d.real.copy()


def count_nonzero(t, tol=1e-12):
    """Number of entries of a dense tensor with |t| > tol (ordered index triples)."""
    return int((np.abs(t) > tol).sum())
