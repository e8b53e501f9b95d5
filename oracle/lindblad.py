"""The Lindbladian and its matrix in the generator basis, by definition, dense (test infrastructure only).

Eq. 1: L(rho) = -i[H, rho] + sum_p gamma_p ( L_p rho L_p^+ - 1/2 {L_p^+ L_p, rho} ),
which is the paper's D_p(rho) = 1/2([L_p, rho L_p^+] + [L_p rho, L_p^+]) multiplied out.

With rho = 1/N + sum_m v_m F_m (Eq. 6) and Tr(F_s F_m) = delta_sm, the unfolded
system dv/dt = (Q + R) v + K of Eq. 8 has, by definition,
    (Q + R)_sm = Tr(F_s L(F_m)),      K_s = Tr(F_s L(1/N)).
This module evaluates exactly that on dense matrices (N <= ~20).
"""
import numpy as np

from . import basis as _b


def lindbladian(rho, H, Ls=(), gammas=()):
    """L(rho) of Eq. 1 for dense H, dissipators Ls and rates gammas."""
    out = -1j * (H @ rho - rho @ H)
    for L, g in zip(Ls, gammas):
        Ld = L.conj().T
        LdL = Ld @ L
        out = out + g * (L @ rho @ Ld - 0.5 * (LdL @ rho + rho @ LdL))
    return out


def unfold_dense(H, Ls=(), gammas=(), B=None, return_imag=False):
    """Brute force (Q+R, K): Q_sm = Tr(F_s L(F_m)), K_s = Tr(F_s L(1/N)) (Eq. 1, 6, 8).

    Returns real arrays; with ``return_imag`` also the largest imaginary part seen,
    which must vanish because L maps Hermitian matrices to Hermitian matrices.
    """
    H = np.asarray(H, dtype=np.complex128)
    N = H.shape[0]
    if B is None:
        B = _b.basis(N)
    LB = np.stack([lindbladian(F, H, Ls, gammas) for F in B])
    Q = np.einsum("sij,mji->sm", B, LB)
    K = np.einsum("sij,ji->s", B, lindbladian(np.eye(N, dtype=np.complex128) / N, H, Ls, gammas))
    im = max(np.abs(Q.imag).max(), np.abs(K.imag).max())
    if return_imag:
        return Q.real.copy(), K.real.copy(), im
    return Q.real.copy(), K.real.copy()


def lindbladian_kossakowski(rho, H, A, B):
    """Eq. 8 form: -i[H, rho] + sum_jk a_jk (F_j rho F_k^+ - 1/2 {F_k^+ F_j, rho}) for a
    Kossakowski matrix A over the generators B (the paper's 1/2([F_j, rho F_k^+] + [F_j rho, F_k^+])
    multiplied out), without decomposing A."""
    out = -1j * (H @ rho - rho @ H)
    M = A.shape[0]
    for j in range(M):
        for k in range(M):
            a = A[j, k]
            if a == 0:
                continue
            Fj, Fk = B[j], B[k].conj().T
            out = out + a * (Fj @ rho @ Fk - 0.5 * (Fk @ Fj @ rho + rho @ Fk @ Fj))
    return out


def unfold_dense_kossakowski(H, A, B=None):
    """(Q + R, K) of the Eq. 8 Lindbladian by Q_sm = Tr(F_s L(F_m)), K_s = Tr(F_s L(1/N))."""
    H = np.asarray(H, dtype=np.complex128)
    N = H.shape[0]
    if B is None:
        B = _b.basis(N)
    LB = np.stack([lindbladian_kossakowski(F, H, A, B) for F in B])
    Q = np.einsum("sij,mji->sm", B, LB)
    K = np.einsum("sij,ji->s", B, lindbladian_kossakowski(np.eye(N, dtype=np.complex128) / N, H, A, B))
    return Q.real.copy(), K.real.copy()


def liouvillian_vec(H, Ls=(), gammas=()):
    """N^2 x N^2 matrix of L acting on vec(rho) (column stacking), from Eq. 1.

    Uses vec(A X B) = (B^T kron A) vec(X); independent of the generator basis.
    """
    H = np.asarray(H, dtype=np.complex128)
    N = H.shape[0]
    I = np.eye(N, dtype=np.complex128)
    S = -1j * (np.kron(I, H) - np.kron(H.T, I))
    for L, g in zip(Ls, gammas):
        L = np.asarray(L, dtype=np.complex128)
        LdL = L.conj().T @ L
        S = S + g * (np.kron(L.conj(), L) - 0.5 * np.kron(I, LdL) - 0.5 * np.kron(LdL.T, I))
    return S


def vec(X):
    return np.asarray(X).reshape(-1, order="F")


def unvec(x, N):
    return np.asarray(x).reshape(N, N, order="F")


def entry_vectors(N):
    """T (scipy CSC, D x N^2) with T[j, x N + y] = (F_j)_xy for every generator j.  Column (x, y)
    is Tr(F_j E_yx), the coefficients of the matrix unit E_yx by the basis expansion."""
    import scipy.sparse as sp
    cols = []
    for x in range(N):
        for y in range(N):
            E = sp.csr_matrix(([1.0 + 0j], ([y], [x])), shape=(N, N))
            cols.append(sp.csc_matrix(_b.expand_sparse(E).reshape(-1, 1)))
    T = sp.hstack(cols).tocsc()
    T.eliminate_zeros()
    return T


def kossakowski_columns(A, N, cols, T=None):
    """Columns m in ``cols`` of R_sm = Re Tr(F_s D(F_m)) and K_s = Re Tr(F_s D(1/N)) for the Eq. 8
    dissipator D(X) = sum_jk a_jk (F_j X F_k - 1/2 {F_k F_j, X}) of a D x D matrix A, at any N and
    without decomposing A.  Every entry of the N x N matrices involved is a bilinear form in A of
    the generator entries t_xy[j] = (F_j)_xy (the columns of ``entry_vectors``):
        (sum_jk a_jk F_j E_cd F_k)_ab = t_ac^T A t_db =: P[a, c, d, b],
        G  = sum_jk a_jk F_k F_j,   G_xy  = sum_z P[z, y, x, z],
        G' = sum_jk a_jk F_j F_k,   G'_xy = sum_z P[x, z, z, y],
    all of them the entries of T^T A T (two library products with the sparse T).  Then
    D(F_m) = sum_cd (F_m)_cd P[:, c, d, :] - 1/2 (G F_m + F_m G) and D(1/N) = (G' - G)/N, each read
    off with ``basis.expand_dense``.  Returns (R[:, cols] as a D x len(cols) array, K)."""
    A = np.asarray(A, dtype=np.complex128)
    if T is None:
        T = entry_vectors(N)
    labs = _b.labels(N)
    AT = np.asarray(T.T @ np.ascontiguousarray(A.T)).T      # A T, D x N^2
    P = np.asarray(T.T @ AT).reshape(N, N, N, N)             # P[a, c, d, b] = t_ac^T A t_db
    del AT
    G = np.einsum("zyxz->xy", P)
    Gp = np.einsum("xzzy->xy", P)
    R = np.zeros((len(labs), len(cols)))
    for i, m in enumerate(cols):
        Fm = _b.generator(N, labs[m])
        Y = -0.5 * (G @ Fm + Fm @ G)
        for c, d in zip(*np.nonzero(Fm)):
            Y = Y + Fm[c, d] * P[:, c, d, :]
        R[:, i] = _b.expand_dense(Y).real
    K = _b.expand_dense((Gp - G) / N).real
    return R, K
