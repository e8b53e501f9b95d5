"""The paper's contraction formulas, written out on dense f/d tensors (test infrastructure only).

Sec. II: H = sum_m h_m F_m, L_p = sum_j l_pj F_j (traceless parts);
Eq. 7:  q_sn = sum_m f_mns h_m;
Eq. 10: r_sm = c * sum_p gamma_p sum_{j,k,l} l_pj conj(l_pk) (z_jlm f_kls + conj(z_klm) f_jls),
        printed with c = -1/2;
Eq. 11: k_s = (i/N) sum_p sum_{j,k} l_pj conj(l_pk) f_jks, printed without gamma_p;
z = f + i d (Sec. IV step 2.2 writes "Z = F + D"; z must carry the factor i for
Eq. 10 to reproduce the definition).

Readings (each pinned by a test against Tr(F_s L(F_m))):
* the prefactor of Eq. 10 is c = -1/4 for the two-term form printed; -1/2 is off by 2;
* Eq. 11 carries the rate gamma_p like Eq. 10;
* the sums start at j = 1, so a dissipator with Tr L_p != 0 loses its trace part
  l0 = Tr(L_p)/N; it re-enters as the Hamiltonian
  H_eff = (i gamma_p / 2)(conj(l0) L_p' - l0 L_p'^+), L_p' = L_p - l0, whose
  coefficients are h_eff_j = -gamma_p Im(conj(l0) l_pj).
"""
import numpy as np

from . import basis as _b


def coefficients(X, B=None):
    """Expansion coefficients Tr(F_j X), j >= 1, and the trace part Tr(X)/N (Sec. IV step 2.1)."""
    return _b.expand(np.asarray(X, dtype=np.complex128), B), np.trace(X) / X.shape[0]


def q_matrix(f, h):
    """Eq. 7: q_sn = sum_m f_mns h_m."""
    return np.einsum("mns,m->sn", f, h)


def r_matrix(f, d, l, gamma, prefactor=-0.25):
    """Eq. 10 for one dissipator (P = 1 term), with an explicit prefactor (reading: -1/4)."""
    z = f + 1j * d
    lc = np.conj(l)
    t1 = np.einsum("j,k,jlm,kls->sm", l, lc, z, f, optimize=True)
    t2 = np.einsum("j,k,klm,jls->sm", l, lc, np.conj(z), f, optimize=True)
    return prefactor * gamma * (t1 + t2)


def k_vector(f, l, gamma, N):
    """Eq. 11 for one dissipator, with the rate gamma (reading)."""
    return (1j / N) * gamma * np.einsum("j,k,jks->s", l, np.conj(l), f)


def h_eff_coefficients(l, l0, gamma):
    """Coefficients of the trace-part Hamiltonian H_eff (reading for Tr L != 0)."""
    return -gamma * np.imag(np.conj(l0) * l)


def unfold_paper(f, d, H, Ls=(), gammas=(), B=None, prefactor=-0.25, fold_trace=True):
    """(Q + R, K) from Eq. 7, 10, 11 on dense tensors, with the readings above.

    Returns complex arrays so that a test can check the imaginary parts vanish.
    """
    H = np.asarray(H, dtype=np.complex128)
    N = H.shape[0]
    if B is None:
        B = _b.basis(N)
    h, _ = coefficients(H, B)
    Q = q_matrix(f, h)
    K = np.zeros(Q.shape[0], dtype=np.complex128)
    for L, g in zip(Ls, gammas):
        l, l0 = coefficients(L, B)
        Q = Q + r_matrix(f, d, l, g, prefactor)
        K = K + k_vector(f, l, g, N)
        if fold_trace and l0 != 0:
            Q = Q + q_matrix(f, h_eff_coefficients(l, l0, g))
    return Q, K
