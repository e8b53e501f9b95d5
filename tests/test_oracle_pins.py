"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test names what fixes the expected value: a textbook result, a closed form,
the nonzero counts printed in Sec. IV step 2.2, an invariant, or an independent
route (the dense density-matrix Liouvillian, the matrix exponential, complex-step
differentiation).
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import basis as B
from oracle import lindblad as Lb
from oracle import native
from oracle import paper_formulas as PF
from oracle import propagate as P
from oracle import structure as S
from oracle import system as SYS
from paper_1812_11626_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------- basis

@pytest.mark.parametrize("N", [2, 3, 4, 6])
def test_basis_hermitian_traceless_orthonormal(N):
    """Sec. II: traceless Hermitian generators with Tr(F_i F_k) = delta_ik."""
    F = B.basis(N)
    assert F.shape == (N * N - 1, N, N)
    assert np.abs(F - F.conj().transpose(0, 2, 1)).max() == 0.0
    assert np.abs(np.einsum("sii->s", F)).max() < 1e-15
    G = np.einsum("sij,tji->st", F, F)
    assert np.abs(G - np.eye(N * N - 1)).max() < 1e-15


def test_pair_index_is_lexicographic():
    N = 7
    pairs = [(j, k) for j in range(N) for k in range(j + 1, N)]
    assert [B.pair_index(N, j, k) for (j, k) in pairs] == list(range(len(pairs)))


@pytest.mark.parametrize("N", [3, 5])
def test_rho_from_v_roundtrip_and_trace(N):
    """Eq. 6: rho = 1/N + sum v F has unit trace, is Hermitian, and v = Tr(F rho)."""
    rng = np.random.default_rng(N)
    v = rng.normal(size=N * N - 1)
    rho = B.rho_from_v(v, N=N)
    assert abs(np.trace(rho) - 1.0) < 1e-15
    assert np.abs(rho - rho.conj().T).max() < 1e-15
    assert np.abs(B.expand(rho).real - v).max() < 1e-14
    assert np.abs(B.expand_sparse(sp.csr_matrix(rho)) - B.expand(rho)).max() < 1e-14


# ------------------------------------------------------ structure constants

def test_su2_pauli():
    """N = 2: F = sigma/sqrt2 in the order (S, J, D) = (x, y, z); f = sqrt2 eps_ijk, d = 0 (textbook)."""
    f, d = S.structure_constants(2)
    eps = np.zeros((3, 3, 3))
    for (i, j, k), s in {(0, 1, 2): 1, (1, 2, 0): 1, (2, 0, 1): 1, (1, 0, 2): -1, (0, 2, 1): -1, (2, 1, 0): -1}.items():
        eps[i, j, k] = s
    assert np.abs(f - np.sqrt(2) * eps).max() < 1e-15
    assert np.abs(d).max() < 1e-15


def _load_gellmann():
    f = np.zeros((8, 8, 8))
    d = np.zeros((8, 8, 8))
    import itertools
    with open(os.path.join(GOLDEN, "gellmann_su3.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            kind, a, b, c, val = line.split()
            idx = (int(a) - 1, int(b) - 1, int(c) - 1)
            for perm in set(itertools.permutations(range(3))):
                p = tuple(idx[i] for i in perm)
                if kind == "f":
                    sign = np.linalg.det(np.eye(3)[list(perm)])
                    f[p] = sign * float(val)
                else:
                    d[p] = float(val)
    return f, d


def test_su3_gellmann_golden():
    """N = 3: F = lambda/sqrt2, so f = sqrt2 f_GM and d = sqrt2 d_GM (Gell-Mann tables, golden file).

    Gell-Mann lambda_1..8 are, in this basis, S01, J01, D1, S02, J02, S12, J12, D2.
    """
    fgm, dgm = _load_gellmann()
    to_ours = [0, 3, 6, 1, 4, 2, 5, 7]
    f, d = S.structure_constants(3)
    perm = np.ix_(to_ours, to_ours, to_ours)
    assert np.abs(f[perm] - np.sqrt(2) * fgm).max() < 1e-14
    assert np.abs(d[perm] - np.sqrt(2) * dgm).max() < 1e-14


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6, 7])
def test_nonzero_counts_match_paper(N):
    """Sec. IV step 2.2 prints NZ_F = 5N^3-9N^2-2N+6 and NZ_D = 6N^3 - N(21N+7)/2 + 1 (ordered triples)."""
    f, d = S.structure_constants(N)
    assert S.count_nonzero(f) == 5 * N**3 - 9 * N**2 - 2 * N + 6
    assert S.count_nonzero(d) == 6 * N**3 - N * (21 * N + 7) // 2 + 1


@pytest.mark.parametrize("N", [3, 4])
def test_f_antisymmetric_d_symmetric_and_complete(N):
    """Sec. II: f totally antisymmetric, d totally symmetric; Eq. 3-4 rebuild [F,F] and {F,F}."""
    F = B.basis(N)
    f, d = S.structure_constants(N, F)
    for perm in [(1, 0, 2), (0, 2, 1), (2, 1, 0)]:
        assert np.abs(f + f.transpose(perm)).max() < 1e-15
        assert np.abs(d - d.transpose(perm)).max() < 1e-15
    M = N * N - 1
    for i in range(M):
        for k in range(M):
            c = F[i] @ F[k] - F[k] @ F[i]
            a = F[i] @ F[k] + F[k] @ F[i]
            assert np.abs(c - 1j * np.einsum("l,lab->ab", f[i, k], F)).max() < 1e-14
            ref = (2.0 / N) * (i == k) * np.eye(N) + np.einsum("l,lab->ab", d[i, k], F)
            assert np.abs(a - ref).max() < 1e-14


# ------------------------------------------------------------- unfolding

def test_qubit_bloch_equations():
    """N = 2, H = (w/2) sigma_z, L = sigma_- = |1><0|, rate g: the textbook Bloch equations.

    With r = sqrt2 v: dr_x/dt = -w r_y - g/2 r_x, dr_y/dt = w r_x - g/2 r_y, dr_z/dt = -g (r_z + 1).
    """
    w, g = 1.3, 0.4
    H = np.diag([w / 2, -w / 2]).astype(complex)
    L = np.array([[0, 0], [1, 0]], dtype=complex)
    Q, K = Lb.unfold_dense(H, [L], [g])
    Qref = np.array([[-g / 2, -w, 0], [w, -g / 2, 0], [0, 0, -g]])
    Kref = np.array([0, 0, -g / np.sqrt(2)])
    assert np.abs(Q - Qref).max() < 1e-15
    assert np.abs(K - Kref).max() < 1e-15
    Gs, Ks, _ = native.unfold(2, sp.csr_matrix(H), sp.csr_matrix(L), g)
    assert np.abs(Gs.toarray() - Qref).max() < 1e-15 and np.abs(Ks - Kref).max() < 1e-15


@pytest.mark.parametrize("N", [2, 3, 4, 5])
def test_paper_formulas_reproduce_definition(N):
    """Eq. 7, 10, 11 with the readings (-1/4 in Eq. 10, gamma in Eq. 11, trace fold-in) equal Tr(F_s L(F_m))."""
    rng = np.random.default_rng(100 + N)
    F = B.basis(N)
    f, d = S.structure_constants(N, F)
    H = rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))
    H = H + H.conj().T
    L = rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))   # not traceless
    g = 0.73
    Q, K = Lb.unfold_dense(H, [L], [g], F)
    Qp, Kp = PF.unfold_paper(f, d, H, [L], [g], F)
    scale = np.abs(Q).max()
    assert np.abs(Qp - Q).max() < 1e-13 * scale
    assert np.abs(Kp - K).max() < 1e-13 * scale
    # the printed prefactor -1/2 does not reproduce the definition
    Qh, _ = PF.unfold_paper(f, d, H, [L], [g], F, prefactor=-0.5)
    assert np.abs(Qh - Q).max() > 1e-3 * scale
    # dropping the trace part of L is wrong when Tr L != 0
    Qn, _ = PF.unfold_paper(f, d, H, [L], [g], F, fold_trace=False)
    assert np.abs(Qn - Q).max() > 1e-6 * scale


def test_kossakowski_form_reduces_to_jump_operators():
    """Eq. 8 with A = sum_p gamma_p l_p l_p^+ (Eq. 9) equals the jump-operator form with
    L_p = sum_j l_pj F_j (Eq. 1), for a rank-2 A."""
    N = 3
    F = B.basis(N)
    rng = np.random.default_rng(12)
    H = rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))
    H = H + H.conj().T
    M = N * N - 1
    ls = [rng.normal(size=M) + 1j * rng.normal(size=M) for _ in range(2)]
    gs = [0.4, 1.3]
    A = sum(g * np.outer(l, l.conj()) for g, l in zip(gs, ls))
    Qa, Ka = Lb.unfold_dense_kossakowski(H, A, F)
    Ls = [np.einsum("j,jab->ab", l, F) for l in ls]
    Ql, Kl = Lb.unfold_dense(H, Ls, gs, F)
    assert np.abs(Qa - Ql).max() < 1e-13 * np.abs(Ql).max()
    assert np.abs(Ka - Kl).max() < 1e-13 * np.abs(Ql).max()


@pytest.mark.parametrize("N", [3, 6])
def test_hamiltonian_part_skew(N):
    """Eq. 7: Q from the Hamiltonian alone is skew-symmetric."""
    H = W.random_operator(N, 0.6, 7 + N, hermitian=True).to_dense()
    Q, K = Lb.unfold_dense(H)
    assert np.abs(Q + Q.T).max() < 1e-14 and np.abs(K).max() == 0.0


@pytest.mark.parametrize("N,dens", [(2, 1.0), (4, 0.5), (7, 0.3), (12, 0.2)])
def test_sparse_c_oracle_matches_dense(N, dens):
    """The sparse C definition route equals the dense brute force (same definition, independent code)."""
    H = W.random_operator(N, dens, 31 + N, hermitian=True)
    A = W.random_operator(N, dens, 41 + N)
    G, K, im = native.unfold(N, H.to_scipy(), A.to_scipy(), 0.29)
    Q, Kd = Lb.unfold_dense(H.to_dense(), [A.to_dense()], [0.29])
    assert np.abs(G.toarray() - Q).max() < 1e-13 * np.abs(Q).max()
    assert np.abs(K - Kd).max() < 1e-13 * np.abs(Q).max()
    assert im < 1e-12 * np.abs(Q).max()
    # column subsets give the same columns
    cols = [0, N * N - 2, (N * N - 1) // 2]
    Gc, _, _ = native.unfold(N, H.to_scipy(), A.to_scipy(), 0.29, cols=cols, want_k=False)
    Gc = Gc.toarray()
    for c in cols:
        assert np.abs(Gc[:, c] - Q[:, c]).max() < 1e-13 * np.abs(Q).max()


def test_dimer_initial_state_and_observable():
    """Model check: rho0 = |0, M><0, M| gives <n1 - n2> = -M and |v|^2 = 1 - 1/N (purity 1)."""
    for N in (2, 10, 57):
        d = W.dimer(N)
        v0 = SYS.initial_v(d)
        w, c0 = P.observable_weights(d.obs_diag)
        assert abs(c0 + w @ v0 - (-(N - 1))) < 1e-12 * N
        assert abs(v0 @ v0 - (1.0 - 1.0 / N)) < 1e-14


def test_dimer_operators():
    """Operators of Sec. III: HJ, L tridiagonal with nnz 3N-2 (Sec. IV step 2.1), L traceless."""
    N = 9
    d = W.dimer(N)
    # the diagonal 2n - M of L vanishes at n = M/2 when M is even
    assert d.HJ.nnz == 2 * (N - 1) and d.L.nnz == 3 * N - 2 - (N % 2)
    assert W.dimer(10).L.nnz == 3 * 10 - 2
    Ld = d.L.to_dense()
    assert abs(np.trace(Ld)) == 0.0
    # L = (b1^+ + b2^+)(b1 - b2) and HJ from ladder operators of the full two-mode Fock
    # space (occupations 0..M per mode), projected on the M-boson states |n, M-n>
    M = N - 1
    a = np.diag(np.sqrt(np.arange(1, M + 1)), 1)          # single-mode annihilator
    I = np.eye(M + 1)
    b1, b2 = np.kron(a, I), np.kron(I, a)
    P = np.zeros(((M + 1) ** 2, N))
    for n in range(N):
        P[n * (M + 1) + (M - n), n] = 1.0
    Lfull = (b1.T + b2.T) @ (b1 - b2)
    assert np.abs(Ld - P.T @ Lfull @ P).max() < 1e-12
    Hj = -(b1.T @ b2 + b1 @ b2.T)
    assert np.abs(d.HJ.to_dense() - P.T @ Hj @ P).max() < 1e-12
    nn1, nn2 = b1.T @ b1, b2.T @ b2
    Hu = 0.5 * (nn1 @ (nn1 - np.eye(len(P))) + nn2 @ (nn2 - np.eye(len(P))))
    assert np.abs(d.HU.to_dense() - P.T @ Hu @ P).max() < 1e-12
    assert np.abs(d.H1.to_dense() - P.T @ (nn1 - nn2) @ P).max() < 1e-12


# ------------------------------------------------------------- propagation

def _small_driven(N=4, seed=5):
    H0 = W.random_operator(N, 0.7, seed, hermitian=True).to_dense()
    H1 = np.diag(np.arange(N, dtype=float)).astype(complex)
    L = W.random_operator(N, 0.7, seed + 1).to_dense()
    return H0, H1, L


def test_rk4_matches_rho_space_rk4():
    """RK4 commutes with v = Tr(F rho): the v-space map equals RK4 on vec(rho) with the dense Liouvillian."""
    N = 4
    H0, H1, L = _small_driven(N)
    g = 0.31
    F = B.basis(N)
    Q0, K = Lb.unfold_dense(H0, [L], [g], F)
    Q1, _ = Lb.unfold_dense(H1, (), (), F)
    rho0 = np.zeros((N, N), complex); rho0[0, 0] = 0.6; rho0[1, 1] = 0.4; rho0[0, 1] = rho0[1, 0] = 0.2
    eps = P.eps_fn(0.4, 0.9, 1.3)
    h, n = 0.01, 300
    v, _ = P.rk4(Q0, Q1, K, eps, B.expand(rho0).real, h, n)
    rho = P.rho_rk4(H0, H1, [L], [g], eps, rho0, h, n)
    assert np.abs(B.rho_from_v(v, F) - rho).max() < 1e-13


def test_rk4_converges_to_expm_fourth_order():
    """Time-independent case: RK4 -> exp(tL) rho0 with global error O(h^4)."""
    N = 3
    H0, _, L = _small_driven(N, seed=9)
    F = B.basis(N)
    Q, K = Lb.unfold_dense(H0, [L], [0.5], F)
    rho0 = np.diag([1.0, 0, 0]).astype(complex)
    t = 2.0
    exact = B.expand(P.rho_expm(H0, [L], [0.5], rho0, t)).real
    errs = []
    for n in (50, 100, 200):
        v, _ = P.rk4(Q, np.zeros_like(Q), K, lambda s: 0.0, B.expand(rho0).real, t / n, n)
        errs.append(np.abs(v - exact).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 13 < r1 < 19 and 13 < r2 < 19, errs


def test_rk4_pair_rotation_closed_form():
    """J = 0 and gamma = 0: each (S_jk, J_jk) pair rotates by the phase int (E_j - E_k) dt (closed form).

    H(t) = diag(e) + eps(t) diag(o); rho_jk(t) = rho_jk(0) exp(-i Phi_jk(t)),
    Phi_jk(t) = (e_j - e_k) t + (o_j - o_k)(E t + A (1 - cos(w t)) / w).
    """
    N = 5
    e = np.array([0.0, 0.7, 1.1, 2.0, 2.2])
    o = np.array([-2.0, -1.0, 0.0, 1.0, 2.0])
    E, A, w = 0.3, 0.8, 1.7
    F = B.basis(N)
    Q0, _ = Lb.unfold_dense(np.diag(e).astype(complex), (), (), F)
    Q1, _ = Lb.unfold_dense(np.diag(o).astype(complex), (), (), F)
    rng = np.random.default_rng(2)
    X = rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))
    rho0 = X @ X.conj().T
    rho0 /= np.trace(rho0)
    t, n = 3.0, 3000
    v, _ = P.rk4(Q0, Q1, np.zeros(N * N - 1), P.eps_fn(E, A, w), B.expand(rho0).real, t / n, n)
    phi = np.subtract.outer(e, e) * t + np.subtract.outer(o, o) * (E * t + A * (1 - np.cos(w * t)) / w)
    exact = rho0 * np.exp(-1j * phi)
    assert np.abs(B.rho_from_v(v, F) - exact).max() < 1e-9


def test_rk4_square_drive_pair_rotation_closed_form():
    """Square drive theta = +-1 (Sec. III, driving (i)), J = 0, gamma = 0: each pair rotates by
    Phi_jk(t) = (e_j - e_k) t + (o_j - o_k) int_0^t eps, with int eps piecewise linear; RK4 with
    the midpoint rule on a grid containing the jumps converges to it at fourth order."""
    N = 4
    e = np.array([0.0, 0.5, 1.3, 1.7])
    o = np.array([-1.5, -0.5, 0.5, 1.5])
    E, A, w = 0.2, 0.9, 1.0
    T = 2 * np.pi / w
    F = B.basis(N)
    Q0, _ = Lb.unfold_dense(np.diag(e).astype(complex), (), (), F)
    Q1, _ = Lb.unfold_dense(np.diag(o).astype(complex), (), (), F)
    rng = np.random.default_rng(8)
    X = rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))
    rho0 = X @ X.conj().T
    rho0 /= np.trace(rho0)
    t = 1.5 * T   # three half-periods: +A, -A, +A
    inteps = E * t + A * (0.5 * T - 0.5 * T + 0.5 * T)
    phi = np.subtract.outer(e, e) * t + np.subtract.outer(o, o) * inteps
    exact = rho0 * np.exp(-1j * phi)
    errs = []
    for spp in (200, 400):
        n = int(round(1.5 * spp))
        v, _ = P.rk4(Q0, Q1, np.zeros(N * N - 1), None, B.expand(rho0).real, T / spp, n,
                     eps_step=P.eps_square_step(E, A, w))
        errs.append(np.abs(B.rho_from_v(v, F) - exact).max())
    assert errs[1] < 1e-6 and 12 < errs[0] / errs[1] < 20, errs


def test_rk4_gamma0_norm_loss_is_fifth_order():
    """gamma = 0: the exact flow is unitary, so |v| is conserved; RK4's amplification on the
    imaginary axis is |R(iy)|^2 = 1 - y^6/72 + y^8/576, so over a fixed time |v| shrinks,
    and the loss falls as h^5 (factor 32 per halving of h)."""
    d = W.dimer(6, dict(gamma=0.0))
    u = SYS.unfold_dimer(d)
    n0 = np.linalg.norm(SYS.initial_v(d))
    loss = []
    for spp in (400, 800, 1600):
        v, _ = SYS.propagate_dimer(d, u, spp, spp)
        loss.append(n0 - np.linalg.norm(v))
    assert all(x > 0 for x in loss)
    assert 28 < loss[0] / loss[1] < 36 and 28 < loss[1] / loss[2] < 36, loss


def test_dimer_rho_positive_trace_one():
    """Eq. 6 reconstruction after 2 periods of the N=8 dimer: Tr rho = 1, eigenvalues >= -1e-8."""
    d = W.dimer(8)
    u = SYS.unfold_dimer(d)
    v, _ = SYS.propagate_dimer(d, u, 200, 400)
    rho = B.rho_from_v(v, N=8)
    assert abs(np.trace(rho) - 1.0) < 1e-14
    assert np.linalg.eigvalsh(rho).min() > -1e-8


# ------------------------------------------------------------- adjoint

def _adjoint_case():
    d = W.dimer(5)
    u = SYS.unfold_dimer(d)
    p = d.params
    return d, u, p


def test_adjoint_matches_complex_step():
    """Discrete adjoint of RK4 equals the complex-step derivative of the same discrete loss (exact to rounding)."""
    d, u, p = _adjoint_case()
    S, period = 40, 2
    h = 2 * np.pi / p["omega"] / S
    w, c0 = P.observable_weights(d.obs_diag)
    v0 = SYS.initial_v(d)
    theta = dict(A=p["A"], rate=d.rate, J=p["J"], U=p["U"])

    def loss(th):
        Q0 = th["J"] * u.QJ + th["U"] * u.QU + th["rate"] * u.R1
        K = th["rate"] * u.K1
        eps = lambda t: p["E"] + th["A"] * np.sin(p["omega"] * t)
        return P.timeavg_loss(Q0, u.Q1, K, eps, v0.astype(complex), w, c0, h, S, period)

    Q0 = u.q0(p["J"], p["U"], d.rate)
    sinw = lambda t: np.sin(p["omega"] * t)
    L, g = P.timeavg_adjoint(Q0, u.Q1, d.rate * u.K1, P.eps_fn(p["E"], p["A"], p["omega"]), v0, w, c0, h, S, period,
                             dQ0=[None, u.R1, u.QJ, u.QU], dQ1=[(u.Q1, sinw), None, None, None],
                             dK=[None, u.K1, None, None])
    assert abs(L - loss(theta).real) < 1e-12
    for i, key in enumerate(["A", "rate", "J", "U"]):
        th = dict(theta)
        th[key] = theta[key] + 1e-30j
        cs = loss(th).imag / 1e-30
        assert abs(g[i] - cs) <= 1e-10 * max(1.0, abs(cs)), (key, g[i], cs)
        # central finite difference agrees to its own truncation error
        hfd = 1e-6
        thp = dict(theta); thp[key] = theta[key] + hfd
        thm = dict(theta); thm[key] = theta[key] - hfd
        fd = (loss(thp).real - loss(thm).real) / (2 * hfd)
        assert abs(fd - cs) <= 1e-6 * max(1.0, abs(cs))


# ------------------------------------------------------------- dense expansion, threaded RK4

@pytest.mark.parametrize("N", [2, 3, 5, 7])
def test_expand_dense_reads_unit_vectors_off_the_generators(N):
    """Orthonormality (Sec. II, Tr(F_i F_k) = delta_ik): the coefficients of generator F_s are the
    unit vector e_s; on random complex matrices the entry formulas equal the trace definition."""
    labs = B.labels(N)
    for s, lab in enumerate(labs):
        x = B.expand_dense(B.generator(N, lab))
        e = np.zeros(len(labs))
        e[s] = 1.0
        assert np.abs(x - e).max() < 1e-15
    rng = np.random.default_rng(N)
    X = rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))
    assert np.abs(B.expand_dense(X) - B.expand(X)).max() < 1e-14


def test_expand_dense_parseval_at_n1000():
    """Eq. 6 with an orthonormal basis: |v|^2 = Tr rho^2 - 1/N for a dense rank-3 state at N = 1000,
    and every coefficient of that state is nonzero."""
    re, im = W.random_density_matrix(1000, 3, 7)
    rho = re + 1j * im
    v = B.expand_dense(rho)
    assert np.abs(v.imag).max() == 0.0
    assert abs(v.real @ v.real - (np.vdot(rho, rho).real - 1e-3)) < 1e-12
    assert np.abs(v.real).min() > 0


def test_c_rk4_pair_rotation_and_fourth_order():
    """The threaded C RK4 (native.rk4) against closed forms, not against the Python RK4: the driven
    pair rotation of a diagonal H (J = 0, gamma = 0) and fourth-order convergence to exp(tL)."""
    N = 5
    e = np.array([0.0, 0.7, 1.1, 2.0, 2.2])
    o = np.array([-2.0, -1.0, 0.0, 1.0, 2.0])
    E, A, w = 0.3, 0.8, 1.7
    F = B.basis(N)
    Q0, _ = Lb.unfold_dense(np.diag(e).astype(complex), (), (), F)
    Q1, _ = Lb.unfold_dense(np.diag(o).astype(complex), (), (), F)
    rng = np.random.default_rng(2)
    X = rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))
    rho0 = X @ X.conj().T
    rho0 /= np.trace(rho0)
    t, n = 3.0, 3000
    v, out = native.rk4(Q0, Q1, None, E, A, w, B.expand(rho0).real, t / n, n, emit_every=1000)
    phi = np.subtract.outer(e, e) * t + np.subtract.outer(o, o) * (E * t + A * (1 - np.cos(w * t)) / w)
    assert np.abs(B.rho_from_v(v, F) - rho0 * np.exp(-1j * phi)).max() < 1e-9
    assert len(out) == 3 and np.array_equal(out[-1], v)
    H0, _, L = _small_driven(3, seed=9)
    F3 = B.basis(3)
    Q, K = Lb.unfold_dense(H0, [L], [0.5], F3)
    r0 = np.diag([1.0, 0, 0]).astype(complex)
    exact = B.expand(P.rho_expm(H0, [L], [0.5], r0, 2.0)).real
    errs = [np.abs(native.rk4(Q, None, K, 0.0, 0.0, 1.0, B.expand(r0).real, 2.0 / n, n)[0] - exact).max()
            for n in (50, 100, 200)]
    assert 13 < errs[0] / errs[1] < 19 and 13 < errs[1] / errs[2] < 19, errs


@pytest.mark.parametrize("drive", ["sin", "square"])
def test_c_rk4_equals_python_rk4_on_the_dimer(drive):
    """Both oracle RK4s run the same map: N = 10 dimer, 3 periods, emitted states at period ends."""
    d = W.dimer(10)
    u = SYS.unfold_dimer(d)
    a, ea = SYS.propagate_dimer(d, u, 200, 600, emit_every=200, drive=drive)
    b, eb = SYS.propagate_dimer(d, u, 200, 600, emit_every=200, drive=drive, threaded=True)
    assert len(ea) == len(eb) == 3
    assert np.abs(a - b).max() < 1e-13 and max(np.abs(x - y).max() for x, y in zip(ea, eb)) < 1e-13


# ------------------------------------------------------------- the loss window (reading O)

def _rk4_factor(z):
    """RK4's stability function: one step of y' = lam y multiplies y by R(h lam)."""
    return 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24


def test_loss_window_and_trapezoid_weights_closed_form():
    """Diagonal H, no drive, no dissipator: rho_jk evolves by rho_jk' = -i (e_j - e_k) rho_jk, so RK4
    multiplies it by r = R(-i (e_j - e_k) h) every step and the S^(j,k) component is
    sqrt2 Re(rho_jk(0) r^n).  The trapezoid mean over the S + 1 grid points of period P,
    n = (P-1) S .. P S, is then a geometric sum in closed form:
        sqrt2 Re( rho_jk(0) r^((P-1) S) [ (1 - r^(S+1)) / (1 - r) - (1 + r^S) / 2 ] / S ).
    A window shifted by one step, uniform weights or a wrong normalisation all miss it."""
    N = 4
    e = np.array([0.0, 0.9, 1.4, 2.35])
    F = B.basis(N)
    Q0, K = Lb.unfold_dense(np.diag(e).astype(complex), (), (), F)
    rng = np.random.default_rng(4)
    X = rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))
    rho0 = X @ X.conj().T
    rho0 /= np.trace(rho0)
    v0 = B.expand(rho0).real
    S, period = 40, 3
    h = 2 * np.pi / S
    zero = np.zeros_like(Q0)
    for (j, k) in ((0, 1), (1, 3)):
        w = np.zeros(N * N - 1)
        w[B.pair_index(N, j, k)] = 1.0
        r = _rk4_factor(-1j * (e[j] - e[k]) * h)
        geo = (1 - r ** (S + 1)) / (1 - r) - 0.5 * (1 + r ** S)
        exact = np.sqrt(2) * (rho0[j, k] * r ** ((period - 1) * S) * geo / S).real
        got = P.timeavg_loss(Q0, zero, K, lambda t: 0.0, v0, w, 0.0, h, S, period)
        assert abs(got - exact) < 1e-13, (j, k, got, exact)
        # the same window through the adjoint's forward sweep
        L, _ = P.timeavg_adjoint(Q0, zero, K, lambda t: 0.0, v0, w, 0.0, h, S, period, [None], [None], [None])
        assert abs(L - exact) < 1e-13
        # a window one step late is measurably different (so the pin can fail)
        late = np.sqrt(2) * (rho0[j, k] * r ** ((period - 1) * S + 1) * geo / S).real
        assert abs(late - exact) > 1e-4


def test_loss_of_a_constant_observable_is_the_constant():
    """O = c 1: <O> = c Tr rho = c at every time, so the period mean is c for any window and state
    (the trapezoid weights sum to one)."""
    d = W.dimer(6)
    u = SYS.unfold_dimer(d)
    p = d.params
    Q0 = u.q0(p["J"], p["U"], d.rate)
    for S, period in ((30, 1), (25, 2)):
        w, c0 = P.observable_weights(np.full(6, 2.5))
        assert np.abs(w).max() < 1e-15 and abs(c0 - 2.5) < 1e-15
        L = P.timeavg_loss(Q0, u.Q1, d.rate * u.K1, P.eps_fn(p["E"], p["A"], p["omega"]), SYS.initial_v(d), w, c0,
                           2 * np.pi / S, S, period)
        assert abs(L - 2.5) < 1e-13


@pytest.mark.parametrize("N", [2, 3, 4])
def test_kossakowski_columns_match_eq8_applied_directly(N):
    """The column-wise Eq. 8 oracle (bilinear forms of generator entries, any N) against Eq. 8
    applied with dense generator matrices (lindbladian_kossakowski), full-rank A, every column."""
    re, im = W.random_kossakowski(N, 40 + N)
    A = re + 1j * im
    assert np.linalg.eigvalsh(A).min() > 0
    D = N * N - 1
    Q, K = Lb.unfold_dense_kossakowski(np.zeros((N, N), complex), A)
    R, K2 = Lb.kossakowski_columns(A, N, list(range(D)))
    assert np.abs(R - Q).max() < 1e-14 * np.abs(Q).max()
    assert np.abs(K - K2).max() < 1e-14 * np.abs(Q).max()


def test_populations_from_v_match_rho():
    """diag of the Eq. 6 reconstruction with the dense basis equals the D-generator formula."""
    for N in (2, 3, 6):
        rng = np.random.default_rng(N)
        X = rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))
        rho = X @ X.conj().T
        rho /= np.trace(rho)
        v = B.expand(rho).real
        assert np.abs(B.populations_from_v(v, N) - np.diag(rho).real).max() < 1e-15
