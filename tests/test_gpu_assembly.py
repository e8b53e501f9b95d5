"""Parity of the CUDA assembly (structure constants, expansion, Q0, Q1, R, K, rho, <O>) with the oracle.

FP64 assembly tolerance: 1e-12 relative to max|Q| (entries are sums of a few products of
square roots of rationals, so rounding differences are O(10 eps max|Q|)).
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import basis as OB
from oracle import lindblad as OL
from oracle import native as ON
from oracle import structure as OS
from oracle import system as SYS
from paper_1812_11626_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL_ASM = 1e-12


@pytest.fixture(scope="module")
def G():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1812_11626_gb300 import gksl
    return gksl


def csr_of(G, ctx, which):
    rp, col, val = G.get_csr_numpy(ctx, which)
    D = G.gksl_get_info(ctx).D
    return sp.csr_matrix((val, col, rp), shape=(D, D))


def rel_err(A, B):
    scale = max(abs(B).max(), 1e-300)
    return abs(A - B).max() / scale


# ------------------------------------------------------------ structure constants (Eq. 5)

@pytest.mark.parametrize("N", [2, 3, 4, 7, 12, 50, 200, 1000])
def test_structure_counts_match_paper(G, N):
    """Device enumeration of the closed-form nonzero set reproduces Sec. IV step 2.2's NZ_F, NZ_D."""
    assert G.gksl_structure_count(N, G.GKSL_STRUCT_F) == 5 * N**3 - 9 * N**2 - 2 * N + 6
    assert G.gksl_structure_count(N, G.GKSL_STRUCT_D) == 6 * N**3 - N * (21 * N + 7) // 2 + 1


@pytest.mark.parametrize("N", [2, 3, 4, 6])
def test_structure_values_match_brute_force(G, N):
    f, d = OS.structure_constants(N)
    for which, ref in ((G.GKSL_STRUCT_F, f), (G.GKSL_STRUCT_D, d)):
        n = G.gksl_structure_count(N, which)
        m_, n_, s_ = (np.zeros(max(n, 1), np.int32) for _ in range(3))
        val = np.zeros(max(n, 1))
        got = G.gksl_structure_enumerate(N, which, n, m_, n_, s_, val)
        assert got == n
        T = np.zeros_like(ref)
        T[m_[:n], n_[:n], s_[:n]] = val[:n]
        assert np.abs(T - ref).max() < 1e-15 * 8
        assert len(set(zip(m_[:n], n_[:n], s_[:n]))) == n   # no duplicates


# ------------------------------------------------------------ expansion (Sec. IV step 2.1)

@pytest.mark.parametrize("N,dens", [(2, 1.0), (7, 0.4), (33, 0.1)])
def test_expansion(G, N, dens):
    X = W.random_operator(N, dens, 100 + N)
    ctx = G.gksl_create(N)
    try:
        D = N * N - 1
        re, im = np.zeros(D), np.zeros(D)
        G.gksl_expand(ctx, X.rowptr, X.col, X.re, X.im, X.nnz, re, im)
        ref = OB.expand_sparse(X.to_scipy())
        assert np.abs((re + 1j * im) - ref).max() < 1e-14 * max(1.0, np.abs(ref).max())
    finally:
        G.gksl_destroy(ctx)


# ------------------------------------------------------------ assembly (Eq. 7, 10, 11)

def _random_ctx(G, N, seed, traceful=True):
    H0a = W.random_operator(N, 0.5, seed, hermitian=True)
    H0b = W.random_operator(N, 0.3, seed + 1, hermitian=True)
    H1 = W.random_operator(N, 0.4, seed + 2, hermitian=True)
    L0 = W.random_operator(N, 0.5, seed + 3, traceless=not traceful)
    L1 = W.random_operator(N, 0.3, seed + 4)
    ctx = G.gksl_create(N)
    G.set_csr_operator(G.gksl_set_h0_component, ctx, 0, 0.7, op=H0a)
    G.set_csr_operator(G.gksl_set_h0_component, ctx, 3, -1.3, op=H0b)
    G.set_csr_operator(G.gksl_set_h1, ctx, op=H1)
    G.set_csr_operator(G.gksl_set_dissipator, ctx, 0, 0.21, op=L0)
    G.set_csr_operator(G.gksl_set_dissipator, ctx, 2, 0.05, op=L1)
    G.gksl_set_drive(ctx, 0.4, 0.9, 1.3)
    G.gksl_assemble(ctx, G.GKSL_ASM_FP32 | G.GKSL_ASM_TRANSPOSE)
    ops = dict(H0a=H0a, H0b=H0b, H1=H1, L0=L0, L1=L1)
    return ctx, ops


@pytest.mark.parametrize("N", [2, 3, 5, 8])
def test_assembly_random_operators_vs_brute_force(G, N):
    """Q0, Q1, R_p, K against the dense definition Tr(F_s L(F_m)) with traceful, non-Hermitian L."""
    ctx, o = _random_ctx(G, N, 10 * N)
    try:
        D = N * N - 1
        d = lambda X: X.to_dense()
        Q0r, Kr = OL.unfold_dense(0.7 * d(o["H0a"]) - 1.3 * d(o["H0b"]), [d(o["L0"]), d(o["L1"])], [0.21, 0.05])
        Q1r, _ = OL.unfold_dense(d(o["H1"]))
        R0r, K0r = OL.unfold_dense(np.zeros((N, N)), [d(o["L0"])], [1.0])
        assert rel_err(csr_of(G, ctx, G.GKSL_MAT_Q0).toarray(), Q0r) < TOL_ASM
        assert rel_err(csr_of(G, ctx, G.GKSL_MAT_Q1).toarray(), Q1r) < TOL_ASM
        assert rel_err(csr_of(G, ctx, G.GKSL_MAT_R + 0).toarray(), R0r) < TOL_ASM
        K = np.zeros(D)
        G.gksl_get_k(ctx, K)
        assert np.abs(K - Kr).max() < TOL_ASM * np.abs(Q0r).max()
        K0 = np.zeros(D)
        G.gksl_get_k_channel(ctx, 0, K0)
        assert np.abs(K0 - K0r).max() < TOL_ASM * max(np.abs(R0r).max(), 1)
        Qh, _ = OL.unfold_dense(d(o["H0b"]))
        assert rel_err(csr_of(G, ctx, G.GKSL_MAT_H0 + 3).toarray(), Qh) < TOL_ASM
    finally:
        G.gksl_destroy(ctx)


@pytest.mark.parametrize("N", [10, 100])
def test_assembly_dimer_vs_oracle(G, N):
    d = W.dimer(N)
    ctx = G.dimer_context(d)
    try:
        u = SYS.unfold_dimer(d)
        p = d.params
        Q0r = u.q0(p["J"], p["U"], d.rate)
        scale = abs(Q0r).max()
        for which, ref in ((G.GKSL_MAT_Q0, Q0r), (G.GKSL_MAT_Q1, u.Q1), (G.GKSL_MAT_H0 + 0, u.QJ),
                           (G.GKSL_MAT_H0 + 1, u.QU), (G.GKSL_MAT_R + 0, u.R1)):
            M = csr_of(G, ctx, which)
            assert abs(M - ref).max() <= TOL_ASM * max(abs(ref).max(), 1e-300), which
        K = np.zeros(N * N - 1)
        G.gksl_get_k(ctx, K)
        assert np.abs(K - d.rate * u.K1).max() <= TOL_ASM * scale
        info = G.gksl_get_info(ctx)
        assert info.ell_width_q0 == 18 and info.ell_width_q1 == 1
    finally:
        G.gksl_destroy(ctx)


def test_assembly_dimer_n1000_full(G, record):
    """Largest configuration: every entry of Q0, Q1, K at N = 1000 (D = 999999) against the oracle."""
    N = 1000
    d = W.dimer(N)
    ctx = G.dimer_context(d, flags=G.GKSL_ASM_FP32)
    try:
        u = SYS.unfold_dimer(d)
        p = d.params
        Q0r = u.q0(p["J"], p["U"], d.rate)
        scale = abs(Q0r).max()
        Q0 = csr_of(G, ctx, G.GKSL_MAT_Q0)
        record("q0_max_abs_err_over_max_q0", abs(Q0 - Q0r).max() / scale)
        assert abs(Q0 - Q0r).max() <= TOL_ASM * scale
        Q1 = csr_of(G, ctx, G.GKSL_MAT_Q1)
        record("q1_max_abs_err_over_max_q1", abs(Q1 - u.Q1).max() / abs(u.Q1).max())
        assert abs(Q1 - u.Q1).max() <= TOL_ASM * abs(u.Q1).max()
        K = np.zeros(N * N - 1)
        G.gksl_get_k(ctx, K)
        record("k_max_abs_err_over_max_q0", np.abs(K - d.rate * u.K1).max() / scale)
        assert np.abs(K - d.rate * u.K1).max() <= TOL_ASM * scale
        info = G.gksl_get_info(ctx)
        # propagation matrix Q0 + E Q1 after the 64 eps max|Q| drop has 18 448 539 entries (oracle,
        # same drop), plus the K column on the N-1 diagonal generators
        Qe = (Q0r + p["E"] * u.Q1).tocsr()
        Qe.data[np.abs(Qe.data) <= 64 * np.finfo(float).eps * abs(Qe).max()] = 0
        Qe.eliminate_zeros()
        nk = int((np.abs(d.rate * u.K1) > 64 * np.finfo(float).eps * abs(Qe).max()).sum())
        record("nnz_q0_gpu", info.nnz_q0)
        record("nnz_q0_oracle", Qe.nnz + nk)
        assert abs(info.nnz_q0 - (Qe.nnz + nk)) <= 10, (info.nnz_q0, Qe.nnz, nk)
        assert info.ell_width_q0 == 18
    finally:
        G.gksl_destroy(ctx)


def test_kossakowski_matrix_vs_eq8(G):
    """General dissipator from a rank-3 Kossakowski matrix (Eq. 8, factorised into three channels)
    against the oracle's Eq. 8 applied with A directly; a rank-9 matrix (more channels than
    GKSL_MAX_P) takes the dense route and matches too; an indefinite one is rejected."""
    N = 5
    M = N * N - 1
    rng = np.random.default_rng(21)
    H = W.random_operator(N, 0.6, 77, hermitian=True)
    C = rng.normal(size=(M, 3)) + 1j * rng.normal(size=(M, 3))
    A = C @ C.conj().T * 0.05
    ctx = G.gksl_create(N)
    try:
        G.set_csr_operator(G.gksl_set_h0_component, ctx, 0, 1.0, op=H)
        G.gksl_set_drive(ctx, 0.0, 0.0, 1.0)
        G.gksl_set_kossakowski(ctx, A.real.copy(), A.imag.copy())
        G.gksl_assemble(ctx, 0)
        Qr, Kr = OL.unfold_dense_kossakowski(H.to_dense(), A)
        assert rel_err(csr_of(G, ctx, G.GKSL_MAT_Q0).toarray(), Qr) < TOL_ASM
        K = np.zeros(M)
        G.gksl_get_k(ctx, K)
        assert np.abs(K - Kr).max() < TOL_ASM * np.abs(Qr).max()
        assert G.gksl_get_info(ctx).nnz_r[2] > 0   # three channels
        C9 = rng.normal(size=(M, 9)) + 1j * rng.normal(size=(M, 9))
        A9 = C9 @ C9.conj().T * 0.05
        G.gksl_set_kossakowski(ctx, A9.real.copy(), A9.imag.copy())
        G.gksl_assemble(ctx, 0)
        assert G.gksl_get_info(ctx).nnz_r[1] == 0   # one channel holds the whole matrix
        Qr, Kr = OL.unfold_dense_kossakowski(H.to_dense(), A9)
        assert rel_err(csr_of(G, ctx, G.GKSL_MAT_Q0).toarray(), Qr) < TOL_ASM
        G.gksl_get_k(ctx, K)
        assert np.abs(K - Kr).max() < TOL_ASM * np.abs(Qr).max()
        Aneg = A.copy()
        Aneg[0, 0] -= 10 * np.abs(A).max()
        with pytest.raises(G.GkslError):
            G.gksl_set_kossakowski(ctx, Aneg.real.copy(), Aneg.imag.copy())
    finally:
        G.gksl_destroy(ctx)


@pytest.mark.parametrize("N", [12, 16])
def test_dense_operators_vs_brute_force(G, N):
    """Fully dense H and a dense non-Hermitian L (the dense column of Table II): assembly against the
    brute-force definition."""
    H = W.random_operator(N, 1.0, 300 + N, hermitian=True)
    L = W.random_operator(N, 1.0, 400 + N)
    ctx = G.gksl_create(N)
    try:
        G.set_csr_operator(G.gksl_set_h0_component, ctx, 0, 1.0, op=H)
        G.set_csr_operator(G.gksl_set_dissipator, ctx, 0, 0.2, op=L)
        G.gksl_set_drive(ctx, 0.0, 0.0, 1.0)
        G.gksl_assemble(ctx, 0)
        Qr, Kr = OL.unfold_dense(H.to_dense(), [L.to_dense()], [0.2])
        assert rel_err(csr_of(G, ctx, G.GKSL_MAT_Q0).toarray(), Qr) < TOL_ASM
        K = np.zeros(N * N - 1)
        G.gksl_get_k(ctx, K)
        assert np.abs(K - Kr).max() < TOL_ASM * np.abs(Qr).max()
    finally:
        G.gksl_destroy(ctx)


# ------------------------------------------------------------ state, rho, observables (Eq. 6)

def test_rho0_rho_and_observable(G):
    N = 9
    rng = np.random.default_rng(5)
    X = rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))
    rho = X @ X.conj().T
    rho /= np.trace(rho)
    d = W.dimer(N)
    ctx = G.dimer_context(d)
    try:
        G.gksl_set_rho0(ctx, rho.real.copy(), rho.imag.copy())
        D = N * N - 1
        v = np.zeros(D)
        t = G.gksl_get_state(ctx, v)
        assert t == 0.0
        assert np.abs(v - OB.expand(rho).real).max() < 1e-15
        re, im = np.zeros((N, N)), np.zeros((N, N))
        G.gksl_rho(ctx, v, re, im)
        assert np.abs(re + 1j * im - rho).max() < 1e-15
        o = np.arange(N, dtype=float) ** 2 - 3.0
        out = np.zeros(2)
        G.gksl_observable_diag(ctx, o, np.stack([v, 2 * v]), 2, out)
        assert abs(out[0] - np.trace(np.diag(o) @ rho).real) < 1e-13
        w, c0 = __import__("oracle.propagate", fromlist=["x"]).observable_weights(o)
        assert abs(out[1] - (c0 + 2 * w @ v)) < 1e-13
    finally:
        G.gksl_destroy(ctx)


def test_argument_validation(G):
    N = 4
    ctx = G.gksl_create(N)
    try:
        H = W.random_operator(N, 1.0, 3)   # not Hermitian
        with pytest.raises(G.GkslError) as e:
            G.set_csr_operator(G.gksl_set_h1, ctx, op=H)
        assert e.value.status == G.GKSL_ERR_ARG
        bad = W.random_operator(N, 1.0, 4, hermitian=True)
        col = bad.col.copy()
        col[0] = N + 3
        with pytest.raises(G.GkslError):
            G.gksl_set_h1(ctx, bad.rowptr, col, bad.re, bad.im, bad.nnz)
        with pytest.raises(G.GkslError) as e:
            G.gksl_assemble(ctx, 0)
        assert e.value.status == G.GKSL_ERR_STATE
        with pytest.raises(G.GkslError) as e:
            G.gksl_propagate(ctx, 10, 10, 64)
        assert e.value.status == G.GKSL_ERR_STATE
    finally:
        G.gksl_destroy(ctx)


def test_assembly_is_well_formed_and_deterministic(G):
    """compute-sanitizer is closed on this machine; in its place every assembled matrix is checked
    for well-formed CSR (monotone row pointers, columns in range, strictly increasing within a
    row, finite values), and two assemblies of the same operators -- a dimer and general random
    operators with two channels -- must agree bit for bit (the atomic-based scatter of the radix
    sort must not leak its ordering into the result), as must two propagations from them."""
    def mats(ctx):
        out = {}
        for which in (G.GKSL_MAT_Q0, G.GKSL_MAT_Q1, G.GKSL_MAT_H0 + 0, G.GKSL_MAT_R + 0):
            out[which] = G.get_csr_numpy(ctx, which)
        K = np.zeros(G.gksl_get_info(ctx).D)
        G.gksl_get_k(ctx, K)
        out["K"] = K
        return out

    def check(m, D):
        for which, val in m.items():
            if which == "K":
                assert np.all(np.isfinite(val))
                continue
            rp, col, v = val
            nnz = int(rp[-1])
            assert rp[0] == 0 and np.all(np.diff(rp) >= 0), which
            col, v = col[:nnz], v[:nnz]
            assert np.all((col >= 0) & (col < D)), which
            for r in range(D):
                c = col[rp[r]:rp[r + 1]]
                assert np.all(np.diff(c) > 0), (which, r)
            assert np.all(np.isfinite(v)), which

    def build_dimer():
        return G.dimer_context(W.dimer(40))

    def build_random():
        N = 9
        ctx = G.gksl_create(N)
        G.set_csr_operator(G.gksl_set_h0_component, ctx, 0, 0.7, op=W.random_operator(N, 0.5, 11, hermitian=True))
        G.set_csr_operator(G.gksl_set_h1, ctx, op=W.random_operator(N, 0.4, 12, hermitian=True))
        G.set_csr_operator(G.gksl_set_dissipator, ctx, 0, 0.3, op=W.random_operator(N, 0.5, 13))
        G.set_csr_operator(G.gksl_set_dissipator, ctx, 1, 0.2, op=W.random_operator(N, 0.5, 14))
        G.gksl_set_drive(ctx, 0.4, 0.6, 1.5)
        G.gksl_assemble(ctx, G.GKSL_ASM_FP32)
        rho0 = np.eye(N) / N
        G.gksl_set_rho0(ctx, rho0)
        return ctx

    for build in (build_dimer, build_random):
        runs = []
        for _ in range(2):
            ctx = build()
            try:
                D = G.gksl_get_info(ctx).D
                m = mats(ctx)
                check(m, D)
                out = np.zeros((1, D))
                G.gksl_propagate(ctx, 400, 100, 64, 0, 100, out)
                runs.append((m, out))
            finally:
                G.gksl_destroy(ctx)
        (m1, o1), (m2, o2) = runs
        for which in m1:
            if which == "K":
                assert np.array_equal(m1[which], m2[which])
            else:
                for a, b in zip(m1[which], m2[which]):
                    assert np.array_equal(a, b), which
        assert np.array_equal(o1, o2)
