"""General dissipators in the dense regime (Table II, dense column; Sec. VI, random Lindbladians):
the dense route of the assembly against the oracle's definition routes.

* small N: every channel forced onto the dense route (GKSL_ASM_DENSE_DISSIPATORS) and the sparse
  route, both against Q_sm = Tr(F_s L(F_m)) on dense matrices, with traceful non-Hermitian L;
* full-rank Kossakowski matrices (Eq. 8) at small N against Eq. 8 applied directly;
* N = 100 with a dense L (the assembly switches to the dense route by itself): every entry of R
  and K against the C oracle's column-by-column definition, then RK4 from a dense state against
  the oracle's RK4;
* N = 100 with a full-rank Kossakowski matrix (D^2 = 1e8 entries of A): sampled columns of R and
  all of K against the oracle's column-wise Eq. 8 (``lindblad.kossakowski_columns``).

Tolerance: 1e-12 of max |Q| on assembled matrices (the FP64 assembly bound); FP64 propagation
1e-10 on v.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import basis as OB
from oracle import lindblad as OL
from oracle import native
from paper_1812_11626_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL_ASM = 1e-12


@pytest.fixture(scope="module")
def G():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1812_11626_gb300 import gksl
    return gksl


def _csr(G, ctx, which):
    rp, col, val = G.get_csr_numpy(ctx, which)
    D = G.gksl_get_info(ctx).D
    return sp.csr_matrix((val, col, rp), shape=(D, D))


@pytest.mark.parametrize("N", [2, 3, 5, 8])
def test_dense_route_small_n_vs_definition(G, N, record):
    """Two traceful non-Hermitian channels and a random H: R_p, K_p and Q0, K from the dense route
    and from the sparse route, each against the dense definition route."""
    H = W.random_operator(N, 0.7, 500 + N, hermitian=True)
    Ls = [W.random_operator(N, 1.0, 510 + N), W.random_operator(N, 0.5, 520 + N)]
    gam = [0.3, 0.7]
    Qr, Kr = OL.unfold_dense(H.to_dense(), [L.to_dense() for L in Ls], gam)
    scale = np.abs(Qr).max()
    for flags in (G.GKSL_ASM_DENSE_DISSIPATORS, 0):
        ctx = G.gksl_create(N)
        try:
            G.set_csr_operator(G.gksl_set_h0_component, ctx, 0, 1.0, op=H)
            for p, (g, L) in enumerate(zip(gam, Ls)):
                G.set_csr_operator(G.gksl_set_dissipator, ctx, 2 * p, g, op=L)
            G.gksl_set_drive(ctx, 0.0, 0.0, 1.0)
            G.gksl_assemble(ctx, flags)
            err = np.abs(_csr(G, ctx, G.GKSL_MAT_Q0).toarray() - Qr).max() / scale
            K = np.zeros(N * N - 1)
            G.gksl_get_k(ctx, K)
            assert err < TOL_ASM and np.abs(K - Kr).max() < TOL_ASM * scale, (flags, err)
            for p, L in enumerate(Ls):
                Rp, Kp = OL.unfold_dense(np.zeros((N, N), complex), [L.to_dense()], [1.0])
                Kg = np.zeros(N * N - 1)
                G.gksl_get_k_channel(ctx, 2 * p, Kg)
                assert np.abs(_csr(G, ctx, G.GKSL_MAT_R + 2 * p).toarray() - Rp).max() < TOL_ASM * np.abs(Rp).max()
                assert np.abs(Kg - Kp).max() < TOL_ASM * np.abs(Rp).max()
            if flags:
                record("dense_route_max_rel_err", err)
        finally:
            G.gksl_destroy(ctx)


@pytest.mark.parametrize("N", [3, 4, 6])
def test_kossakowski_full_rank_small_n_vs_eq8(G, N):
    """A full-rank Kossakowski matrix (rank D > 8 channels) goes to the dense route; Q0 and K match
    Eq. 8 applied with A directly, with a random H."""
    re, im = W.random_kossakowski(N, 60 + N, scale=0.2)
    A = re + 1j * im
    H = W.random_operator(N, 0.8, 70 + N, hermitian=True)
    ctx = G.gksl_create(N)
    try:
        G.set_csr_operator(G.gksl_set_h0_component, ctx, 0, 1.0, op=H)
        G.gksl_set_drive(ctx, 0.0, 0.0, 1.0)
        G.gksl_set_kossakowski(ctx, re, im)
        G.gksl_assemble(ctx, G.GKSL_ASM_TRANSPOSE)
        Qr, Kr = OL.unfold_dense_kossakowski(H.to_dense(), A)
        scale = np.abs(Qr).max()
        assert np.abs(_csr(G, ctx, G.GKSL_MAT_Q0).toarray() - Qr).max() < TOL_ASM * scale
        K = np.zeros(N * N - 1)
        G.gksl_get_k(ctx, K)
        assert np.abs(K - Kr).max() < TOL_ASM * scale
        assert G.gksl_min_stable_steps(ctx) >= 1
    finally:
        G.gksl_destroy(ctx)


def test_kossakowski_dense_route_rejects_indefinite(G):
    """On the dense route positive semidefiniteness is checked through the diagonal and the 2 x 2
    principal minors: a negative diagonal entry and an oversized off-diagonal pair are rejected,
    and a rejected matrix leaves the channels set before it untouched."""
    N = 9   # N > 64 is not needed: rank D > 8 sends any full-rank matrix to the dense route
    re, im = W.random_kossakowski(N, 5)
    ctx = G.gksl_create(N)
    try:
        L = W.random_operator(N, 0.5, 6)
        G.set_csr_operator(G.gksl_set_dissipator, ctx, 1, 0.3, op=L)   # kept if a matrix is rejected
        G.gksl_set_drive(ctx, 0.0, 0.0, 1.0)
        bad = re.copy()
        bad[3, 3] = -1.0
        with pytest.raises(G.GkslError) as e:
            G.gksl_set_kossakowski(ctx, bad, im)
        assert e.value.status == G.GKSL_ERR_ARG
        bad = re.copy()
        bad[1, 2] = bad[2, 1] = 10.0 * np.sqrt(re[1, 1] * re[2, 2])
        with pytest.raises(G.GkslError):
            G.gksl_set_kossakowski(ctx, bad, im)
        # the rejected calls left the channel set before them in place
        G.gksl_assemble(ctx, 0)
        Rp, _ = OL.unfold_dense(np.zeros((N, N), complex), [L.to_dense()], [1.0])
        assert np.abs(_csr(G, ctx, G.GKSL_MAT_R + 1).toarray() - Rp).max() < TOL_ASM * np.abs(Rp).max()
    finally:
        G.gksl_destroy(ctx)


def test_dense_l_n100_every_entry_and_propagation(G, record):
    """N = 100 (D = 9 999) with a fully dense, traceful, non-Hermitian L and a random sparse H: the
    assembly takes the dense route by itself (the sparse route's product would have ~5e9 terms);
    every entry of R and K against the C oracle's definition route, then 40 FP64 RK4 steps from a
    dense state against the oracle's RK4 on its own matrices."""
    N, g = 100, 0.02
    D = N * N - 1
    H = W.random_operator(N, 0.05, 900, hermitian=True)
    H1 = W.CSR.from_dense(np.diag(np.linspace(-1.0, 1.0, N)).astype(complex))
    L = W.random_operator(N, 1.0, 901)
    ctx = G.gksl_create(N)
    try:
        G.set_csr_operator(G.gksl_set_h0_component, ctx, 0, 1.0, op=H)
        G.set_csr_operator(G.gksl_set_h1, ctx, op=H1)
        G.set_csr_operator(G.gksl_set_dissipator, ctx, 0, g, op=L)
        G.gksl_set_drive(ctx, 0.3, 0.5, 1.0)
        sec = G.gksl_assemble(ctx, 0)
        info = G.gksl_get_info(ctx)
        record("assemble_seconds", sec)
        record("nnz_R", info.nnz_r[0])
        record("nnz_Q0_plus_E_Q1", info.nnz_q0)
        Rg = _csr(G, ctx, G.GKSL_MAT_R)
        Kg = np.zeros(D)
        G.gksl_get_k_channel(ctx, 0, Kg)
        Ro, Ko, _ = native.unfold(N, A=L.to_scipy(), gamma=1.0)
        scale = abs(Ro).max()
        errR = abs(Rg - Ro).max() / scale
        record("R_max_abs_diff_over_max", errR)
        assert errR < TOL_ASM
        assert np.abs(Kg - Ko).max() < TOL_ASM * scale
        assert info.nnz_r[0] > 0.9 * D * D   # dense
        # propagation from a dense state
        QH, _, _ = native.unfold(N, H=H.to_scipy(), want_k=False)
        Q1, _, _ = native.unfold(N, H=H1.to_scipy(), want_k=False)
        re, im = W.random_density_matrix(N, 3, 902)
        v0 = OB.expand_dense(re + 1j * im).real
        spp = G.gksl_min_stable_steps(ctx)
        n = 40
        G.gksl_set_rho0(ctx, re, im)
        out = np.zeros((1, D))
        G.gksl_propagate(ctx, spp, n, 64, 0, n, out)
        ref, _ = native.rk4((QH + g * Ro).tocsr(), Q1, g * Ko, 0.3, 0.5, 1.0, v0, 2 * np.pi / spp, n)
        err = np.abs(out[0] - ref).max()
        record("rk4_max_abs_dv_vs_oracle", err)
        assert err < 1e-10 and err < 1e-9 * np.abs(ref - v0).max(), err
    finally:
        G.gksl_destroy(ctx)


def test_kossakowski_full_rank_n100_vs_eq8_columns(G, record):
    """N = 100 with a full-rank Kossakowski matrix (D = 9 999, A of 1e8 complex entries) contracted on
    the device: 12 columns of R (the first and last S, J and D generators and six others) and all of
    K against Eq. 8 evaluated column by column by the oracle; then a few RK4 steps keep rho a
    density matrix (trace 1, eigenvalues >= -1e-8)."""
    N = 100
    D = N * N - 1
    re, im = W.random_kossakowski(N, 1812, scale=0.05)
    ctx = G.gksl_create(N)
    try:
        H = W.random_operator(N, 0.05, 903, hermitian=True)
        G.set_csr_operator(G.gksl_set_h0_component, ctx, 0, 1.0, op=H)
        G.gksl_set_drive(ctx, 0.0, 0.0, 1.0)
        G.gksl_set_kossakowski(ctx, re, im)
        sec = G.gksl_assemble(ctx, 0)
        info = G.gksl_get_info(ctx)
        record("assemble_seconds", sec)
        record("nnz_R", info.nnz_r[0])
        Rg = _csr(G, ctx, G.GKSL_MAT_R)
        Kg = np.zeros(D)
        G.gksl_get_k_channel(ctx, 0, Kg)
        P2 = N * (N - 1) // 2
        rng = np.random.default_rng(7)
        cols = sorted({0, P2 - 1, P2, 2 * P2 - 1, 2 * P2, D - 1} | set(rng.integers(0, D, 6).tolist()))
        Ro, Ko = OL.kossakowski_columns(re + 1j * im, N, cols)
        scale = np.abs(Ro).max()
        errR = np.abs(Rg[:, cols].toarray() - Ro).max() / scale
        record("R_sampled_columns_max_abs_diff_over_max", errR)
        assert errR < TOL_ASM
        assert np.abs(Kg - Ko).max() < TOL_ASM * scale
        # physical sanity of the propagated state (Eq. 6): trace one, positive
        rr, ri = W.random_density_matrix(N, 3, 904)
        G.gksl_set_rho0(ctx, rr, ri)
        spp = G.gksl_min_stable_steps(ctx)
        out = np.zeros((1, D))
        G.gksl_propagate(ctx, spp, 50, 64, 0, 50, out)
        re_o, im_o = np.zeros((N, N)), np.zeros((N, N))
        G.gksl_rho(ctx, out[0], re_o, im_o)
        rho = re_o + 1j * im_o
        assert abs(np.trace(rho) - 1) < 1e-12
        assert np.linalg.eigvalsh(rho).min() > -1e-8
    finally:
        G.gksl_destroy(ctx)


def test_dense_routes_reject_sizes_past_their_limits(G):
    """The dense dissipator route holds R as D^2 < 2^31 entries (N <= 200) and the Kossakowski form
    holds the kernel M of N^4 complex entries (N <= 128).  Past those sizes the calls return
    GKSL_ERR_ARG before reading or allocating anything, and the context stays usable: at N = 201
    the sparse route still assembles the same operators."""
    N = 201
    d = W.dimer(N)
    ctx = G.dimer_context(d, assemble=False)
    try:
        with pytest.raises(G.GkslError) as e:
            G.gksl_assemble(ctx, G.GKSL_ASM_DENSE_DISSIPATORS)
        assert e.value.status == G.GKSL_ERR_ARG and "N <= 200" in str(e.value)
        G.gksl_assemble(ctx, 0)
        assert G.gksl_get_info(ctx).nnz_q0 > 0
    finally:
        G.gksl_destroy(ctx)
    ctx = G.gksl_create(129)
    try:
        with pytest.raises(G.GkslError) as e:
            # the size is checked before A is read, so a placeholder array suffices
            G.gksl_set_kossakowski(ctx, np.zeros(1))
        assert e.value.status == G.GKSL_ERR_ARG and "N <= 128" in str(e.value)
    finally:
        G.gksl_destroy(ctx)


def test_kossakowski_device_checks_at_n65(G):
    """Above N = 64 a Kossakowski matrix is copied to the device and checked there.  At N = 65
    (D = 4 224): a non-finite entry, a non-Hermitian pair, a negative diagonal entry and an
    oversized off-diagonal pair (a negative 2 x 2 principal minor) are each rejected with the host
    route's status and message, and leave the channel set before them in place (its assembled R
    equals that of a context holding only that channel, bit for bit); a valid matrix given as host
    arrays and as CUDA tensors assembles to the same R bit for bit."""
    import torch
    N = 65
    D = N * N - 1
    re, im = W.random_kossakowski(N, 65, scale=0.1)
    L = W.random_operator(N, 0.05, 66)

    def assembled_r(ctx, p):
        G.gksl_set_drive(ctx, 0.0, 0.0, 1.0)
        G.gksl_assemble(ctx, 0)
        return _csr(G, ctx, G.GKSL_MAT_R + p)

    ref = G.gksl_create(N)
    try:
        G.set_csr_operator(G.gksl_set_dissipator, ref, 1, 0.3, op=L)
        R_ref = assembled_r(ref, 1)
    finally:
        G.gksl_destroy(ref)
    ctx = G.gksl_create(N)
    try:
        G.set_csr_operator(G.gksl_set_dissipator, ctx, 1, 0.3, op=L)
        cases = []
        bad = re.copy(); bad[7, 11] = np.nan
        cases.append((bad, im, "non-finite"))
        bad = re.copy(); bad[3, 9] += 1e-3 * np.abs(re).max()
        cases.append((bad, im, "not Hermitian"))
        bad = re.copy(); bad[D - 1, D - 1] = -1.0
        cases.append((bad, im, "not positive semidefinite"))
        bad = re.copy(); bad[1, 2] = bad[2, 1] = 10.0 * np.sqrt(re[1, 1] * re[2, 2])
        cases.append((bad, im, "2 x 2 principal minor"))
        for a_re, a_im, what in cases:
            with pytest.raises(G.GkslError) as e:
                G.gksl_set_kossakowski(ctx, a_re, a_im)
            assert e.value.status == G.GKSL_ERR_ARG and what in str(e.value), (what, str(e.value))
        R_kept = assembled_r(ctx, 1)
        assert (R_kept != R_ref).nnz == 0
    finally:
        G.gksl_destroy(ctx)
    Rs = []
    for on_device in (False, True):
        ctx = G.gksl_create(N)
        try:
            if on_device:
                dev = torch.device("cuda", 0)
                G.gksl_set_kossakowski(ctx, torch.as_tensor(re, device=dev), torch.as_tensor(im, device=dev))
            else:
                G.gksl_set_kossakowski(ctx, re, im)
            Rs.append(assembled_r(ctx, 0))
        finally:
            G.gksl_destroy(ctx)
    assert Rs[0].nnz > 0 and (Rs[0] != Rs[1]).nnz == 0
