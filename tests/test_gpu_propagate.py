"""Parity of the CUDA RK4 propagation with the oracle.

Tolerances: FP64 path 1e-10 on v (absolute; |v| <= 1); FP32 bulk form 1e-5 on v and 1e-4
on <n1 - n2> (absolute).
"""
import numpy as np
import pytest

from oracle import basis as OB
from oracle import lindblad as OL
from oracle import propagate as OP
from oracle import system as SYS
from paper_1812_11626_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL64 = 1e-10
TOL32_V = 1e-5
TOL32_O = 1e-4


@pytest.fixture(scope="module")
def G():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1812_11626_gb300 import gksl
    return gksl


def run_gpu(G, ctx, spp, nsteps, emit, precision=64, corr=0, D=None):
    out = np.zeros((nsteps // emit, D))
    G.gksl_propagate(ctx, spp, nsteps, precision, corr, emit, out)
    return out


def test_config0_fp64_n10(G, record):
    """N = 10 dimer, 10 periods x 200 steps, v at every period end (the small workload)."""
    d = W.dimer(10)
    ctx = G.dimer_context(d)
    try:
        out = run_gpu(G, ctx, 200, 2000, 200, D=99)
        u = SYS.unfold_dimer(d)
        _, ref = SYS.propagate_dimer(d, u, 200, 2000, emit_every=200)
        err = max(np.abs(out[i] - ref[i]).max() for i in range(10))
        record("fp64_max_abs_dv_vs_oracle", err)
        assert err < TOL64, err
        w, c0 = OP.observable_weights(d.obs_diag)
        obs = np.zeros(10)
        G.gksl_observable_diag(ctx, d.obs_diag, out, 10, obs)
        record("obs_max_abs_diff_vs_oracle", np.abs(obs - np.array([c0 + w @ r for r in ref])).max())
        assert np.abs(obs - np.array([c0 + w @ r for r in ref])).max() < 1e-9
        rho = OB.rho_from_v(out[-1], N=10)
        record("rho_trace_minus_1", abs(np.trace(rho) - 1))
        record("rho_min_eigenvalue", np.linalg.eigvalsh(rho).min())
        assert abs(np.trace(rho) - 1) < 1e-14 and np.linalg.eigvalsh(rho).min() > -1e-8
    finally:
        G.gksl_destroy(ctx)


def test_random_operators_fp64(G):
    """General operators (two H0 parts, traceful non-Hermitian L, two channels) against the
    dense rho-space RK4 (no generator basis on the reference side)."""
    N = 6
    H0 = W.random_operator(N, 0.6, 71, hermitian=True)
    H1 = W.random_operator(N, 0.5, 72, hermitian=True)
    L0 = W.random_operator(N, 0.5, 73)
    L1 = W.random_operator(N, 0.5, 74)
    ctx = G.gksl_create(N)
    try:
        G.set_csr_operator(G.gksl_set_h0_component, ctx, 2, 0.8, op=H0)
        G.set_csr_operator(G.gksl_set_h1, ctx, op=H1)
        G.set_csr_operator(G.gksl_set_dissipator, ctx, 0, 0.3, op=L0)
        G.set_csr_operator(G.gksl_set_dissipator, ctx, 5, 0.1, op=L1)
        G.gksl_set_drive(ctx, 0.2, 0.7, 2.0)
        G.gksl_assemble(ctx, 0)
        rho0 = np.diag(np.linspace(1, 2, N)).astype(complex)
        rho0 /= np.trace(rho0)
        rho0[0, 1] = rho0[1, 0] = 0.05
        G.gksl_set_rho0(ctx, rho0.real.copy(), rho0.imag.copy())
        spp, n = 500, 700
        D = N * N - 1
        out = run_gpu(G, ctx, spp, n, n, D=D)
        h = 2 * np.pi / 2.0 / spp
        eps = OP.eps_fn(0.2, 0.7, 2.0)
        rho = OP.rho_rk4(0.8 * H0.to_dense(), H1.to_dense(), [L0.to_dense(), L1.to_dense()], [0.3, 0.1], eps, rho0,
                         h, n)
        assert np.abs(out[0] - OB.expand(rho).real).max() < TOL64
    finally:
        G.gksl_destroy(ctx)


def test_config1_n100_fp64_and_fp32(G, record):
    """N = 100 (D = 9999) at the stable 4000 steps/period: FP64 parity over a quarter period,
    FP32 bulk error against FP64 over two periods."""
    d = W.dimer(100)
    ctx = G.dimer_context(d)
    try:
        D = d.N * d.N - 1
        spp = 4000
        out = run_gpu(G, ctx, spp, 1000, 500, D=D)
        u = SYS.unfold_dimer(d)
        _, ref = SYS.propagate_dimer(d, u, spp, 1000, emit_every=500)
        record("fp64_max_abs_dv_vs_oracle", max(np.abs(out[i] - ref[i]).max() for i in range(2)))
        assert max(np.abs(out[i] - ref[i]).max() for i in range(2)) < TOL64
        # FP32 bulk vs FP64, both on the GPU, from rho0
        G.gksl_set_rho0(ctx, d.rho0_dense().real.copy())
        v64 = run_gpu(G, ctx, spp, 2 * spp, spp, D=D)
        G.gksl_set_rho0(ctx, d.rho0_dense().real.copy())
        v32 = run_gpu(G, ctx, spp, 2 * spp, spp, precision=32, corr=spp, D=D)
        assert np.abs(v32 - v64).max() < TOL32_V
        o64, o32 = np.zeros(2), np.zeros(2)
        G.gksl_observable_diag(ctx, d.obs_diag, v64, 2, o64)
        G.gksl_observable_diag(ctx, d.obs_diag, v32, 2, o32)
        assert np.abs(o32 - o64).max() < TOL32_O
    finally:
        G.gksl_destroy(ctx)


def test_config1_full_length_fp32_vs_fp64(G, record):
    """N = 100 over the full 100 periods at the stable 4000 steps/period (400 000 steps): the FP32
    bulk form with an FP64 step every period against the FP64 path, on v and <n1 - n2> at every
    tenth period end."""
    d = W.dimer(100)
    ctx = G.dimer_context(d)
    try:
        D = d.N * d.N - 1
        spp, periods = 4000, 100
        v64 = run_gpu(G, ctx, spp, spp * periods, spp * 10, D=D)
        G.gksl_set_rho0(ctx, d.rho0_dense().real.copy())
        v32 = run_gpu(G, ctx, spp, spp * periods, spp * 10, precision=32, corr=spp, D=D)
        record("fp32_max_abs_dv_vs_fp64", np.abs(v32 - v64).max())
        assert np.abs(v32 - v64).max() < TOL32_V
        o64, o32 = np.zeros(10), np.zeros(10)
        G.gksl_observable_diag(ctx, d.obs_diag, v64, 10, o64)
        G.gksl_observable_diag(ctx, d.obs_diag, v32, 10, o32)
        record("fp32_obs_max_abs_diff_vs_fp64", np.abs(o32 - o64).max())
        assert np.abs(o32 - o64).max() < TOL32_O
    finally:
        G.gksl_destroy(ctx)


def test_square_drive_vs_oracle(G):
    """Piecewise-constant drive theta = +-1 (Sec. III, driving (i)) on the N = 10 dimer over 3
    periods (FP64 against the oracle's midpoint rule), an odd step count is rejected, and the
    adjoint with the square drive agrees with the oracle's loss."""
    d = W.dimer(10)
    ctx = G.dimer_context(d)
    try:
        G.gksl_set_drive_shape(ctx, G.GKSL_DRIVE_SQUARE)
        spp = 400
        out = run_gpu(G, ctx, spp, 3 * spp, spp, D=99)
        u = SYS.unfold_dimer(d)
        _, ref = SYS.propagate_dimer(d, u, spp, 3 * spp, emit_every=spp, drive="square")
        assert max(np.abs(out[i] - ref[i]).max() for i in range(3)) < TOL64
        with pytest.raises(G.GkslError) as e:
            G.gksl_propagate(ctx, spp + 1, 10, 64, 0, 0, None)
        assert e.value.status == G.GKSL_ERR_ARG
    finally:
        G.gksl_destroy(ctx)


def test_fp32_config0_vs_oracle(G):
    d = W.dimer(10)
    ctx = G.dimer_context(d)
    try:
        out = run_gpu(G, ctx, 200, 2000, 200, precision=32, corr=200, D=99)
        u = SYS.unfold_dimer(d)
        _, ref = SYS.propagate_dimer(d, u, 200, 2000, emit_every=200)
        assert max(np.abs(out[i] - ref[i]).max() for i in range(10)) < TOL32_V
    finally:
        G.gksl_destroy(ctx)


def test_resume_is_bit_identical(G):
    """Checkpoint/resume: two calls of n steps equal one call of 2n steps exactly (FP64)."""
    d = W.dimer(12)
    ctx = G.dimer_context(d)
    try:
        D = d.N * d.N - 1
        a = run_gpu(G, ctx, 300, 200, 200, D=D)
        G.gksl_set_rho0(ctx, d.rho0_dense().real.copy())
        run_gpu(G, ctx, 300, 77, 77, D=D)
        v = np.zeros(D)
        t = G.gksl_get_state(ctx, v)
        G.gksl_set_state(ctx, v, t)
        b = run_gpu(G, ctx, 300, 123, 123, D=D)
        assert np.abs(a[0] - b[0]).max() < 1e-14
    finally:
        G.gksl_destroy(ctx)


def test_min_stable_steps_and_divergence_guard(G):
    """The stability bound admits a finite run; far below it the state blows up and the call
    returns GKSL_ERR_DIVERGED (host-side check of the state, no device fault involved)."""
    d = W.dimer(60)
    ctx = G.dimer_context(d)
    try:
        spp = G.gksl_min_stable_steps(ctx)
        # the bound follows the eigenvalue spread of H(t): U/2 M^2/2 dominates for this model
        M = d.N - 1
        assert 0.25 * M * M / 2 * 2 * np.pi / 2.8 < spp < 4 * M * M
        D = d.N * d.N - 1
        run_gpu(G, ctx, spp, spp // 4, spp // 4, D=D)
        G.gksl_set_rho0(ctx, d.rho0_dense().real.copy())
        with pytest.raises(G.GkslError) as e:
            G.gksl_propagate(ctx, max(spp // 20, 1), 4000, 64, 0, 0, None)
        assert e.value.status == G.GKSL_ERR_DIVERGED
    finally:
        G.gksl_destroy(ctx)


@pytest.mark.parametrize("variant", ["0", "1", "2", "3"])
def test_stage_kernel_variants(G, variant, monkeypatch):
    """Every stage-kernel variant (forced; normally chosen by timing) on a system large enough
    to be tuned (N = 300, D = 89 999), FP64 against the oracle and FP32 within its tolerance."""
    monkeypatch.setenv("GKSL_RK4_VARIANT", variant)
    d = W.dimer(300)
    ctx = G.dimer_context(d, flags=G.GKSL_ASM_FP32)
    try:
        spp = G.gksl_min_stable_steps(ctx)
        D = d.N * d.N - 1
        nst = 70   # one 64-step graph chunk plus a remainder
        out = run_gpu(G, ctx, spp, nst, nst, D=D)
        info = G.gksl_get_info(ctx)
        assert info.rk4_variant[0] == int(variant)
        u = SYS.unfold_dimer(d)
        v_ref, _ = SYS.propagate_dimer(d, u, spp, nst)
        assert np.abs(out[0] - v_ref).max() < TOL64
        G.gksl_set_rho0(ctx, d.rho0_dense().real.copy())
        o32 = run_gpu(G, ctx, spp, nst, nst, precision=32, D=D)
        assert G.gksl_get_info(ctx).rk4_variant[1] == int(variant)
        assert np.abs(o32[0] - v_ref).max() < TOL32_V
    finally:
        G.gksl_destroy(ctx)


def test_config4_n1000_fp64_steps(G, record):
    """Largest workload (N = 1000, D = 999999) in the launch configuration of the benchmark:
    a few FP64 steps at the stable step size against the oracle's RK4 on its own matrices."""
    d = W.dimer(1000)
    ctx = G.dimer_context(d, flags=G.GKSL_ASM_FP32)
    try:
        spp = G.gksl_min_stable_steps(ctx)
        D = d.N * d.N - 1
        nst = 6
        out = run_gpu(G, ctx, spp, nst, nst, D=D)
        u = SYS.unfold_dimer(d)
        v_ref, _ = SYS.propagate_dimer(d, u, spp, nst)
        record("fp64_max_abs_dv_vs_oracle", np.abs(out[0] - v_ref).max())
        assert np.abs(out[0] - v_ref).max() < TOL64
        G.gksl_set_rho0(ctx, d.rho0_dense().real.copy())
        o32 = run_gpu(G, ctx, spp, nst, nst, precision=32, corr=0, D=D)
        record("fp32_max_abs_dv_vs_oracle", np.abs(o32[0] - v_ref).max())
        assert np.abs(o32[0] - v_ref).max() < TOL32_V
    finally:
        G.gksl_destroy(ctx)


def _oracle_system(H0, H1, Ls, gammas):
    """(Q0, Q1, K) by the definition Tr(F_s L(F_m)) on dense matrices (Q1 = 0 without H1)."""
    N = H0.shape[0]
    Q0, K = OL.unfold_dense(H0, Ls, gammas)
    Q1 = OL.unfold_dense(H1)[0] if H1 is not None else np.zeros_like(Q0)
    return Q0, Q1, K


def test_smallest_and_degenerate_systems(G):
    """N = 2 (D = 3: one S, one J, one D generator) with a drive and a decay channel; N = 3 with
    no drive operator and no dissipator (pure Hamiltonian: |v| conserved up to RK4's h^5 loss);
    and zero steps, which leave state and time as they were."""
    # qubit: H0 = (w0/2) sz, H1 = sx, L = sigma_minus at rate 0.2
    w0, E, A, omega, gam = 1.7, 0.1, 0.5, 1.3, 0.2
    H0 = np.diag([0.5 * w0, -0.5 * w0]).astype(complex)
    H1 = np.array([[0, 1], [1, 0]], dtype=complex)
    L = np.array([[0, 1], [0, 0]], dtype=complex)
    rho0 = np.array([[0.3, 0.2 - 0.1j], [0.2 + 0.1j, 0.7]])
    ctx = G.gksl_create(2)
    try:
        G.set_csr_operator(G.gksl_set_h0_component, ctx, 0, 1.0, op=W.CSR.from_dense(H0))
        G.set_csr_operator(G.gksl_set_h1, ctx, op=W.CSR.from_dense(H1))
        G.set_csr_operator(G.gksl_set_dissipator, ctx, 0, gam, op=W.CSR.from_dense(L))
        G.gksl_set_drive(ctx, E, A, omega)
        G.gksl_assemble(ctx, G.GKSL_ASM_FP32)
        G.gksl_set_rho0(ctx, rho0.real.copy(), rho0.imag.copy())
        spp, n, emit = 100, 250, 50
        # zero steps: nothing moves
        v_before = np.zeros(3)
        t_before = G.gksl_get_state(ctx, v_before)
        G.gksl_propagate(ctx, spp, 0, 64, 0, 0, None)
        v_after = np.zeros(3)
        assert G.gksl_get_state(ctx, v_after) == t_before
        assert np.array_equal(v_before, v_after)
        out = run_gpu(G, ctx, spp, n, emit, D=3)
        Q0, Q1, K = _oracle_system(H0, H1, [L], [gam])
        h = 2 * np.pi / omega / spp
        _, ref = OP.rk4(Q0, Q1, K, OP.eps_fn(E, A, omega), OB.expand(rho0).real, h, n, emit_every=emit)
        assert max(np.abs(out[i] - ref[i]).max() for i in range(len(ref))) < TOL64
    finally:
        G.gksl_destroy(ctx)
    # N = 3, Hamiltonian only, no H1
    H = W.random_operator(3, 0.8, 33, hermitian=True)
    rho0 = np.diag([0.5, 0.3, 0.2]).astype(complex)
    rho0[0, 1] = rho0[1, 0] = 0.1
    ctx = G.gksl_create(3)
    try:
        G.set_csr_operator(G.gksl_set_h0_component, ctx, 0, 1.0, op=H)
        G.gksl_set_drive(ctx, 0.0, 0.0, 1.0)
        G.gksl_assemble(ctx, 0)
        G.gksl_set_rho0(ctx, rho0.real.copy(), rho0.imag.copy())
        spp, n = 400, 800
        out = run_gpu(G, ctx, spp, n, n, D=8)
        Q0, Q1, K = _oracle_system(H.to_dense(), None, [], [])
        v0 = OB.expand(rho0).real
        h = 2 * np.pi / spp
        vref, _ = OP.rk4(Q0, Q1, K, OP.eps_fn(0.0, 0.0, 1.0), v0, h, n)
        assert np.abs(out[0] - vref).max() < TOL64
        # Q0 is skew (unitary evolution): each eigenmode of frequency y/h shrinks by |R(iy)| per
        # step with |R(iy)|^2 = 1 - y^6/72 + y^8/576 (RK4's stability function on the imaginary
        # axis), so |v0| |R(i h rho)|^n <= |v(t)| <= |v0| with rho the largest |eigenvalue|
        y = h * np.abs(np.linalg.eigvals(Q0)).max()
        shrink = np.sqrt(1 - y ** 6 / 72 + y ** 8 / 576) ** n
        nv, n0 = np.linalg.norm(out[0]), np.linalg.norm(v0)
        assert n0 * shrink - 1e-13 <= nv <= n0 + 1e-13, (nv, n0, shrink)
    finally:
        G.gksl_destroy(ctx)


def test_compact_columns_match_wide(G):
    """16-bit stage columns (the default once Q1 is folded) against 32-bit columns
    (GKSL_ASM_WIDE_COLUMNS): the same stored entries in the same slot order and the same
    arithmetic, so every stage-kernel variant gives bit-identical states in both precisions.  At
    N = 200 some short rows reach a column farther than 16383 from both the row and its S/J
    partner and take the 32-bit path inside the 16-bit form."""
    import os
    d = W.dimer(200)
    D = d.N * d.N - 1
    spp, n = 20000, 120
    outs = {}
    for wide in (False, True):
        flags = G.GKSL_ASM_FP32 | (G.GKSL_ASM_WIDE_COLUMNS if wide else 0)
        ctx = G.dimer_context(d, flags=flags)
        try:
            info = G.gksl_get_info(ctx)
            assert info.q1_folded == 1
            assert list(info.compact_columns) == ([0, 0] if wide else [1, 1])
            assert wide or 0 < info.compact_escaped_rows < D // 8
            for var in ("0", "1", "2", "3"):
                os.environ["GKSL_RK4_VARIANT"] = var
                try:
                    for prec in (64, 32):
                        G.gksl_set_rho0(ctx, d.rho0_dense().real.copy())
                        outs[(wide, var, prec)] = run_gpu(G, ctx, spp, n, n, precision=prec, D=D)[0]
                        used = G.gksl_get_info(ctx).rk4_compact[0 if prec == 64 else 1]
                        assert used == (0 if wide or var == "2" else 1)
                finally:
                    del os.environ["GKSL_RK4_VARIANT"]
                G.gksl_assemble(ctx, flags)
            if not wide:
                # the 32-bit columns forced on a context that has the 16-bit ones
                os.environ["GKSL_RK4_VARIANT"], os.environ["GKSL_RK4_COLUMNS"] = "0", "32"
                try:
                    G.gksl_set_rho0(ctx, d.rho0_dense().real.copy())
                    outs[(True, "0f", 64)] = run_gpu(G, ctx, spp, n, n, precision=64, D=D)[0]
                    assert G.gksl_get_info(ctx).rk4_compact[0] == 0
                finally:
                    del os.environ["GKSL_RK4_VARIANT"], os.environ["GKSL_RK4_COLUMNS"]
                # no override: the first propagation times every variant with both column widths
                G.gksl_assemble(ctx, flags)
                G.gksl_set_rho0(ctx, d.rho0_dense().real.copy())
                run_gpu(G, ctx, spp, 8, 8, precision=64, D=D)
                info = G.gksl_get_info(ctx)
                assert all(info.rk4_variant_us[0][v] > 0 for v in range(4))
                assert [info.rk4_variant_us_c16[0][v] > 0 for v in range(4)] == [True, True, False, True]
                # reassembled with 32-bit columns only: the copy and its escape list are gone
                G.gksl_assemble(ctx, flags | G.GKSL_ASM_WIDE_COLUMNS)
                info2 = G.gksl_get_info(ctx)
                assert list(info2.compact_columns) == [0, 0] and info2.compact_escaped_rows == 0
                assert info2.device_bytes < info.device_bytes
        finally:
            G.gksl_destroy(ctx)
    assert np.array_equal(outs[(True, "0f", 64)], outs[(True, "0", 64)])
    for var in ("0", "1", "2", "3"):
        for prec in (64, 32):
            a, b = outs[(False, var, prec)], outs[(True, var, prec)]
            assert np.isfinite(a).all() and np.abs(a).max() > 0
            assert np.array_equal(a, b), (var, prec, np.abs(a - b).max())


def test_compact_columns_dropped_for_nonlocal_operators(G):
    """A random sparse H0 at N = 260 couples pairs (j, k) to pairs far away in the basis (about
    4 rows in 10 reach a column beyond 16383 of both the row and its S/J partner), so assembly
    keeps Q1 folded but builds no 16-bit copy, and propagation gives the same states as with
    GKSL_ASM_WIDE_COLUMNS."""
    N = 260
    D = N * N - 1
    H0 = W.random_operator(N, 0.005, 41, hermitian=True)
    H1 = W.CSR.from_dense(np.diag(np.linspace(-1.0, 1.0, N)).astype(complex))
    outs = {}
    for flags in (G.GKSL_ASM_FP32, G.GKSL_ASM_FP32 | G.GKSL_ASM_WIDE_COLUMNS):
        ctx = G.gksl_create(N)
        try:
            G.set_csr_operator(G.gksl_set_h0_component, ctx, 0, 1.0, op=H0)
            G.set_csr_operator(G.gksl_set_h1, ctx, op=H1)
            G.gksl_set_drive(ctx, 0.5, 0.5, 1.0)
            G.gksl_assemble(ctx, flags)
            info = G.gksl_get_info(ctx)
            assert info.q1_folded == 1
            assert list(info.compact_columns) == [0, 0] and info.compact_escaped_rows == 0
            spp = G.gksl_min_stable_steps(ctx)
            rho0 = np.zeros((N, N))
            rho0[0, 0] = 1.0
            for prec in (64, 32):
                G.gksl_set_rho0(ctx, rho0.copy())
                outs[(flags, prec)] = run_gpu(G, ctx, spp, 40, 40, precision=prec, D=D)[0]
                assert G.gksl_get_info(ctx).rk4_compact[0 if prec == 64 else 1] == 0
        finally:
            G.gksl_destroy(ctx)
    for prec in (64, 32):
        a, b = outs[(G.GKSL_ASM_FP32, prec)], outs[(G.GKSL_ASM_FP32 | G.GKSL_ASM_WIDE_COLUMNS, prec)]
        assert np.isfinite(a).all() and np.abs(a).max() > 0
        assert np.array_equal(a, b)


def test_folded_q1_matches_separate_stream(G):
    """Q1 folded into the propagation format (the default for the dimer, whose H1 is diagonal)
    against Q1 as a separate stream (GKSL_ASM_NO_FOLD): the same RK4 map up to rounding, in
    every stage-kernel variant and both precisions; general operators do not fold."""
    import os
    d = W.dimer(60)
    D = d.N * d.N - 1
    spp, n = 2000, 300
    outs = {}
    for flags in (G.GKSL_ASM_FP32, G.GKSL_ASM_FP32 | G.GKSL_ASM_NO_FOLD):
        ctx = G.dimer_context(d, flags=flags)
        try:
            assert G.gksl_get_info(ctx).q1_folded == (0 if flags & G.GKSL_ASM_NO_FOLD else 1)
            for var in ("0", "1", "2", "3"):
                os.environ["GKSL_RK4_VARIANT"] = var
                try:
                    for prec in (64, 32):
                        G.gksl_set_rho0(ctx, d.rho0_dense().real.copy())
                        outs[(flags, var, prec)] = run_gpu(G, ctx, spp, n, n, precision=prec, D=D)[0]
                finally:
                    del os.environ["GKSL_RK4_VARIANT"]
                G.gksl_assemble(ctx, flags)   # a new assembly times/chooses the variant again
        finally:
            G.gksl_destroy(ctx)
    ref = outs[(G.GKSL_ASM_FP32 | G.GKSL_ASM_NO_FOLD, "0", 64)]
    for (flags, var, prec), v in outs.items():
        tol = 1e-12 if prec == 64 else 1e-5
        assert np.abs(v - ref).max() < tol, (flags, var, prec, np.abs(v - ref).max())
    ctx = G.gksl_create(5)
    try:
        G.set_csr_operator(G.gksl_set_h0_component, ctx, 0, 1.0, op=W.random_operator(5, 0.6, 3, hermitian=True))
        G.set_csr_operator(G.gksl_set_h1, ctx, op=W.random_operator(5, 0.6, 4, hermitian=True))
        G.gksl_set_drive(ctx, 0.5, 0.5, 1.0)
        G.gksl_assemble(ctx, 0)
        assert G.gksl_get_info(ctx).q1_folded == 0
    finally:
        G.gksl_destroy(ctx)


@pytest.mark.parametrize("case", ["dimer6", "dimer10", "dimer24", "dimer64", "dimer10_nofold", "general7"])
def test_block_path_matches_stage_kernels(G, case, monkeypatch):
    """Small systems run a whole chunk of RK4 steps in one thread block with the state in shared
    memory (by default up to D + 1 = 256 rows in FP64 and 576 in FP32; GKSL_RK4_BLOCK=1 forces it
    wherever D + 1 <= 4096).  Each row is summed as in the stage kernels and updated by the same
    stage functions, so the states equal the stage kernels' (GKSL_RK4_BLOCK=0) bit for bit: the
    dimer with 18 ELL slots and Q1 folded (N = 6, 10, 24, and 64, the largest that fits), Q1 kept
    apart (GKSL_ASM_NO_FOLD), and a general system whose ELL width differs from 18 and whose long
    rows go to warps; both precisions, with the FP32 form's FP64 correction steps, over 300 steps
    emitted every 75 (chunks that are not multiples of the stage kernels' 64-step graphs)."""
    import os
    if case.startswith("dimer"):
        N = int(case[5:].split("_")[0])
        d = W.dimer(N)
        flags = G.GKSL_ASM_FP32 | (G.GKSL_ASM_NO_FOLD if case.endswith("nofold") else 0)
        make = lambda: G.dimer_context(d, flags=flags)
        rho = d.rho0_dense()
    else:
        N = 7
        H = W.random_operator(N, 0.6, 31, hermitian=True)
        H1 = W.random_operator(N, 0.4, 32, hermitian=True)
        L = W.random_operator(N, 0.5, 33)
        re, im = W.random_density_matrix(N, 2, 34)
        rho = re + 1j * im

        def make():
            ctx = G.gksl_create(N)
            G.set_csr_operator(G.gksl_set_h0_component, ctx, 0, 0.8, op=H)
            G.set_csr_operator(G.gksl_set_h1, ctx, op=H1)
            G.set_csr_operator(G.gksl_set_dissipator, ctx, 0, 0.1, op=L)
            G.gksl_set_drive(ctx, 0.2, 0.6, 1.5)
            G.gksl_assemble(ctx, G.GKSL_ASM_FP32)
            return ctx
    D = N * N - 1
    outs = {}
    for block in ("0", "1"):
        monkeypatch.setenv("GKSL_RK4_BLOCK", block)
        ctx = make()
        try:
            spp = G.gksl_min_stable_steps(ctx) * 2
            info = G.gksl_get_info(ctx)
            if case == "general7":
                assert info.ell_width_q0 != 18 and info.long_rows > 0
            for prec, corr in ((64, 0), (32, 0), (32, 100)):
                G.gksl_set_rho0(ctx, rho.real.copy(), rho.imag.copy())
                outs[(block, prec, corr)] = run_gpu(G, ctx, spp, 300, 75, precision=prec, corr=corr, D=D)
        finally:
            G.gksl_destroy(ctx)
    for key in ((64, 0), (32, 0), (32, 100)):
        a, b = outs[("0",) + key], outs[("1",) + key]
        assert np.isfinite(a).all() and np.abs(a).max() > 0
        assert np.array_equal(a, b), (key, np.abs(a - b).max())
