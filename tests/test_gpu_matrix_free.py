"""Parity of the matrix-free RK4 stages (GKSL_ASM_MATRIX_FREE) with the oracle.

The matrix-free form applies Q(t) v + K as Tr(F_s L_t(rho)) with banded operators, so its
references are the oracle's generator-basis RK4 (dimer) and the dense rho-space RK4 (random
banded operators); both are the same RK4 map in exact arithmetic.  Tolerances as for the CSR
path: FP64 1e-10 on v, FP32 bulk 1e-5 on v and 1e-4 on <n1 - n2>.
"""
import numpy as np
import pytest

from oracle import basis as OB
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


def mf_flags(G, fp32=False):
    return G.GKSL_ASM_MATRIX_FREE | (G.GKSL_ASM_FP32 if fp32 else 0)


def test_mf_config0_vs_oracle(G):
    """N = 10 dimer, 10 periods x 200 steps, v at every period end, on the tridiagonal real
    instantiation (one tile with a ragged edge)."""
    d = W.dimer(10)
    ctx = G.dimer_context(d, flags=mf_flags(G))
    try:
        out = np.zeros((10, 99))
        G.gksl_propagate(ctx, 200, 2000, 64, 0, 200, out)
        u = SYS.unfold_dimer(d)
        _, ref = SYS.propagate_dimer(d, u, 200, 2000, emit_every=200)
        assert max(np.abs(out[i] - ref[i]).max() for i in range(10)) < TOL64
    finally:
        G.gksl_destroy(ctx)


@pytest.mark.parametrize("N", [2, 5, 33, 70])
def test_mf_random_banded_vs_rho_rk4(G, N):
    """Complex banded H0 (two components), H1 and three traceful non-Hermitian channels on the
    general instantiation, FP64 and FP32: N = 33 and 70 span several 32 x 32 tiles with ragged
    edges."""
    H0a = W.random_banded(N, 3, 100 + N, hermitian=True)
    H0b = W.random_banded(N, 1, 200 + N, hermitian=True)
    H1 = W.random_banded(N, 2, 300 + N, hermitian=True)
    Ls = [W.random_banded(N, b, 400 + 10 * N + b) for b in (0, 2, 4)]
    gam = [0.05, 0.1, 0.02]
    ctx = G.gksl_create(N)
    try:
        G.set_csr_operator(G.gksl_set_h0_component, ctx, 0, 0.3, op=H0a)
        G.set_csr_operator(G.gksl_set_h0_component, ctx, 4, -0.2, op=H0b)
        G.set_csr_operator(G.gksl_set_h1, ctx, op=H1)
        for p, (L, g) in enumerate(zip(Ls, gam)):
            G.set_csr_operator(G.gksl_set_dissipator, ctx, 2 * p, g, op=L)
        G.gksl_set_drive(ctx, 0.2, 0.7, 2.0)
        G.gksl_assemble(ctx, mf_flags(G, fp32=True))
        rng = np.random.default_rng(N)
        X = rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))
        rho0 = X @ X.conj().T
        rho0 /= np.trace(rho0)
        G.gksl_set_rho0(ctx, rho0.real.copy(), rho0.imag.copy())
        spp, n = 2000, 300
        D = N * N - 1
        out = np.zeros((1, D))
        G.gksl_propagate(ctx, spp, n, 64, 0, n, out)
        h = 2 * np.pi / 2.0 / spp
        rho = OP.rho_rk4(0.3 * H0a.to_dense() - 0.2 * H0b.to_dense(), H1.to_dense(), [L.to_dense() for L in Ls],
                         gam, OP.eps_fn(0.2, 0.7, 2.0), rho0, h, n)
        ref = OB.expand(rho).real
        assert np.abs(out[0] - ref).max() < TOL64
        G.gksl_set_rho0(ctx, rho0.real.copy(), rho0.imag.copy())
        G.gksl_propagate(ctx, spp, n, 32, 0, n, out)
        assert np.abs(out[0] - ref).max() < TOL32_V
    finally:
        G.gksl_destroy(ctx)


def test_mf_config1_n100_fp64_and_fp32(G):
    """N = 100 dimer at 4000 steps/period: FP64 against the oracle over a quarter period, the
    FP32 bulk form (FP64 step every period) against FP64 over two periods."""
    d = W.dimer(100)
    ctx = G.dimer_context(d, flags=mf_flags(G, fp32=True))
    try:
        D = d.N * d.N - 1
        spp = 4000
        out = np.zeros((2, D))
        G.gksl_propagate(ctx, spp, 1000, 64, 0, 500, out)
        u = SYS.unfold_dimer(d)
        _, ref = SYS.propagate_dimer(d, u, spp, 1000, emit_every=500)
        assert max(np.abs(out[i] - ref[i]).max() for i in range(2)) < TOL64
        G.gksl_set_rho0(ctx, d.rho0_dense().real.copy())
        v64 = np.zeros((2, D))
        G.gksl_propagate(ctx, spp, 2 * spp, 64, 0, spp, v64)
        G.gksl_set_rho0(ctx, d.rho0_dense().real.copy())
        v32 = np.zeros((2, D))
        G.gksl_propagate(ctx, spp, 2 * spp, 32, spp, spp, v32)
        assert np.abs(v32 - v64).max() < TOL32_V
        o64, o32 = np.zeros(2), np.zeros(2)
        G.gksl_observable_diag(ctx, d.obs_diag, v64, 2, o64)
        G.gksl_observable_diag(ctx, d.obs_diag, v32, 2, o32)
        assert np.abs(o32 - o64).max() < TOL32_O
    finally:
        G.gksl_destroy(ctx)


def test_mf_square_drive_vs_oracle(G):
    """Square drive theta = +-1 on the N = 10 dimer over 3 periods, matrix-free FP64."""
    d = W.dimer(10)
    ctx = G.dimer_context(d, flags=mf_flags(G))
    try:
        G.gksl_set_drive_shape(ctx, 1)
        out = np.zeros((3, 99))
        G.gksl_propagate(ctx, 400, 1200, 64, 0, 400, out)
        u = SYS.unfold_dimer(d)
        _, ref = SYS.propagate_dimer(d, u, 400, 1200, emit_every=400, drive="square")
        assert max(np.abs(out[i] - ref[i]).max() for i in range(3)) < TOL64
    finally:
        G.gksl_destroy(ctx)


def test_mf_n1000_vs_csr_sampled(G):
    """N = 1000 dimer (D = 999 999, 528 tiles) at the stable step size: 64 matrix-free FP64 steps
    against the oracle's generator-basis RK4 from the same state, compared on every entry."""
    d = W.dimer(1000)
    ctx = G.dimer_context(d, flags=mf_flags(G, fp32=True))
    try:
        spp = G.gksl_min_stable_steps(ctx)
        D = d.N * d.N - 1
        out = np.zeros((1, D))
        G.gksl_propagate(ctx, spp, 64, 64, 0, 64, out)
        u = SYS.unfold_dimer(d)
        _, ref = SYS.propagate_dimer(d, u, spp, 64, emit_every=64)
        assert np.abs(out[0] - ref[0]).max() < TOL64
        info = G.gksl_get_info(ctx)
        assert info.nnz_q0 == 0 and info.device_bytes < 200e6
    finally:
        G.gksl_destroy(ctx)


def test_mf_errors(G):
    """Operators wider than the band limit, MATRIX_FREE with TRANSPOSE, and CSR getters."""
    N = 20
    ctx = G.gksl_create(N)
    try:
        G.set_csr_operator(G.gksl_set_h0_component, ctx, 0, 1.0, op=W.random_banded(N, 5, 1, hermitian=True))
        G.gksl_set_drive(ctx, 0.0, 0.0, 1.0)
        with pytest.raises(G.GkslError):
            G.gksl_assemble(ctx, G.GKSL_ASM_MATRIX_FREE)
        G.set_csr_operator(G.gksl_set_h0_component, ctx, 0, 1.0, op=W.random_banded(N, 4, 1, hermitian=True))
        with pytest.raises(G.GkslError):
            G.gksl_assemble(ctx, G.GKSL_ASM_MATRIX_FREE | G.GKSL_ASM_TRANSPOSE)
        G.gksl_assemble(ctx, G.GKSL_ASM_MATRIX_FREE)
        with pytest.raises(G.GkslError):
            G.gksl_get_csr(ctx, G.GKSL_MAT_Q0)
        with pytest.raises(G.GkslError):
            G.gksl_get_k(ctx, np.zeros(N * N - 1))
        G.gksl_assemble(ctx, 0)   # the CSR form again on the same context
        assert G.gksl_get_csr(ctx, G.GKSL_MAT_Q0) > 0
    finally:
        G.gksl_destroy(ctx)
