"""Adjoint gradient of the period-averaged <n1 - n2> against the oracle's discrete adjoint and
against central finite differences of the GPU's own forward loss."""
import numpy as np
import pytest

from oracle import propagate as OP
from oracle import system as SYS
from paper_1812_11626_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1812_11626_gb300 import gksl
    return gksl


def oracle_grad(d, S, period):
    """[d/dA, d/d(rate), d/dJ, d/dU] of the oracle's discrete adjoint."""
    u = SYS.unfold_dimer(d)
    p = d.params
    h = 2 * np.pi / p["omega"] / S
    w, c0 = OP.observable_weights(d.obs_diag)
    v0 = SYS.initial_v(d)
    Q0 = u.q0(p["J"], p["U"], d.rate)
    sinw = lambda t: np.sin(p["omega"] * t)
    return OP.timeavg_adjoint(Q0, u.Q1, d.rate * u.K1, OP.eps_fn(p["E"], p["A"], p["omega"]), v0, w, c0, h, S,
                              period, dQ0=[None, u.R1, u.QJ, u.QU], dQ1=[(u.Q1, sinw), None, None, None],
                              dK=[None, u.K1, None, None])


# forms of the reverse stage: the library's choice (FP32: all of a row's stacked channel slots
# loaded at once and summed in float; FP64, small systems: the four channels' first slots loaded
# together), one row per thread channel by channel, the latter with the first slots together, and
# the wide form in both precisions
FORMS = {"auto": {}, "rows": {"GKSL_ADJ_WIDE": "0", "GKSL_ADJ_PIPE": "0"},
         "rows-pipe": {"GKSL_ADJ_WIDE": "0", "GKSL_ADJ_PIPE": "1"}, "wide": {"GKSL_ADJ_WIDE": "1"}}


def set_form(monkeypatch, form):
    for k, v in FORMS[form].items():
        monkeypatch.setenv(k, v)


@pytest.mark.parametrize("form", list(FORMS))
@pytest.mark.parametrize("precision,tol", [(64, 1e-9), (32, 1e-5)])
def test_adjoint_vs_oracle(G, precision, tol, record, form, monkeypatch):
    """N = 6 over 3 periods against the oracle's discrete adjoint, in every form of the reverse
    stage."""
    set_form(monkeypatch, form)
    d = W.dimer(6)
    S, period = 60, 3
    ctx = G.dimer_context(d)
    try:
        grad = np.zeros(4)   # [A, rate (gamma_0), J (theta_0), U (theta_1)]
        loss = G.gksl_adjoint_timeavg(ctx, d.obs_diag, S, period, precision, grad)
        L, g = oracle_grad(d, S, period)
        record("loss_abs_diff_vs_oracle", abs(loss - L))
        assert abs(loss - L) < (1e-11 if precision == 64 else 1e-4)
        scale = np.abs(g).max()
        record("grad_max_abs_diff_vs_oracle_over_max", np.abs(grad - g).max() / scale)
        assert np.abs(grad - g).max() < tol * scale, (grad, g)
        # the state is left unchanged
        v = np.zeros(d.N * d.N - 1)
        assert G.gksl_get_state(ctx, v) == 0.0
        assert np.abs(v - SYS.initial_v(d)).max() < 1e-15
    finally:
        G.gksl_destroy(ctx)


def test_adjoint_vs_finite_differences(G):
    """Central differences (h = 1e-6) of the GPU's FP64 forward loss; relative 1e-6."""
    d = W.dimer(8)
    S, period = 120, 2
    ctx = G.dimer_context(d)
    try:
        grad = np.zeros(4)
        G.gksl_adjoint_timeavg(ctx, d.obs_diag, S, period, 64, grad)
        p = d.params
        base = dict(A=p["A"], rate=d.rate, J=p["J"], U=p["U"])

        def loss(th):
            G.gksl_set_drive(ctx, p["E"], th["A"], p["omega"])
            G.gksl_set_gamma(ctx, 0, th["rate"])
            G.gksl_set_theta(ctx, 0, th["J"])
            G.gksl_set_theta(ctx, 1, th["U"])
            G.gksl_assemble(ctx, G.GKSL_ASM_FP32 | G.GKSL_ASM_TRANSPOSE)
            g = np.zeros(4)
            return G.gksl_adjoint_timeavg(ctx, d.obs_diag, S, period, 64, g)

        for i, key in enumerate(["A", "rate", "J", "U"]):
            hfd = 1e-6 * max(1.0, abs(base[key]))
            tp = dict(base); tp[key] += hfd
            tm = dict(base); tm[key] -= hfd
            fd = (loss(tp) - loss(tm)) / (2 * hfd)
            assert abs(fd - grad[i]) <= 1e-6 * max(abs(grad[i]), 1e-3 * np.abs(grad).max()), (key, fd, grad[i])
    finally:
        G.gksl_destroy(ctx)


def test_adjoint_n200_stable_steps_vs_finite_differences(G):
    """The adjoint workload's size (N = 200, D = 39 999) at its stable step count: every component
    of the gradient of the mean of <n1 - n2> over period 1 against central differences
    (h = 1e-6 relative) of the GPU's own FP64 loss.  Bound: 1e-6 of the gradient's largest
    component plus the differences' own rounding, 1e-13 |L| / h (the loss is O(N) while single
    components can be 1e-6 of it, so a per-component relative bound would test the rounding)."""
    d = W.dimer(200)
    ctx = G.dimer_context(d)
    try:
        S = G.gksl_min_stable_steps(ctx)
        grad = np.zeros(4)
        L0 = G.gksl_adjoint_timeavg(ctx, d.obs_diag, S, 1, 64, grad)
        p = d.params
        base = dict(A=p["A"], rate=d.rate, J=p["J"], U=p["U"])

        def loss(th):
            G.gksl_set_drive(ctx, p["E"], th["A"], p["omega"])
            G.gksl_set_gamma(ctx, 0, th["rate"])
            G.gksl_set_theta(ctx, 0, th["J"])
            G.gksl_set_theta(ctx, 1, th["U"])
            G.gksl_assemble(ctx, G.GKSL_ASM_FP32 | G.GKSL_ASM_TRANSPOSE)
            return G.gksl_adjoint_timeavg(ctx, d.obs_diag, S, 1, 64, np.zeros(4))

        gmax = np.abs(grad).max()
        for i, key in enumerate(["A", "rate", "J", "U"]):
            hfd = 1e-6 * abs(base[key])
            tp = dict(base); tp[key] += hfd
            tm = dict(base); tm[key] -= hfd
            fd = (loss(tp) - loss(tm)) / (2 * hfd)
            bound = 1e-6 * gmax + 1e-13 * abs(L0) / hfd
            assert abs(fd - grad[i]) <= bound, (key, fd, grad[i], bound)
    finally:
        G.gksl_destroy(ctx)


def test_adjoint_workload_period20_vs_finite_differences(G, record):
    """The adjoint workload at full size: N = 200 (D = 39 999), loss = mean of <n1 - n2> over
    period 20 at the stable step count (20 x 13 906 RK4 steps).  The FP64 adjoint's loss equals
    the forward loss; its gradient with respect to (A, gamma, J, U) matches central differences
    (h = 1e-6 relative) of that forward loss, computed from every grid point of period 20 emitted
    to device memory and reduced by the library's observable kernel; the FP32 adjoint stays
    within 1e-4 of each FP64 component (plus 1e-6 of the largest)."""
    import torch
    d = W.dimer(200)
    P = 20
    D = d.N * d.N - 1
    rho0 = d.rho0_dense()
    ctx = G.dimer_context(d)
    try:
        S = G.gksl_min_stable_steps(ctx)
        grad, grad32 = np.zeros(4), np.zeros(4)
        L_adj = G.gksl_adjoint_timeavg(ctx, d.obs_diag, S, P, 64, grad)
        G.gksl_adjoint_timeavg(ctx, d.obs_diag, S, P, 32, grad32)
        dev = torch.device("cuda", 0)
        buf = torch.empty((S + 1) * D, dtype=torch.float64, device=dev)
        obs = torch.empty(S + 1, dtype=torch.float64, device=dev)
        wt = np.full(S + 1, 1.0 / S)
        wt[0] = wt[S] = 0.5 / S
        wt = torch.as_tensor(wt, device=dev)

        def forward_loss():
            G.gksl_set_rho0(ctx, rho0.real.copy(), rho0.imag.copy())
            G.gksl_propagate(ctx, S, (P - 1) * S, 64, 0, 0, None)
            G.gksl_get_state(ctx, buf[:D])
            G.gksl_propagate(ctx, S, S, 64, 0, 1, buf[D:])
            G.gksl_observable_diag(ctx, d.obs_diag, buf, S + 1, obs)
            torch.cuda.synchronize()
            return float((wt * obs).sum())

        L0 = forward_loss()
        record("loss_rel_diff_adjoint_vs_forward", abs(L0 - L_adj) / abs(L0))
        assert abs(L0 - L_adj) <= 1e-12 * abs(L0), (L0, L_adj)
        p = d.params
        base = dict(A=p["A"], rate=d.rate, J=p["J"], U=p["U"])

        def loss(th):
            G.gksl_set_drive(ctx, p["E"], th["A"], p["omega"])
            G.gksl_set_gamma(ctx, 0, th["rate"])
            G.gksl_set_theta(ctx, 0, th["J"])
            G.gksl_set_theta(ctx, 1, th["U"])
            G.gksl_assemble(ctx, G.GKSL_ASM_FP32 | G.GKSL_ASM_TRANSPOSE)
            return forward_loss()

        gmax = np.abs(grad).max()
        for i, key in enumerate(["A", "rate", "J", "U"]):
            hfd = 1e-6 * abs(base[key])
            tp = dict(base); tp[key] += hfd
            tm = dict(base); tm[key] -= hfd
            fd = (loss(tp) - loss(tm)) / (2 * hfd)
            bound = 1e-6 * gmax + 1e-13 * abs(L0) / hfd
            record(f"grad_{key}_rel_diff_vs_central_differences", abs(fd - grad[i]) / abs(grad[i]))
            assert abs(fd - grad[i]) <= bound, (key, fd, grad[i], bound)
        record("fp32_grad_max_rel_diff_vs_fp64", np.max(np.abs(grad32 - grad) / np.abs(grad)))
        assert np.all(np.abs(grad32 - grad) <= 1e-4 * np.abs(grad) + 1e-6 * gmax), (grad32, grad)
    finally:
        G.gksl_destroy(ctx)


def test_autograd_function(G):
    import torch
    d = W.dimer(5)
    ctx = G.dimer_context(d)
    try:
        p = d.params
        G.set_param_layout(ctx, p["A"], p["E"], p["omega"], channels=[0], components=[0, 1])
        fn = G.TimeAvgObservable.make(ctx, d.obs_diag, 40, 2, 64)
        theta = torch.tensor([p["A"], d.rate, p["J"], p["U"]], dtype=torch.float64, requires_grad=True)
        L = fn(theta)
        L.backward()
        ref = np.zeros(4)
        Lr = G.gksl_adjoint_timeavg(ctx, d.obs_diag, 40, 2, 64, ref)
        assert abs(L.item() - Lr) < 1e-14 and np.abs(theta.grad.numpy() - ref).max() < 1e-14
    finally:
        G.gksl_destroy(ctx)


@pytest.mark.parametrize("precision,tol", [(64, 1e-9), (32, 1e-5)])
def test_adjoint_ragged_segments_vs_oracle(G, precision, tol, record):
    """S = 66 steps per period: the reverse sweep's checkpoint segments do not divide S, so the
    last segment of every period is shorter than the others."""
    d = W.dimer(5)
    S, period = 66, 2
    ctx = G.dimer_context(d)
    try:
        grad = np.zeros(4)
        loss = G.gksl_adjoint_timeavg(ctx, d.obs_diag, S, period, precision, grad)
        L, g = oracle_grad(d, S, period)
        record("grad_max_abs_diff_vs_oracle_over_max", np.abs(grad - g).max() / np.abs(g).max())
        assert abs(loss - L) < (1e-11 if precision == 64 else 1e-4)
        assert np.abs(grad - g).max() < tol * np.abs(g).max(), (grad, g)
        # a second call on the same context gives the same result bit for bit
        grad2 = np.zeros(4)
        assert G.gksl_adjoint_timeavg(ctx, d.obs_diag, S, period, precision, grad2) == loss
        assert np.array_equal(grad, grad2)
    finally:
        G.gksl_destroy(ctx)


@pytest.mark.parametrize("precision,tol", [(64, 1e-9), (32, 1e-5)])
def test_adjoint_general_operators_vs_oracle(G, precision, tol, record):
    """Three H0 components, a drive operator and two dissipators (six gradient channels, more
    than the four-channel kernel holds), with gaps in the component and channel indices; the
    oracle side unfolds each operator by the definition Tr(F_s L(F_m)) on dense matrices."""
    from oracle import basis as OB
    from oracle import lindblad as LB
    N = 4
    Hs = [W.random_operator(N, 0.7, 80 + k, hermitian=True) for k in range(3)]
    H1 = W.random_operator(N, 0.6, 90, hermitian=True)
    Ls = [W.random_operator(N, 0.6, 91), W.random_operator(N, 0.6, 92)]
    theta, comps = [0.7, -0.4, 1.1], [0, 2, 5]
    gam, chans = [0.3, 0.15], [0, 3]
    E, A, omega = 0.3, 0.8, 2.0
    S, period = 42, 2
    o_diag = np.linspace(-1.0, 2.0, N)
    rho0 = np.diag(np.linspace(1, 3, N)).astype(complex)
    rho0 /= np.trace(rho0)
    rho0[0, 2] = 0.05 + 0.02j
    rho0[2, 0] = np.conj(rho0[0, 2])
    ctx = G.gksl_create(N)
    try:
        for k, th, H in zip(comps, theta, Hs):
            G.set_csr_operator(G.gksl_set_h0_component, ctx, k, th, op=H)
        G.set_csr_operator(G.gksl_set_h1, ctx, op=H1)
        for p, g, L in zip(chans, gam, Ls):
            G.set_csr_operator(G.gksl_set_dissipator, ctx, p, g, op=L)
        G.gksl_set_drive(ctx, E, A, omega)
        G.gksl_assemble(ctx, G.GKSL_ASM_FP32 | G.GKSL_ASM_TRANSPOSE)
        G.gksl_set_rho0(ctx, rho0.real.copy(), rho0.imag.copy())
        grad = np.zeros(6)   # [A, gamma_0, gamma_3, theta_0, theta_2, theta_5]
        loss = G.gksl_adjoint_timeavg(ctx, o_diag, S, period, precision, grad)
    finally:
        G.gksl_destroy(ctx)
    Z = np.zeros((N, N))
    Qk = [LB.unfold_dense(H.to_dense())[0] for H in Hs]
    Q1 = LB.unfold_dense(H1.to_dense())[0]
    RK = [LB.unfold_dense(Z, [L.to_dense()], [1.0]) for L in Ls]
    Q0 = sum(th * Q for th, Q in zip(theta, Qk)) + sum(g * R for g, (R, _) in zip(gam, RK))
    K = sum(g * Kp for g, (_, Kp) in zip(gam, RK))
    w, c0 = OP.observable_weights(o_diag)
    v0 = OB.expand(rho0).real
    h = 2 * np.pi / omega / S
    sinw = lambda t: np.sin(omega * t)
    L_ref, g_ref = OP.timeavg_adjoint(Q0, Q1, K, OP.eps_fn(E, A, omega), v0, w, c0, h, S, period,
                                      dQ0=[None, RK[0][0], RK[1][0]] + Qk, dQ1=[(Q1, sinw)] + [None] * 5,
                                      dK=[None, RK[0][1], RK[1][1]] + [None] * 3)
    record("grad_max_abs_diff_vs_oracle_over_max", np.abs(grad - g_ref).max() / np.abs(g_ref).max())
    assert abs(loss - L_ref) < (1e-11 if precision == 64 else 1e-4) * max(1.0, abs(L_ref))
    assert np.abs(grad - g_ref).max() < tol * np.abs(g_ref).max(), (grad, g_ref)


@pytest.mark.parametrize("N", [3, 6])
@pytest.mark.parametrize("form", ["auto", "rows", "wide"])
@pytest.mark.parametrize("precision,tol", [(64, 1e-9), (32, 1e-5)])
def test_adjoint_dense_four_channels_vs_oracle(G, N, precision, tol, record, form, monkeypatch):
    """Two dense H0 components, a dense drive operator and one dense traceful dissipator: four
    gradient channels whose rows hold up to D entries each.  At N = 3 (D = 8) the four channels'
    slots together fill the wide reverse stage's largest form (up to 32 stacked slots); at
    N = 6 (D = 35) they exceed it and the library keeps the channel-by-channel form."""
    from oracle import basis as OB
    from oracle import lindblad as LB
    set_form(monkeypatch, form)
    Hs = [W.random_operator(N, 1.0, 60 + k, hermitian=True) for k in range(2)]
    H1 = W.random_operator(N, 1.0, 62, hermitian=True)
    L = W.random_operator(N, 1.0, 63)
    theta, gam = [0.5, -0.8], 0.2
    E, A, omega = 0.2, 0.6, 3.0
    S, period = 120, 2
    o_diag = np.linspace(1.0, -1.0, N)
    rho0 = np.diag(np.linspace(2, 1, N)).astype(complex)
    rho0 /= np.trace(rho0)
    rho0[0, N - 1] = 0.03 - 0.04j
    rho0[N - 1, 0] = np.conj(rho0[0, N - 1])
    ctx = G.gksl_create(N)
    try:
        for k, (th, H) in enumerate(zip(theta, Hs)):
            G.set_csr_operator(G.gksl_set_h0_component, ctx, k, th, op=H)
        G.set_csr_operator(G.gksl_set_h1, ctx, op=H1)
        G.set_csr_operator(G.gksl_set_dissipator, ctx, 0, gam, op=L)
        G.gksl_set_drive(ctx, E, A, omega)
        G.gksl_assemble(ctx, G.GKSL_ASM_FP32 | G.GKSL_ASM_TRANSPOSE)
        assert G.gksl_min_stable_steps(ctx) <= S
        G.gksl_set_rho0(ctx, rho0.real.copy(), rho0.imag.copy())
        grad = np.zeros(4)   # [A, gamma_0, theta_0, theta_1]
        loss = G.gksl_adjoint_timeavg(ctx, o_diag, S, period, precision, grad)
    finally:
        G.gksl_destroy(ctx)
    Z = np.zeros((N, N))
    Qk = [LB.unfold_dense(H.to_dense())[0] for H in Hs]
    Q1 = LB.unfold_dense(H1.to_dense())[0]
    R, K = LB.unfold_dense(Z, [L.to_dense()], [1.0])
    Q0 = sum(th * Q for th, Q in zip(theta, Qk)) + gam * R
    w, c0 = OP.observable_weights(o_diag)
    v0 = OB.expand(rho0).real
    h = 2 * np.pi / omega / S
    sinw = lambda t: np.sin(omega * t)
    L_ref, g_ref = OP.timeavg_adjoint(Q0, Q1, gam * K, OP.eps_fn(E, A, omega), v0, w, c0, h, S, period,
                                      dQ0=[None, R] + Qk, dQ1=[(Q1, sinw), None, None, None],
                                      dK=[None, K, None, None])
    record("grad_max_abs_diff_vs_oracle_over_max", np.abs(grad - g_ref).max() / np.abs(g_ref).max())
    assert abs(loss - L_ref) < (1e-11 if precision == 64 else 1e-4) * max(1.0, abs(L_ref))
    assert np.abs(grad - g_ref).max() < tol * np.abs(g_ref).max(), (grad, g_ref)


@pytest.mark.parametrize("with_l", [False, True], ids=["h0_h1", "h0_h1_l"])
@pytest.mark.parametrize("form", ["auto", "rows", "wide"])
@pytest.mark.parametrize("precision,tol", [(64, 1e-9), (32, 1e-5)])
def test_adjoint_fewer_channels_vs_oracle(G, with_l, precision, tol, record, form, monkeypatch):
    """One H0 component and a drive operator, with and without one dissipator (two or three
    gradient channels, fewer than the four-channel kernels hold, and no K column without the
    dissipator) at N = 4, against the oracle's discrete adjoint in every form of the reverse stage."""
    from oracle import basis as OB
    from oracle import lindblad as LB
    set_form(monkeypatch, form)
    N = 4
    # rows of at most 5, 3 and 7 entries: 8 stacked slots without the dissipator (the smallest
    # wide form, full), 15 with it
    H = W.random_operator(N, 0.2, 70, hermitian=True)
    H1 = W.random_operator(N, 0.2, 71, hermitian=True)
    L = W.random_operator(N, 0.2, 72)
    theta, gam = 0.9, 0.25
    E, A, omega = 0.4, 0.7, 2.5
    S, period = 80, 2
    o_diag = np.linspace(0.5, -1.5, N)
    rho0 = np.diag(np.linspace(3, 1, N)).astype(complex)
    rho0 /= np.trace(rho0)
    rho0[1, 2] = 0.04 + 0.01j
    rho0[2, 1] = np.conj(rho0[1, 2])
    ctx = G.gksl_create(N)
    try:
        G.set_csr_operator(G.gksl_set_h0_component, ctx, 0, theta, op=H)
        G.set_csr_operator(G.gksl_set_h1, ctx, op=H1)
        if with_l:
            G.set_csr_operator(G.gksl_set_dissipator, ctx, 0, gam, op=L)
        G.gksl_set_drive(ctx, E, A, omega)
        G.gksl_assemble(ctx, G.GKSL_ASM_FP32 | G.GKSL_ASM_TRANSPOSE)
        assert G.gksl_min_stable_steps(ctx) <= S
        G.gksl_set_rho0(ctx, rho0.real.copy(), rho0.imag.copy())
        grad = np.zeros(3 if with_l else 2)   # [A, (gamma_0,) theta_0]
        loss = G.gksl_adjoint_timeavg(ctx, o_diag, S, period, precision, grad)
    finally:
        G.gksl_destroy(ctx)
    Z = np.zeros((N, N))
    Qh = LB.unfold_dense(H.to_dense())[0]
    Q1 = LB.unfold_dense(H1.to_dense())[0]
    D = N * N - 1
    if with_l:
        R, K = LB.unfold_dense(Z, [L.to_dense()], [1.0])
        Q0, Kv = theta * Qh + gam * R, gam * K
        dQ0, dK = [None, R, Qh], [None, K, None]
    else:
        Q0, Kv = theta * Qh, np.zeros(D)
        dQ0, dK = [None, Qh], [None, None]
    sinw = lambda t: np.sin(omega * t)
    dQ1 = [(Q1, sinw)] + [None] * (len(dQ0) - 1)
    w, c0 = OP.observable_weights(o_diag)
    v0 = OB.expand(rho0).real
    h = 2 * np.pi / omega / S
    L_ref, g_ref = OP.timeavg_adjoint(Q0, Q1, Kv, OP.eps_fn(E, A, omega), v0, w, c0, h, S, period,
                                      dQ0=dQ0, dQ1=dQ1, dK=dK)
    record("grad_max_abs_diff_vs_oracle_over_max", np.abs(grad - g_ref).max() / np.abs(g_ref).max())
    assert abs(loss - L_ref) < (1e-11 if precision == 64 else 1e-4) * max(1.0, abs(L_ref))
    assert np.abs(grad - g_ref).max() < tol * np.abs(g_ref).max(), (grad, g_ref)
